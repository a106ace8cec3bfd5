"""Benchmark: batched MDHP-GDS window fits per second on GB300.

One step = one complete batched fit (mdhp_fit_batch: length sort, validation,
staging, every projected-gradient iteration) of the 4,096-window workload:
M = 16 message IDs, counts log-uniform in [200, 5000], scalar beta fixed per
batch, 200 iterations, cold start, learning rate 1e-2.  Inputs are simulated
(Ogata thinning, seed 2024 + rank) and resident in HBM before timing; L2 is
flushed (256 MB write) before every timed step.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
checker instead (the reference arm of this method has no runnable code; the
checker is the slow, obviously-correct CPU program the library is compared
against), on a fixed sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MDHP window fits/s to fixed logL tol (warm vs cold); LL+grad events/s vs roofline"
# DRAM read + write of one fit of the default workload (4,096 windows x M=16,
# 200 iterations), from an ncu app-range capture of one --profile-step fit
# (summary under profiles/); to be re-taken whenever the fit kernels change
FIT_DRAM_BYTES_4096xM16 = 75271168 + 39822080
UNIT = "windows/s"
WORKLOAD = "4096 windows x M=16, counts log-uniform[200,5000], scalar beta=1 fixed, 200 PGD iterations (lr 1e-2), cold start"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--windows", type=int, default=4096)
    ap.add_argument("--iters", type=int, default=200)
    ap.add_argument("--beta", type=float, default=1.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", default="2", choices=["2", "3", "5", "6", "attack", "lstm"],
                    help="2: fixed-iteration fits (default line); 5: warm vs cold fits to tolerance")
    ap.add_argument("--tol", type=float, default=1e-5)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--clocks-dir", default=None,
                    help="folder for the raw nvidia-smi clock samples (default: the temp folder)")
    ap.add_argument("--attack-windows", type=int, default=128,
                    help="attacked (and as many normal) windows per combination (--workload attack)")
    ap.add_argument("--profile-step", action="store_true",
                    help="bracket the first timed step with cudaProfilerStart/Stop (for ncu "
                         "--replay-mode app-range: one fit's launches measured as one range)")
    ap.add_argument("--train-windows", type=int, default=65536)
    ap.add_argument("--train-steps", type=int, default=4000)
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per fit from an ncu capture (default: the committed "
                         "capture of the default workload)")
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, directory: str | None = None):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(directory or tempfile.gettempdir(), f"mdhp_clocks_gpu{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(sm_count: int, mhz: float) -> float:
    # 128 FP32 lanes per SM, one FMA (2 FLOP) per lane per clock
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


def flops_per_event_iter(M: int) -> int:
    """Algorithmic FP32 work of one event in one evaluation of the decoupled
    fixed-beta fit (features x_n = R(t_n) precomputed once per window):
    lambda = mu + alpha_u . x_n (2M), d/dalpha_u += r x_n (2M), plus the
    d/dmu sum, 1/lambda and the Kahan sum of ln lambda (8)."""
    return 4 * M + 8


def feature_bytes_per_event_iter(M: int) -> int:
    """Bytes of features each evaluation reads per event (float32 x_n)."""
    return 4 * M


WORKLOAD6 = ("4096 windows x M=16, counts log-uniform[200,5000], beta_ij matrix log-uniform[0.5,2] "
             "fixed, 200 PGD iterations (lr 1e-2), cold start")


def make_inputs(args, rank):
    from paper_2411_10258_gb300.workload import workload

    name = 6 if args.workload == '6' else 2
    bt = workload.make_workload(name, B=args.windows, seed=2024 + rank, beta=args.beta)
    return bt


def cpu_baseline(bt, args, seconds: float):
    """The FP64 checker as it stands on a bounded sample: OpenMP over windows."""
    from oracle import oracle

    ncores = len(os.sched_getaffinity(0))
    o = oracle.fit_opts(max_iters=args.iters, lr=1e-2)
    rng = np.random.default_rng(0)
    order = rng.permutation(bt.B)
    # size the sample from a short probe so that it takes ~`seconds`
    probe = bt.subset(order[: max(ncores, 8)])
    t0 = time.perf_counter()
    _fit_sample(oracle, probe, o, ncores)
    dt = time.perf_counter() - t0
    per_window = dt / probe.B
    n = int(min(bt.B, max(probe.B, seconds / max(per_window, 1e-6))))
    sample = bt.subset(order[:n])
    t0 = time.perf_counter()
    _fit_sample(oracle, sample, o, ncores)
    dt = time.perf_counter() - t0
    return {"value": sample.B / dt, "unit": UNIT, "cores": ncores, "kind": "oracle",
            "sample": f"{sample.B} random windows of the same workload, {args.iters} iterations each, "
                      f"FP64, OpenMP over windows on {ncores} threads ({dt:.1f} s)",
            "events": int(sample.n_events)}


def _fit_sample(oracle, bt, o, ncores):
    M = bt.M
    mu0 = np.zeros((bt.B, M))
    a0 = np.zeros((bt.B, M, M))
    for b in range(bt.B):
        t, ids, T, _ = bt.window(b)
        mu0[b], a0[b] = oracle.cold_init(ids, float(T), M, bt.beta[b])
    return oracle.fit_batch(bt.offsets, bt.t, bt.id, bt.T, M, bt.beta_mode, mu0, a0,
                            bt.beta.astype(np.float64), o, nthreads=ncores)


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    from oracle import oracle

    oracle.build()
    bt = make_inputs(args, 0)
    ncores = len(os.sched_getaffinity(0))
    o = oracle.fit_opts(max_iters=args.iters, lr=1e-2)
    rng = np.random.default_rng(1)
    per_step = max(ncores, 16)
    for _ in range(args.warmup):
        _fit_sample(oracle, bt.subset(rng.choice(bt.B, per_step, replace=False)), o, ncores)
    tot, n = 0.0, 0
    for _ in range(args.steps):
        s = bt.subset(rng.choice(bt.B, per_step, replace=False))
        t0 = time.perf_counter()
        _fit_sample(oracle, s, o, ncores)
        tot += time.perf_counter() - t0
        n += s.B
    v = n / tot
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "parallelism": "OpenMP over windows",
                       "l2": "not applicable (CPU)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": ncores, "kind": "oracle",
                             "sample": f"{per_step} random windows per step, {args.iters} iterations, FP64"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    rank, world, local = dist_info()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_2411_10258_gb300 import DeviceBatch, FitOptions, Plan, shard
    from paper_2411_10258_gb300 import build as libbuild

    if not os.path.exists(os.path.join(ROOT, "paper_2411_10258_gb300", "_build", "libmdhp.so")):
        libbuild.build()
    bt = make_inputs(args, rank)
    B, M = bt.B, bt.M
    max_ev = int(bt.counts.max())
    db = DeviceBatch.from_host(bt, dev)
    plan = Plan(M, bt.beta_mode, B, max_ev)
    opts = FitOptions(max_iters=args.iters, lr=1e-2, init=1)
    beta = torch.from_numpy(bt.beta.astype(np.float32)).to(dev)
    mu = torch.zeros(B, M, device=dev)
    alpha = torch.zeros(B, M, M, device=dev)
    out = {k: torch.empty(B, dtype=d, device=dev) for k, d in
           (("loglik", torch.float64), ("iters", torch.int32), ("status", torch.int32))}
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream()

    # launch shape chosen by the library's autotuner on this batch (untimed)
    tuned = plan.autotune(db, opts, mu, alpha, beta, tune_iters=20) if not args.no_autotune else None

    def step():
        plan.fit(db, opts, mu, alpha, beta, out=out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st = out["status"].cpu().numpy()
    bad = int(np.sum((st != 0)))
    plan.set_timing(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    kern_ms = []
    sampler = ClockSampler(local, args.clocks_dir)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with sampler:
        for i in range(args.steps):
            flush.fill_(float(i))
            if args.profile_step and i == 0:  # one step as a profiler range (ncu app-range replay)
                torch.cuda.synchronize()
                torch.cuda.cudart().cudaProfilerStart()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
            if args.profile_step and i == 0:
                torch.cuda.synchronize()
                torch.cuda.cudart().cudaProfilerStop()
            kern_ms.append(plan.last_fit_ms())
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = float(np.sum(step_ms))
    kern_avg = float(np.mean(kern_ms))
    tot_ms = shard.max_over_ranks(tot_ms, device=dev)  # whole-job time: the slowest rank
    value = world * B * args.steps / (tot_ms / 1000.0)
    events_iters = float(bt.n_events) * args.iters
    llg_events_per_s = events_iters / (kern_avg / 1000.0)

    # end to end through the public API: pinned host inputs -> fit -> host results
    e2e = e2e_run(args, bt, plan, opts, dev)

    peaks, src = measured_peaks()
    traffic = args.traffic
    if traffic is None and B == 4096 and M == 16 and args.iters == 200 and args.beta == 1.0 \
            and args.workload == '2':
        traffic = FIT_DRAM_BYTES_4096xM16
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = fp32_peak_tflops(sm_count, float(peaks.get("sm_max_mhz", 2070.0)))
    flops = events_iters * flops_per_event_iter(M)
    achieved = flops / (kern_avg / 1000.0) / 1e12
    clocks = sampler.summary()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD6 if args.workload == '6' else WORKLOAD,
                       "windows_per_gpu": B, "M": M,
                       "events_per_gpu": int(bt.n_events), "iterations": args.iters,
                       "parallelism": f"windows sharded over {world} GPU(s), no collective",
                       "l2": "flushed (256 MB write) before every timed step",
                       "autotuned": tuned},
            "llg_events_per_s": llg_events_per_s,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "traffic_note": "DRAM read+write bytes of one fit (both k_fit_x launches "
                                         "and the sort), ncu app-range capture; ncu serialises the "
                                         "two launches (summary under profiles/)",
                         "kernel": "k_fit_x: decoupled features, two concurrent launches sharing a "
                                   "length-sorted queue (256 threads/window from the front, 64 from "
                                   "the back)",
                         "peak_source": f"FP32 FMA: {sm_count} SMs x 128 lanes x 2 FLOP x "
                                        f"{peaks.get('sm_max_mhz', 2070.0)} MHz ({src} max clock)",
                         "flops_per_event_iteration": flops_per_event_iter(M),
                         "feature_bytes_per_event_iteration": feature_bytes_per_event_iter(M),
                         "feature_read_gbs": events_iters * feature_bytes_per_event_iter(M)
                                             / (kern_avg / 1000.0) / 1e9},
            "gpu_launches": plan.last_launches() * args.steps,
            "invalid_windows": bad,
            "clocks": clocks, "e2e": e2e}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(bt, args, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def e2e_run(args, bt, plan, opts, dev):
    """Same metric through the public API with host buffers: H2D of the batch
    from pinned memory, the fit, D2H of lnL and the fitted parameters."""
    import torch
    from paper_2411_10258_gb300 import DeviceBatch

    B, M = bt.B, bt.M
    host = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in
            (("offsets", bt.offsets), ("t", bt.t), ("id", bt.id), ("T", bt.T),
             ("beta", bt.beta.astype(np.float32)))}
    res_h = {"loglik": torch.empty(B, dtype=torch.float64).pin_memory(),
             "mu": torch.empty(B, M).pin_memory(),
             "alpha": torch.empty(B, M, M).pin_memory()}
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = sum(v.numel() * v.element_size() for v in res_h.values())
    dev_bufs = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
    mu = torch.empty(B, M, device=dev)
    alpha = torch.empty(B, M, M, device=dev)
    stream = torch.cuda.current_stream()

    def one():
        for k in dev_bufs:
            dev_bufs[k].copy_(host[k], non_blocking=True)
        db = DeviceBatch(M, bt.beta_mode, dev_bufs["offsets"], dev_bufs["t"], dev_bufs["id"], dev_bufs["T"],
                         None, int(bt.counts.max()))
        out = plan.fit(db, opts, mu, alpha, dev_bufs["beta"])
        res_h["loglik"].copy_(out["loglik"], non_blocking=True)
        res_h["mu"].copy_(mu, non_blocking=True)
        res_h["alpha"].copy_(alpha, non_blocking=True)

    one()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = max(1, min(args.steps, 3))
    e0.record(stream)
    for _ in range(n):
        one()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    return {"value": B / (ms / 1000.0), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": n}


def flops_per_event_iter_learned(M: int) -> int:
    """Algorithmic FP32 work of one event in one evaluation with beta learned
    per source (event recursion, nothing hoisted): per source the decay
    2^(-beta dt log2 e) (range reduction + degree-7 polynomial + scaling, 10),
    the R and S updates (3), the lambda dot (2), d/dalpha (2) and d/dbeta (2)."""
    return 19 * M


def run_long_learned(args):
    """Workload 3: 512 windows, M = 64, counts log-uniform [2e4, 1e5], beta per
    source learned by projected Adam (lr 1e-2) from the generating beta,
    `--iters` iterations, cold start of mu and alpha.  Windows simulated by the
    library's GPU simulator.  value = windows/s."""
    import torch

    from paper_2411_10258_gb300 import FitOptions, Plan, simulate
    from paper_2411_10258_gb300.workload import workload

    dev = torch.device("cuda", 0)
    p = workload.make_params(3, B=512, seed=2024)
    db, sst = simulate(64, 1, p["mu"], p["alpha"], p["beta"], p["counts"], seed=2024, stream_id=3)
    if int((sst != 0).sum().item()):
        raise RuntimeError("simulation failed")
    B, M = db.B, 64
    beta0 = torch.from_numpy(p["beta"]).float().to(dev)
    plan = Plan(M, 1, B, 0)
    opts = FitOptions(optimizer=1, max_iters=args.iters, lr=1e-2, init=1, fit_beta=1)
    mu = torch.zeros(B, M, device=dev)
    al = torch.zeros(B, M, M, device=dev)
    be = beta0.clone()
    out = None
    for _ in range(args.warmup):
        out = plan.fit(db, opts, mu, al, be.copy_(beta0))
    torch.cuda.synchronize()
    plan.set_timing(True)
    ms = []
    sampler = ClockSampler(0, args.clocks_dir)
    with sampler:
        for _ in range(args.steps):
            out = plan.fit(db, opts, mu, al, be.copy_(beta0))
            ms.append(plan.last_fit_ms())
        torch.cuda.synchronize()
    avg = float(np.mean(ms))
    ev_it = float(p["counts"].sum()) * args.iters
    peaks, src = measured_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = fp32_peak_tflops(sm_count, float(peaks.get("sm_max_mhz", 2070.0)))
    achieved = ev_it * flops_per_event_iter_learned(M) / (avg / 1000.0) / 1e12
    line = {"metric": "MDHP window fits/s (beta learned per source)", "value": B / (avg / 1000.0),
            "unit": "windows/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": avg, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"512 windows x M=64, counts log-uniform[2e4,1e5] "
                                   f"({int(p['counts'].sum())} events), beta per source learned, "
                                   f"projected Adam lr 1e-2, {args.iters} iterations",
                       "shape": plan.shape()},
            "llg_events_per_s": ev_it / (avg / 1000.0),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "k_fit (event recursion, events streamed from device memory)",
                         "flops_per_event_iteration": flops_per_event_iter_learned(M),
                         "peak_source": f"FP32 FMA ({src} max clock)"},
            "gpu_launches": plan.last_launches() * args.steps,
            "invalid_windows": int((out["status"] != 0).sum().item()),
            "clocks": sampler.summary()}
    print(json.dumps(line), flush=True)


def _auc(pos, neg):
    """Area under the ROC curve of scores pos (attacked) vs neg (normal),
    by the Mann-Whitney rank sum (ties counted half)."""
    pos, neg = np.asarray(pos, dtype=np.float64), np.asarray(neg, dtype=np.float64)
    allv = np.concatenate([pos, neg])
    order = np.argsort(allv, kind="stable")
    ranks = np.empty(len(allv))
    ranks[order] = np.arange(1, len(allv) + 1)
    for v in np.unique(allv):  # average ranks of ties
        sel = allv == v
        if sel.sum() > 1:
            ranks[sel] = ranks[sel].mean()
    return float((ranks[:len(pos)].sum() - len(pos) * (len(pos) + 1) / 2) / (len(pos) * len(neg)))


def run_attacks(args):
    """Separability of MDHP-GDS parameters between normal and attacked windows
    (a synthetic analogue of the paper's CDF experiment): background windows
    of workload-2 shape (M = 16, beta = 1, 1,000-3,000 events); half of each
    group receive one time-exciting injection stream (each strategy with NPP
    and ND candidates, and DRP) on a random message ID k; every window is
    fitted by projected Adam to tol 1e-6; two scores of ID k (k random in
    normal windows): the baseline share mu_k / (N_k / T) and the
    self-excitation alpha_kk / beta.  Reports the AUC per combination."""
    import torch

    from paper_2411_10258_gb300 import DeviceBatch, FitOptions, Plan
    from paper_2411_10258_gb300.workload import attacks, workload

    dev = torch.device("cuda", 0)
    M, n = 16, args.attack_windows
    combos = [(sp, st) for sp in ("NPP", "ND") for st in attacks.STRATEGIES] + [("DRP", "DAM")]
    rng = np.random.default_rng(77)
    B = 2 * n * len(combos)
    betas = np.ones((B, 1))
    mu, alpha = workload.sample_params(rng, B, M, 0, betas, rng.uniform(0.2, 0.8, B))
    counts = workload.log_uniform_counts(rng, B, 1000, 3000)
    bg = workload.simulate(M, 0, mu, alpha, betas, counts, 7, 21)
    ts, ids, Ts, ks, labels, combo_of = [], [], [], [], [], []
    for c, (sp, st) in enumerate(combos):
        for r in range(2 * n):
            b = c * 2 * n + r
            t, u, T, _ = bg.window(b)
            k = int(rng.integers(M))
            if r < n:  # attacked
                a = attacks.sample(sp, st, rng)
                t, u = attacks.inject(t, u, float(T), a, k)
            ts.append(np.asarray(t, dtype=np.float32))
            ids.append(np.asarray(u, dtype=np.int16))
            Ts.append(max(float(T), float(np.float32(t[-1])) if len(t) else 0.0))
            ks.append(k)
            labels.append(r < n)
            combo_of.append(c)
    off = np.zeros(B + 1, dtype=np.int64)
    np.cumsum([len(x) for x in ts], out=off[1:])
    up = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    db = DeviceBatch(M, 0, up(off), up(np.concatenate(ts)), up(np.concatenate(ids)),
                     up(np.asarray(Ts, dtype=np.float32)), None, int(np.diff(off).max()))
    plan = Plan(M, 0, B, int(np.diff(off).max()))
    beta = torch.ones(B, 1, device=dev)
    mu_d = torch.zeros(B, M, device=dev)
    al_d = torch.zeros(B, M, M, device=dev)
    opts = FitOptions(optimizer=1, max_iters=2000, lr=1e-2, tol=1e-6, init=1)
    plan.set_timing(True)
    out = plan.fit(db, opts, mu_d, al_d, beta)
    torch.cuda.synchronize()
    ms = plan.last_fit_ms()
    mu_h, al_h = mu_d.cpu().numpy(), al_d.cpu().numpy()
    n_k = np.array([np.sum(x == k) for x, k in zip(ids, ks)], dtype=np.float64)
    base_share = np.array([mu_h[b, ks[b]] * Ts[b] / max(n_k[b], 1.0) for b in range(B)])
    self_exc = np.array([al_h[b, ks[b], ks[b]] for b in range(B)])
    labels, combo_of = np.asarray(labels), np.asarray(combo_of)
    res = {}
    for c, (sp, st) in enumerate(combos):
        sel = combo_of == c
        pos, neg = sel & labels, sel & ~labels
        res[f"{sp}/{st}"] = {"auc_mu_share": _auc(-base_share[pos], -base_share[neg]),
                             "auc_alpha_kk": _auc(self_exc[pos], self_exc[neg]),
                             "injected_mean": float(np.mean([len(ts[b]) for b in np.nonzero(pos)[0]])
                                                    - np.mean(counts[pos]))}
    st_bad = int((out["status"].cpu().numpy() != 0).sum())
    line = {"metric": "AUC of MDHP-GDS parameters, attacked vs normal windows", "value": None,
            "unit": "AUC", "n_gpus": 1, "data": "synthetic", "dtype": "f32",
            "config": {"workload": f"{B} windows, M=16, beta=1, 1,000-3,000 background events, "
                                   f"{n} attacked + {n} normal per combination, Adam lr 1e-2 to tol 1e-6",
                       "scores": "mu_k T / N_k (lower when injected events are not baseline) and "
                                 "alpha_kk (self-excitation of the attacked ID)"},
            "fit_ms": ms, "fits_per_s": B / (ms / 1000.0), "invalid_windows": st_bad,
            "iters_median": float(np.median(out["iters"].cpu().numpy())), "auc": res}
    line["value"] = float(np.mean([max(v["auc_mu_share"], v["auc_alpha_kk"]) for v in res.values()]))
    print(json.dumps(line), flush=True)


def run_lstm(args):
    """MDHP-LSTM cell, forward + backward over a batch of windows: 4,096
    windows of 128 messages with 11 inputs each (the paper's SOME/IP window
    shape: 10 fields and the time), H = 64, the windows' MDHP parameters with
    M = 16 and a scalar beta, one output.  value = windows/s for forward +
    backward; FLOP count of the gate, cell and output arithmetic."""
    import torch

    from paper_2411_10258_gb300 import MdhpLSTMFunction

    dev = torch.device("cuda", 0)
    B, L, D, H, M, O = 4096, 128, 11, 64, 16, 1
    g = torch.Generator(device=dev).manual_seed(3)
    r = lambda *s, lo=0.0, hi=1.0: (torch.rand(*s, generator=g, device=dev) * (hi - lo) + lo)
    k = 1.0 / np.sqrt(H)
    leaf = lambda t: t.requires_grad_(True)
    x = leaf(r(B, L, D, lo=-1.0))
    mu, alpha, beta = leaf(r(B, M, lo=0.1)), leaf(r(B, M, M, hi=0.05)), leaf(r(B, 1, lo=0.5, hi=2.0))
    T = r(B, lo=5.0, hi=20.0)
    W, U, b = leaf(r(4 * H, D, lo=-k, hi=k)), leaf(r(4 * H, H, lo=-k, hi=k)), leaf(r(4 * H, lo=-k, hi=k))
    A, Bm, C = leaf(r(H, M * M, lo=-k, hi=k)), leaf(r(H, 1, lo=-k / 20, hi=k / 20)), leaf(r(H, M, lo=-k, hi=k))
    Wy = leaf(r(O, H, lo=-k, hi=k))
    dy = torch.ones(B, L, O, device=dev)

    def step():
        y = MdhpLSTMFunction.apply(x, mu, alpha, beta, T, W, U, b, A, Bm, C, Wy)
        y.backward(dy)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(0, args.clocks_dir)
    with sampler:
        e0.record()
        for _ in range(args.steps):
            step()
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    G = 4 * H
    fwd = 2 * G * (D + H) + 10 * H + 2 * O * H           # per step and sequence
    bwd = 2 * G * (D + H) + 2 * G * (D + H) + 20 * H + 4 * O * H  # dx, dh, and the weight sums
    flops = float(B) * L * (fwd + bwd)
    peaks, src = measured_peaks()
    peak = fp32_peak_tflops(torch.cuda.get_device_properties(dev).multi_processor_count,
                            float(peaks.get("sm_max_mhz", 2070.0)))
    ach = flops / (ms / 1000.0) / 1e12
    line = {"metric": "MDHP-LSTM forward+backward windows/s", "value": B / (ms / 1000.0),
            "unit": "windows/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{B} windows x {L} messages x {D} inputs, H={H}, M={M}, scalar beta, O={O}"},
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                         "flops_per_step_sequence": fwd + bwd, "traffic": None,
                         "kernel": "k_lstm_fwd_s / k_lstm_bwd_s (S sequences per CTA through time)"},
            "clocks": sampler.summary()}
    print(json.dumps(line), flush=True)


def run_warm_cold(args):
    """Workload 5: 65,536 windows (M = 32, counts log-uniform [100, 10000], 10 %
    with an injected self-exciting component), fitted to |dlnL| <= tol |lnL|
    (3 in a row) by projected Adam, from the cold rule and from the learned
    initializer (trained first, untimed, on separately simulated windows with
    known parameters).  value = warm-start windows/s; the cold figure, the
    iteration counts and the distance to a long-run optimum are reported too."""
    import torch

    from paper_2411_10258_gb300 import DeviceBatch, FitOptions, InitModel, Plan, simulate
    from paper_2411_10258_gb300.workload import workload

    dev = torch.device("cuda", 0)
    B = args.windows if args.windows != 4096 else 65536
    bt = workload.make_workload(5, B=B, seed=2024)
    M = bt.M
    db = DeviceBatch.from_host(bt, dev)
    beta = torch.from_numpy(bt.beta).to(dev)
    # training windows: workload-5 parameters, simulated by the library's GPU simulator
    tp = workload.make_params(5, B=args.train_windows, seed=4048)
    dtr, sst = simulate(M, 0, tp["mu"], tp["alpha"], tp["beta"], tp["counts"], seed=4048, stream_id=5)
    if int((sst != 0).sum().item()):
        raise RuntimeError("training-window simulation failed")
    btr = torch.from_numpy(tp["beta"]).float().to(dev)
    model = InitModel(M, hidden=256, max_batch=4096, seed=1024)
    feat, mu_cold = model.features(dtr, btr)
    mu_t = torch.from_numpy(tp["mu"].astype(np.float32)).to(dev)
    al_t = torch.from_numpy(tp["alpha"].astype(np.float32)).to(dev)
    rng = np.random.default_rng(0)
    for _ in range(args.train_steps):
        idx = torch.from_numpy(rng.choice(dtr.B, 512, replace=False)).to(dev)
        model.train_step(feat[idx], mu_cold[idx], btr[idx].reshape(-1), mu_t[idx], al_t[idx],
                         lr=3e-4, weight_decay=5e-5)
    del feat, dtr
    plan = Plan(M, 0, B, int(bt.counts.max()))
    model.attach(plan)
    # launch shape from the library's autotuner on this batch (untimed; tol = 0)
    tuned = None if args.no_autotune else plan.autotune(
        db, FitOptions(optimizer=1, lr=2e-2, init=1), torch.zeros(B, M, device=dev),
        torch.zeros(B, M, M, device=dev), beta.clone(), tune_iters=20)
    res = {}
    for name, init in (("cold", 1), ("warm", 2)):
        opts = FitOptions(optimizer=1, max_iters=3000, lr=2e-2, tol=args.tol, init=init)
        mu = torch.zeros(B, M, device=dev)
        al = torch.zeros(B, M, M, device=dev)
        be = beta.clone()
        plan.fit(db, opts, mu, al, be)  # warm-up
        torch.cuda.synchronize()
        # median of three fits: the time is set by the slowest windows' tail
        times = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = plan.fit(db, opts, mu, al, be.copy_(beta))
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = float(np.median(times))
        res[name] = dict(ms=ms, fits_per_s=B / (ms / 1e3), ms_runs=times,
                         iters_median=float(out["iters"].float().median().item()),
                         iters_p90=float(torch.quantile(out["iters"].float(), 0.9).item()),
                         loglik=out["loglik"].cpu().numpy())
    # bound on any warm start: the same fit started at the generating parameters
    opts = FitOptions(optimizer=1, max_iters=3000, lr=2e-2, tol=args.tol, init=0)
    mu_g = torch.from_numpy(bt.mu_true.astype(np.float32)).to(dev)
    al_g = torch.from_numpy(bt.alpha_true.astype(np.float32)).to(dev)
    out = plan.fit(db, opts, mu_g.clone(), al_g.clone(), beta.clone())
    torch.cuda.synchronize()
    res["generating_params_start"] = dict(
        iters_median=float(out["iters"].float().median().item()),
        iters_p90=float(torch.quantile(out["iters"].float(), 0.9).item()),
        loglik=out["loglik"].cpu().numpy())
    for _ in range(2):
        model.predict(db, beta)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    model.predict(db, beta)
    e1.record()
    torch.cuda.synchronize()
    res["warm"]["predict_ms"] = e0.elapsed_time(e1)
    ref = plan.fit(db, FitOptions(optimizer=1, max_iters=3000, lr=2e-2, init=1),
                   torch.zeros(B, M, device=dev), torch.zeros(B, M, M, device=dev), beta.clone())
    torch.cuda.synchronize()
    arms = ("cold", "warm", "generating_params_start")
    lref = np.maximum.reduce([ref["loglik"].cpu().numpy()] + [res[k]["loglik"] for k in arms])
    for name in arms:
        gap = (lref - res[name].pop("loglik")) / np.abs(lref)
        res[name]["within_1e-4_of_best"] = float(np.mean(gap <= 1e-4))
        res[name]["gap_median"] = float(np.median(gap))
    line = {"metric": METRIC, "value": res["warm"]["fits_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": 3, "warmup": 1, "ms_per_step": res["warm"]["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{B} windows x M=32, counts log-uniform[100,10000], 10% injected "
                                   f"component, projected Adam lr 2e-2 to tol {args.tol}",
                       "init_training": f"{args.train_windows} GPU-simulated windows (generating "
                                        f"parameters as targets), {args.train_steps} AdamW steps of 512",
                       "autotuned": tuned},
            "warm": res["warm"], "cold": res["cold"],
            "generating_params_start": res["generating_params_start"]}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == '5':
        run_warm_cold(args)
    elif args.workload == '3':
        run_long_learned(args)
    elif args.workload == "attack":
        run_attacks(args)
    elif args.workload == "lstm":
        run_lstm(args)
    else:  # 2, or 6 (the same with the full decay matrix)
        run_ours(args)


if __name__ == "__main__":
    main()
