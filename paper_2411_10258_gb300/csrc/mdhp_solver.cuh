// Device side of MDHP-GDS for sm_103a: one CTA owns one window at a time.
//
// Model (arXiv 2411.10258): MDHP intensity of Sec. II and the closed-form
// log-likelihood of Sec. IV-B.1 (Part1 + Part2 + Part3, App. B).  Instead of
// the paper's padded O(D^2 L^2) broadcast (Alg. 1-3) the window is walked in
// time order with the exact recursion
//   R_j(t) = sum_{k: u_k = j, t_k < t} w_k exp(-beta_j (t - t_k))      (decay state of source j)
//   S_j(t) = sum_{k: u_k = j, t_k < t} w_k (t - t_k) exp(-beta_j (t - t_k))   (its beta-derivative)
//   lambda_n = mu_{u_n} + sum_j alpha_{u_n j} R_j(t_n)
// which costs O(N M) per evaluation.  The compensator (Part2 + Part3) comes
// from the state at T_span: C_j = (W_j - R_j(T)) / beta_j, W_j = sum of source
// j's weights, and d C_j / d beta_j = (S_j(T) - C_j) / beta_j.
//
// Parallel decomposition of a window (events are sorted by time):
//   * the CTA's threads form NC = blockDim / SPL chunk groups; chunk c owns the
//     contiguous events [b_c, b_{c+1}), boundaries moved past tie groups so that
//     a timestamp never straddles two chunks;
//   * SPL threads of a chunk split the M sources (MS = M / SPL each, a multiple
//     of 4 so rows move as float4), so the per-thread state R[MS] (and S[MS])
//     lives in registers;
//   * pass 1 computes each chunk's local effect (state at the next chunk's
//     anchor, starting from zero), a per-source scan over chunks composes the
//     affine maps (R, S) -> (A R + R_loc, A (S + D R) + S_loc), A = exp(-beta D),
//     and gives every chunk its entering state; with fixed beta this runs once
//     per window, with learned beta once per evaluation;
//   * pass 2 walks each chunk from its entering state and accumulates ln lambda
//     (Kahan, FP32), d/dmu and d/dalpha and d/dbeta.  The d/dalpha row of an
//     event is selected by its id, which differs from lane to lane; it is
//     accumulated without atomics in per-thread private slots laid out
//     [id][float4 slice][thread] (conflict-free: a warp's 32 lanes always hit 32
//     distinct 16-byte slots in consecutive banks), and summed over threads
//     once per evaluation.  For M = 64 the private slots would not fit, and the
//     sums go to one shared copy with shared-memory atomics instead.
// Ties (Sec. II: the inner sum is strict): the increments of a tie group are
// added only when time advances past it.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mdhp_async.cuh"

namespace mdhp {

constexpr float kLog2e = 1.4426950408889634f;
constexpr double kLn2 = 0.69314718055994530942;

enum : int {
  kOK = 0, kE_ARG = 1, kE_UNSORTED = 2, kE_ID_RANGE = 3, kE_TIME_RANGE = 4,
  kE_NONFINITE = 5, kE_MAXITER = 6, kE_TIMEOUT = 7
};

// private accumulators for template capacity M (atomics beyond)
template <int M>
struct UsePriv {
  static constexpr bool value = M <= 32;
};

// 2^f for |f| <= 1/2: Taylor series of e^(f ln 2) to degree 7 (truncation
// below 6e-9 relative), evaluated by Horner so the last rounding is a plain
// round-to-nearest.
__device__ __forceinline__ float exp2_poly(float f) {
  float p = 1.5252733804059840e-05f;
  p = fmaf(p, f, 1.5403530393381608e-04f);
  p = fmaf(p, f, 1.3333558146428443e-03f);
  p = fmaf(p, f, 9.6181291076284772e-03f);
  p = fmaf(p, f, 5.5504108664821580e-02f);
  p = fmaf(p, f, 2.4022650695910071e-01f);
  p = fmaf(p, f, 6.9314718055994531e-01f);
  return fmaf(p, f, 1.0f);
}
// 2^x for the decay factors of the recursion.  x = k + f with k the nearest
// integer to x and |f| <= 1/2; 2^f from exp2_poly; 2^k applied exactly by
// adding k to the exponent field.  Unlike the approximate hardware
// exponential its error has no one-sided bias, which matters because the
// recursion multiplies thousands of these factors.
//
// The rounding to k adds 1.5 * 2^23 (where the float spacing is 1, so the sum
// is rounded to an integer, half to even) and subtracts it again: f is then
// exact, and k sits in the low bits of the sum, two's complement, so that
// shifting the sum's bit pattern left by 23 gives k << 23.  Everything runs on
// the FMA and integer pipes (no float-to-int conversion, no multiply by 2^k).
// Arguments below -125 are taken as -125: the factor is then 2^-125 instead
// of the exact value below it, a difference no recursion state can resolve
// against intensities of at least mu_floor.  Callers keep x <= 64.
__device__ __forceinline__ float exp2_acc(float x) {
  constexpr float kRound = 12582912.f;  // 1.5 * 2^23
  const float xc = fmaxf(x, -125.f);
  const float kt = xc + kRound;
  const float f = xc - (kt - kRound);
  const float p = exp2_poly(f);
  return __int_as_float(__float_as_int(p) + (__float_as_int(kt) << 23));
}

// Hardware base-2 logarithm and reciprocal of an intensity (PTX lg2.approx /
// rcp.approx, flush-to-zero forms: no subnormal scaling).  An intensity is at
// least mu_floor (default 1e-10), far above the subnormal range; one below
// 2^-126 reads as 0, its log as -inf, and the evaluation is reported
// non-finite.
__device__ __forceinline__ float lg2_ftz(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_ftz(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// approximate square root (PTX sqrt.approx, flush-to-zero) of a second moment >= 0
__device__ __forceinline__ float sqrt_ftz(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Double-float numbers (hi + lo, about 48 significant bits) for the lnL total,
// the convergence test and the compensator constants of every iteration: on
// GB300 a dependent FP64 add takes about 64 cycles (FP32: 4.5) and a
// float<->double conversion about 50, which put FP64 arithmetic on every
// iteration's critical path.  TwoSum
// (Knuth) for additions, an FMA-based exact product for the scaling by ln 2;
// the result goes to FP64 once, when the window is done.
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_norm(float s, float e) {
  const float h = s + e;
  return {h, e - (h - s)};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = ((a.hi - (s - bb)) + (b.hi - bb)) + (a.lo + b.lo);
  return ff_norm(s, e);
}
__device__ __forceinline__ FF ff_mul(FF a, float bh, float bl) {
  const float p = a.hi * bh;
  const float e = fmaf(a.hi, bh, -p) + fmaf(a.hi, bl, a.lo * bh);
  return ff_norm(p, e);
}
__device__ __forceinline__ FF ff_div(FF a, float b) {
  const float q = a.hi / b;
  const float r = fmaf(-q, b, a.hi) + a.lo;
  return ff_norm(q, r / b);
}
__device__ __forceinline__ double ff_to_double(FF v) { return (double)v.hi + (double)v.lo; }
constexpr float kLn2Hi = 0.693147182464599609375f;  // the float nearest ln 2
constexpr float kLn2Lo = -1.9046542999e-09f;          // ln 2 - kLn2Hi


// ---------------------------------------------------------------------------
// Event access: staged in shared memory (t float, id uint16: 6 bytes per
// event) or read from global memory.
// ---------------------------------------------------------------------------
struct EvS {
  const float *t;
  const uint16_t *u;
  const float *w;
  __device__ __forceinline__ void get(int n, float &tt, int &uu) const {
    tt = t[n];
    uu = (int)u[n];
  }
  __device__ __forceinline__ float time(int n) const { return t[n]; }
  __device__ __forceinline__ int id(int n) const { return (int)u[n]; }
  __device__ __forceinline__ float wt(int n) const { return w ? w[n] : 1.f; }
  // a chunk's events in order (pass 2): nothing to stage
  __device__ __forceinline__ void chunk_begin(int, int, int, int, unsigned) const {}
  __device__ __forceinline__ void next(int n, float &tt, int &uu) const { get(n, tt, uu); }
  __device__ __forceinline__ void chunk_end() const {}
};

struct EvG {
  const float *t;
  const int16_t *u;
  const float *w;
  __device__ __forceinline__ void get(int n, float &tt, int &uu) const {
    tt = __ldg(t + n);
    uu = (int)__ldg(u + n);
  }
  __device__ __forceinline__ float time(int n) const { return __ldg(t + n); }
  __device__ __forceinline__ int id(int n) const { return (int)__ldg(u + n); }
  __device__ __forceinline__ float wt(int n) const { return w ? __ldg(w + n) : 1.f; }
  __device__ __forceinline__ void chunk_begin(int, int, int, int, unsigned) const {}
  __device__ __forceinline__ void next(int n, float &tt, int &uu) const { get(n, tt, uu); }
  __device__ __forceinline__ void chunk_end() const {}
};

// Streamed events of a window too long to stage whole, delivered to pass 2
// through a ring of shared-memory stages per chunk, each stage filled by bulk
// copies (the TMA engine's linear mode, CTA-local, no multicast) of the
// chunk's next kRingK times and ids, completed on the stage's mbarrier.  The
// chunk's first thread (source slice 0) issues the copies kRingD stages ahead;
// all SPL threads of the chunk wait (bounded) on a stage before reading it.
// A copy must start on a 16-byte boundary and move a multiple of 16 bytes, so
// a stage copies the 16-byte-aligned span around its events, clamped to the
// batch arrays; events past the clamp (the batch's last few) and the tie
// groups that reach back into an earlier stage are read from global memory.
// A wait that gives up sets the CTA's flag, and the ring is not used again
// by that CTA: its chunks read global memory from then on (same results).
// Random access (chunk boundaries, pass 1) reads global memory directly.
constexpr int kRingK = 128, kRingD = 2;
constexpr int kRingKT = kRingK + 8;   // time slots per stage (alignment slack)
constexpr int kRingKU = kRingK + 16;  // id slots per stage
__host__ __device__ inline int ring_bytes(int NC) {
  return NC * kRingD * (kRingKT * 4 + kRingKU * 2 + 8);
}

struct EvRing {
  const float *t;      // window's events (global)
  const int16_t *u;
  const float *w;      // always nullptr: weighted windows do not use the ring
  const float *tb;     // batch arrays (16-byte aligned)
  const int16_t *ub;
  int64_t o0, ntot;    // window's first event in the batch; events in the batch
  float *rt;           // [NC][kRingD][kRingKT]
  uint16_t *ru;        // [NC][kRingD][kRingKU]
  uint64_t *bar;       // [NC][kRingD]
  int *fillc;          // [NC] stages each chunk has consumed (persists across windows)
  int *dead;           // a wait gave up: the ring is off for this CTA
  uint32_t polls;      // bound of a stage wait (0: the default)
  // current chunk (set by chunk_begin, advanced by next)
  mutable int c, s, b0, b1, nst, g, f0;
  mutable int64_t S0, S1, U0, U1;
  mutable unsigned gm;
  mutable bool on;

  __device__ __forceinline__ void get(int n, float &tt, int &uu) const {
    tt = __ldg(t + n);
    uu = (int)__ldg(u + n);
  }
  __device__ __forceinline__ float time(int n) const { return __ldg(t + n); }
  __device__ __forceinline__ int id(int n) const { return (int)__ldg(u + n); }
  __device__ __forceinline__ float wt(int) const { return 1.f; }

  __device__ __forceinline__ int slot(int gg) const { return (f0 + gg) % kRingD; }
  __device__ __forceinline__ uint32_t parity(int gg) const { return (uint32_t)(((f0 + gg) / kRingD) & 1); }
  // aligned spans of stage gg (absolute batch indices), clamped to the arrays
  __device__ __forceinline__ void span(int gg, int64_t &s0, int64_t &s1, int64_t &u0, int64_t &u1) const {
    const int e0 = b0 + gg * kRingK, e1 = min(e0 + kRingK, b1);
    const int64_t a0 = o0 + e0, a1 = o0 + e1;
    s0 = a0 & ~(int64_t)3;
    s1 = (a1 + 3) & ~(int64_t)3;
    const int64_t lt = ntot & ~(int64_t)3;
    if (s1 > lt) s1 = lt > s0 ? lt : s0;
    u0 = a0 & ~(int64_t)7;
    u1 = (a1 + 7) & ~(int64_t)7;
    const int64_t lu = ntot & ~(int64_t)7;
    if (u1 > lu) u1 = lu > u0 ? lu : u0;
  }
  __device__ __forceinline__ void issue(int gg) const {
    int64_t s0, s1, u0, u1;
    span(gg, s0, s1, u0, u1);
    const int sl = slot(gg);
    uint64_t *br = bar + c * kRingD + sl;
    const uint32_t bt = (uint32_t)(s1 - s0) * 4u, bu = (uint32_t)(u1 - u0) * 2u;
    fence_proxy_async_shared();  // the slot's earlier reads before the copy's writes
    mbar_expect_tx(br, bt + bu);
    if (bt) bulk_copy_g2s(rt + (c * kRingD + sl) * kRingKT, tb + s0, bt, br);
    if (bu) bulk_copy_g2s(ru + (c * kRingD + sl) * kRingKU, ub + u0, bu, br);
  }
  // wait for stage gg (every thread of the chunk; the outcome is made uniform)
  __device__ __forceinline__ void enter(int gg) const {
    const bool ok = __all_sync(gm, mbar_wait_for(bar + c * kRingD + slot(gg), parity(gg), polls));
    g = gg;
    if (!ok) {
      if (s == 0) *dead = 1;
      on = false;
      return;
    }
    span(gg, S0, S1, U0, U1);
  }
  __device__ __forceinline__ void chunk_begin(int cc, int ss, int bb0, int bb1, unsigned mask) const {
    c = cc;
    s = ss;
    b0 = bb0;
    b1 = bb1;
    gm = mask;
    g = 0;
    const int lead = __ffs(mask) - 1;
    const int off = __shfl_sync(mask, *dead, lead);  // one reading for the whole chunk
    f0 = __shfl_sync(mask, fillc[cc], lead);
    nst = off ? 0 : (bb1 - bb0 + kRingK - 1) / kRingK;
    on = nst > 0;
    if (!on) return;
    if (s == 0)
      for (int gg = 0; gg < kRingD && gg < nst; ++gg) issue(gg);
    enter(0);
  }
  __device__ __forceinline__ void next(int n, float &tt, int &uu) const {
    if (on) {
      const int gn = (n - b0) / kRingK;
      if (gn != g) {  // the chunk's threads are done with stage g: refill its slot
        __syncwarp(gm);
        if (s == 0 && g + kRingD < nst) issue(g + kRingD);
        enter(gn);
      }
    }
    if (on) {
      const int64_t a = o0 + n;
      const int sl = slot(g);
      tt = a < S1 ? rt[(c * kRingD + sl) * kRingKT + (int)(a - S0)] : __ldg(t + n);
      uu = a < U1 ? (int)ru[(c * kRingD + sl) * kRingKU + (int)(a - U0)] : (int)__ldg(u + n);
    } else {
      get(n, tt, uu);
    }
  }
  // Every stage was issued and entered by the end of a chunk, unless a wait
  // gave up at stage g: then stages g .. g + kRingD - 1 (those issued) are
  // waited out here, bounded, before the chunk's threads go on.
  __device__ __forceinline__ void chunk_end() const {
    if (nst > 0 && !on) {
      for (int gg = g; gg < nst && gg < g + kRingD; ++gg)
        mbar_wait(bar + c * kRingD + slot(gg), parity(gg));
    }
    __syncwarp(gm);
    if (s == 0) fillc[c] = f0 + nst;
  }
};

// First event of chunk c out of NC over [0, N): the even split moved forward
// past any tie group, so every chunk starts at a new timestamp.
template <typename EV>
__device__ __forceinline__ int chunk_begin(int c, int NC, int N, const EV &ev) {
  if (c >= NC) return N;
  int b = (int)(((long long)c * (long long)N) / NC);
  while (b > 0 && b < N && ev.time(b) == ev.time(b - 1)) ++b;
  return b;
}

// ---------------------------------------------------------------------------
// Shared-memory carve of one CTA (sizes depend on M, NT, NC, event capacity).
// ---------------------------------------------------------------------------
struct Carve {
  // byte offsets
  int alpha, oh, ga, mu, gm, beta, bl2, gb, W, cnt, C, dC, endR, endS, anc, bnd, encR, encS, prev,
      gbuf, am, av, red, ctl, gpriv, mpriv, ev_t, ev_u, ev_w, tstart, tf, tl, P, xs, ring, mbar,
      rt, ru, rbar, rfill;  // streamed events' bulk-copy ring (recursion fit)
  int total;
};

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }
__host__ __device__ inline int pitch4(int M) { return M + 4; }  // 16-byte rows, staggered banks
// Shared d/dalpha copy (M = 64, updated with shared atomics): one pad word
// after every 8 columns and an odd row pitch, so that the 8 threads of a
// chunk (8 consecutive sources each) hit 8 different banks for any target row.
__host__ __device__ inline int ga_pitch(int M) { return M + M / 8 + 1; }
__host__ __device__ inline int ga_col(int j) { return j + (j >> 3); }

// prev_smem = false: theta_{k-1}, the gradient buffer and the Adam moments
// live in the launch's per-CTA device slot instead of shared memory.
// ring: the streamed events' bulk-copy ring (ring_bytes(NC)).
__host__ __device__ inline Carve make_carve(int M, int NT, int SPL, int ev_cap, bool weights,
                                            bool learn, bool adam, bool fit, bool priv,
                                            bool prev_smem = true, bool ring = false) {
  const int NC = NT / SPL;
  Carve c = {};
  int o = 0;
  const int AP = pitch4(M);
  const int npm = M + M * M + M;
  auto take = [&](int bytes) { int r = o; o = align_up(o + bytes, 16); return r; };
  c.red = take(32 * 8);
  c.ctl = take(16 * 4);
  c.alpha = take(M * AP * 4);
  c.ga = priv ? 0 : take(M * ga_pitch(M) * 4);
  c.mu = take(M * 4);
  c.gm = take(M * 4);
  c.beta = take(M * 4);
  c.bl2 = take(M * 4);
  c.gb = take(M * 4);
  c.W = take(M * 8);
  c.cnt = take(M * 4);
  c.C = take(M * 4);
  c.dC = take(M * 4);
  c.endR = take(M * 4);
  c.endS = take(M * 4);
  c.anc = take((NC + 1) * 4);
  c.bnd = take((NC + 1) * 4);
  c.encR = take(NC * M * 4);
  c.encS = learn ? take(NC * M * 4) : c.encR;
  c.prev = (fit && prev_smem) ? take(npm * 4) : 0;  // else in the launch's per-CTA device slot
  c.gbuf = (fit && prev_smem) ? take(npm * 4) : 0;
  c.am = (fit && adam && prev_smem) ? take(npm * 4) : 0;
  c.av = (fit && adam && prev_smem) ? take(npm * 4) : 0;
  c.gpriv = priv ? take(M * (M / SPL) * NT * 4) : 0;  // [id][slice][thread] float4
  c.mpriv = priv ? take(M * NC * 4) : 0;                // [id][chunk]
  c.ev_t = ev_cap > 0 ? take(ev_cap * 4) : 0;
  c.ev_w = (ev_cap > 0 && weights) ? take(ev_cap * 4) : 0;
  c.ev_u = ev_cap > 0 ? take(ev_cap * 2) : 0;
  if (ring && ev_cap == 0) {
    c.rt = take(NC * kRingD * kRingKT * 4);
    c.ru = take(NC * kRingD * kRingKU * 2);
    c.rbar = take(NC * kRingD * 8);
    c.rfill = take(NC * 4);
  }
  c.total = o;
  return c;
}

// Carve of the decoupled fixed-beta fit (features x_n = R(t_n) stored once per
// window, grouped by event type).  NT threads = NT chunks; P holds the
// per-thread segment sums, (NT + M) slots of M + 4 floats (the chunk/type
// counters of the feature pass share the same space); xcap > 0 places the
// features in shared memory (xcap events x M floats).
__host__ __device__ inline Carve make_carve_x(int M, int NT, int xcap, bool adam,
                                              int pipe_steps = 0, int pipe_stages = 0,
                                              bool matrix = false) {
  const int MB = matrix ? M * M : M;  // beta, beta log2(e) and C: one per pair for matrix beta
  Carve c = {};
  int o = 0;
  const int AP = pitch4(M);
  const int npm = M + M * M + M;
  auto take = [&](int bytes) { int r = o; o = align_up(o + bytes, 16); return r; };
  c.red = take(32 * 8);
  c.ctl = take(16 * 4);
  c.alpha = take(M * AP * 4);
  c.mu = take(M * 4);
  c.gm = take(M * 4);
  c.beta = take(MB * 4);
  c.bl2 = take(MB * 4);
  c.gb = take(M * 4);
  c.W = take(M * 8);
  c.cnt = take(M * 4);
  c.C = take(MB * 4);
  c.dC = take(M * 4);
  c.endR = take(M * 4);
  c.endS = take(M * 4);
  c.anc = take((NT + 1) * 4);
  c.bnd = take((NT + 1) * 4);
  c.encR = take(NT * M * 4);
  c.encS = c.encR;
  c.prev = take(npm * 4);
  c.gbuf = take(npm * 4);
  c.am = adam ? take(npm * 4) : 0;
  c.av = adam ? take(npm * 4) : 0;
  c.tstart = take((M + 1) * 4);
  c.tf = take(M * 4);
  c.tl = take(M * 4);
  c.P = take((NT + M) * (M + 4) * 4);
  c.xs = xcap > 0 ? take(xcap * M * 4) : 0;
  // streamed features: a ring of pipe_stages buffers of pipe_steps steps
  // (NT float4 per slice and step) filled by bulk copies, one mbarrier each
  const bool pipe = xcap == 0 && pipe_stages > 0 && pipe_steps > 0;
  c.mbar = pipe ? take(pipe_stages * 8) : 0;
  c.ring = pipe ? take(pipe_stages * pipe_steps * (M / 4) * NT * 16) : 0;
  c.total = o;
  return c;
}

template <int M>
struct Sm {
  double *W;  // per-type weight sums (exact for counts, FP64 for weights)
  float *alpha, *oh, *ga, *mu, *gm, *beta, *bl2, *gb, *C, *dC, *endR, *endS, *anc, *encR,
      *encS, *prev, *gbuf, *am, *av, *gpriv, *mpriv;
  int *bnd, *cnt, *ctl, *tstart, *tf, *tl;
  float *P;
  float4 *xs, *ring;
  uint64_t *mbar;
  float *rt;         // streamed events' ring: times [NC][kRingD][kRingKT]
  uint16_t *ru;      //   ids [NC][kRingD][kRingKU]
  uint64_t *rbar;    //   one mbarrier per chunk and stage
  int *rfill;        //   stages consumed per chunk
  double *red;
  float *ev_t, *ev_w;
  uint16_t *ev_u;
  __device__ void bind(unsigned char *base, const Carve &c) {
    alpha = (float *)(base + c.alpha); oh = (float *)(base + c.oh); ga = (float *)(base + c.ga);
    mu = (float *)(base + c.mu); gm = (float *)(base + c.gm); beta = (float *)(base + c.beta);
    bl2 = (float *)(base + c.bl2); gb = (float *)(base + c.gb); W = (double *)(base + c.W);
    cnt = (int *)(base + c.cnt); C = (float *)(base + c.C); dC = (float *)(base + c.dC);
    endR = (float *)(base + c.endR); endS = (float *)(base + c.endS);
    anc = (float *)(base + c.anc); bnd = (int *)(base + c.bnd);
    encR = (float *)(base + c.encR); encS = (float *)(base + c.encS);
    prev = (float *)(base + c.prev); gbuf = (float *)(base + c.gbuf);
    am = (float *)(base + c.am); av = (float *)(base + c.av);
    gpriv = (float *)(base + c.gpriv); mpriv = (float *)(base + c.mpriv);
    red = (double *)(base + c.red); ctl = (int *)(base + c.ctl);
    ev_t = (float *)(base + c.ev_t); ev_w = (float *)(base + c.ev_w);
    ev_u = (uint16_t *)(base + c.ev_u);
    tstart = (int *)(base + c.tstart); tf = (int *)(base + c.tf); tl = (int *)(base + c.tl);
    P = (float *)(base + c.P); xs = (float4 *)(base + c.xs);
    ring = (float4 *)(base + c.ring); mbar = (uint64_t *)(base + c.mbar);
    rt = (float *)(base + c.rt); ru = (uint16_t *)(base + c.ru);
    rbar = (uint64_t *)(base + c.rbar); rfill = (int *)(base + c.rfill);
  }
};

// ---------------------------------------------------------------------------
// Block reduction (every thread receives the same sum, in the same order)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum_double(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

// ---------------------------------------------------------------------------
// Which sources a thread of a chunk holds.  The M sources form M/4 groups of
// 4; thread s of the chunk's SPL threads holds groups s, s + SPL, s + 2 SPL,
// ... (MS/4 of them), its state slot jj being source src_of(s, jj).  With
// this interleaving the SPL threads that read an alpha row together read
// SPL consecutive 16-byte groups at every step (no bank conflict), where
// contiguous slices of MS sources would put threads s and s + 4 on the same
// banks once MS >= 8.  (For MS = 4 both are the same mapping.)
// ---------------------------------------------------------------------------
template <int SPL>
__device__ __forceinline__ int src_of(int s, int jj) {
  static_assert((SPL & (SPL - 1)) == 0, "threads per chunk: a power of two");
  return 4 * (s + SPL * (jj >> 2)) + (jj & 3);
}
// the slot of source u in thread s, or -1 when another thread of the chunk holds it
template <int SPL>
__device__ __forceinline__ int slot_of(int s, int u) {
  const int g = u >> 2;
  return (g & (SPL - 1)) == s ? 4 * (g / SPL) + (u & 3) : -1;
}

// ---------------------------------------------------------------------------
// Per-thread recursion over MS sources (MS % 4 == 0), slot jj = source
// src_of(s, jj).
// ---------------------------------------------------------------------------
template <int MS, int BM, bool LEARN>
struct Walker {
  static_assert(MS % 4 == 0, "sources per thread must be a multiple of 4");
  float R[MS];
  float S[LEARN ? MS : 1];
  float b2[BM == 0 ? 1 : MS];  // beta * log2(e)
  float bmax;                   // the largest of b2

  template <int SPL>
  __device__ __forceinline__ void load_beta(const float *bl2, int s) {
    bmax = 0.f;
#pragma unroll
    for (int jj = 0; jj < (BM == 0 ? 1 : MS); ++jj) {
      b2[jj] = bl2[BM == 0 ? 0 : src_of<SPL>(s, jj)];
      bmax = fmaxf(bmax, b2[jj]);
    }
  }
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int jj = 0; jj < MS; ++jj) {
      R[jj] = 0.f;
      if (LEARN) S[jj] = 0.f;
    }
  }
  __device__ __forceinline__ void decay(float dt) {
    if (BM == 0) {
      const float a = exp2_acc(-b2[0] * dt);
#pragma unroll
      for (int jj = 0; jj < MS; ++jj) {
        if (LEARN) S[jj] = a * fmaf(dt, R[jj], S[jj]);
        R[jj] *= a;
      }
    } else if (bmax * dt <= 0.5f) {
      // every exponent in [-1/2, 0]: exp2_acc reduces to its polynomial
      // (k = 0, f = x), so the same factors come without the range reduction
#pragma unroll
      for (int jj = 0; jj < MS; ++jj) {
        const float a = exp2_poly(-b2[BM == 0 ? 0 : jj] * dt);
        if (LEARN) S[jj] = a * fmaf(dt, R[jj], S[jj]);
        R[jj] *= a;
      }
    } else {
#pragma unroll
      for (int jj = 0; jj < MS; ++jj) {
        const float a = exp2_acc(-b2[BM == 0 ? 0 : jj] * dt);
        if (LEARN) S[jj] = a * fmaf(dt, R[jj], S[jj]);
        R[jj] *= a;
      }
    }
  }
  // R += w * e_u restricted to my sources; u_rel = slot_of(s, u), outside
  // [0, MS) for another thread's source
  __device__ __forceinline__ void add(int u_rel, float w) {
#pragma unroll
    for (int jj = 0; jj < MS; ++jj) R[jj] += (jj == u_rel) ? w : 0.f;
  }
};

// Pass 1 for chunk [b0, b1), ending at a1: the chunk's own contribution to the
// state at a1 -> encR/encS[c].  With a scalar beta, a walk from the chunk's
// first time a0 with one decay per timestamp.  With beta per source, each
// event is taken directly,
//   R_j(a1) = sum_{k in chunk, u_k = j} w_k exp(-beta_j (a1 - t_k)),
//   S_j(a1) = sum_{k in chunk, u_k = j} w_k (a1 - t_k) exp(-beta_j (a1 - t_k)),
// by the one thread of the chunk that owns source u_k: one exponential per
// event instead of one per source and timestamp, and no compounding of decay
// factors.  Every event of the chunk precedes a1 (chunk ends are moved past
// tie groups; the last chunk ends at T_span, where d = 0).
template <int M, int SPL, int BM, bool LEARN, typename EV>
__device__ __forceinline__ void pass1_chunk(int c, int s, int b0, int b1, float a0, float a1,
                                            const EV &ev, const Sm<M> &sm) {
  constexpr int MS = M / SPL;
  constexpr int AP = M + 4;
  if constexpr (BM == 0) {
    // one decay factor serves every source: walk the chunk from a0 (one
    // exponential per distinct timestamp)
    Walker<MS, BM, LEARN> wk;
    wk.template load_beta<SPL>(sm.bl2, s);
    wk.zero();
    float tprev = a0;
    int gs = b0;
    float tnx = b0 < b1 ? ev.time(b0) : 0.f;  // the next time, loaded one step ahead
    for (int n = b0; n < b1; ++n) {
      const float tn = tnx;
      if (n + 1 < b1) tnx = ev.time(n + 1);
      if (tn > tprev) {
        for (int k = gs; k < n; ++k) wk.add(slot_of<SPL>(s, ev.id(k)), ev.wt(k));
        wk.decay(tn - tprev);
        tprev = tn;
        gs = n;
      }
    }
    for (int k = gs; k < b1; ++k) wk.add(slot_of<SPL>(s, ev.id(k)), ev.wt(k));
    if (a1 > tprev) wk.decay(a1 - tprev);
#pragma unroll
    for (int jj = 0; jj < MS; ++jj) {
      sm.encR[c * M + src_of<SPL>(s, jj)] = wk.R[jj];
      if (LEARN) sm.encS[c * M + src_of<SPL>(s, jj)] = wk.S[jj];
    }
    return;
  }
  if constexpr (!UsePriv<M>::value) {
    // the d/dalpha sums of this capacity already meet in shared atomics, so
    // the run-to-run order of the sums is not fixed anyway: the chunk's SPL
    // threads take every SPL-th event each and add its contribution to the
    // chunk's state with shared atomics (one exponential per event in all,
    // instead of a walk of every event by every thread of the chunk)
    const unsigned gmask =
        (SPL >= 32) ? 0xffffffffu : (((1u << SPL) - 1u) << ((threadIdx.x & 31) & ~(SPL - 1)));
#pragma unroll
    for (int jj = 0; jj < MS; ++jj) {
      sm.encR[c * M + src_of<SPL>(s, jj)] = 0.f;
      if (LEARN) sm.encS[c * M + src_of<SPL>(s, jj)] = 0.f;
    }
    __syncwarp(gmask);
    for (int n = b0 + s; n < b1; n += SPL) {
      const int u = ev.id(n);
      const float d = a1 - ev.time(n);
      const float we = ev.wt(n) * exp2_acc(-sm.bl2[BM == 0 ? 0 : u] * d);
      atomicAdd(&sm.encR[c * M + u], we);
      if (LEARN) atomicAdd(&sm.encS[c * M + u], we * d);
    }
    __syncwarp(gmask);
    return;
  }
  float R[MS], S[LEARN ? MS : 1];
#pragma unroll
  for (int jj = 0; jj < MS; ++jj) {
    R[jj] = 0.f;
    if (LEARN) S[jj] = 0.f;
  }
  for (int n = b0; n < b1; ++n) {
    const int uid = ev.id(n);
    const int u = slot_of<SPL>(s, uid);
    if ((unsigned)u < (unsigned)MS) {
      const float d = a1 - ev.time(n);
      const float we = ev.wt(n) * exp2_acc(-sm.bl2[BM == 0 ? 0 : uid] * d);
#pragma unroll
      for (int jj = 0; jj < MS; ++jj) {
        if (u == jj) {
          R[jj] += we;
          if (LEARN) S[jj] = fmaf(we, d, S[jj]);
        }
      }
    }
  }
#pragma unroll
  for (int jj = 0; jj < MS; ++jj) {
    sm.encR[c * M + src_of<SPL>(s, jj)] = R[jj];
    if (LEARN) sm.encS[c * M + src_of<SPL>(s, jj)] = S[jj];
  }
}

// Per-source scan over chunks: encR/encS[c] become entering states; the end
// state (at T_span, all events included) goes to endR/endS.
//
// The effect of chunk c on source j's state is the affine map
//   R -> A_c R + r_c,   S -> A_c (S + D_c R) + s_c,   A_c = exp(-beta_j D_c),
// D_c the chunk's length in time and (r_c, s_c) its own contribution (pass 1).
// Such maps compose associatively (g after f):
//   A = A_g A_f,  D = D_f + D_g,  r = A_g r_f + r_g,  s = A_g (s_f + D_g r_f) + s_g,
// so every chunk's entering state is an exclusive scan of the maps applied to
// the zero state.  It runs as a warp-level scan: warp w takes sources w,
// w + (warps), ...; lane l first composes its ceil(NC / 32) consecutive chunks,
// the warp scans the 32 lane aggregates with shuffles (five steps), and each
// lane then walks its own chunks from its exclusive prefix.
template <int M, int BM, bool LEARN>
__device__ __forceinline__ void scan_chunks(int NC, const Sm<M> &sm) {
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int G = (NC + 31) >> 5;
  const int c0 = min(lane * G, NC), c1 = min(c0 + G, NC);
  for (int j = threadIdx.x >> 5; j < M; j += nw) {
    const float b = sm.bl2[BM == 0 ? 0 : j];
    float A = 1.f, D = 0.f, r = 0.f, s = 0.f;  // this lane's chunks, composed
    for (int c = c0; c < c1; ++c) {
      const float Dc = sm.anc[c + 1] - sm.anc[c];
      const float Ac = exp2_acc(-b * Dc);
      if (LEARN) s = fmaf(Ac, fmaf(Dc, r, s), sm.encS[c * M + j]);
      r = fmaf(Ac, r, sm.encR[c * M + j]);
      A *= Ac;
      D += Dc;
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {  // inclusive scan: earlier lanes' maps first
      const float Ap = __shfl_up_sync(0xffffffffu, A, o);
      const float Dp = __shfl_up_sync(0xffffffffu, D, o);
      const float rp = __shfl_up_sync(0xffffffffu, r, o);
      const float sp = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) {
        if (LEARN) s = fmaf(A, fmaf(D, rp, sp), s);
        r = fmaf(A, rp, r);
        A *= Ap;
        D += Dp;
      }
    }
    float R = __shfl_up_sync(0xffffffffu, r, 1);  // state entering this lane's first chunk
    float S = __shfl_up_sync(0xffffffffu, s, 1);
    if (lane == 0) {
      R = 0.f;
      S = 0.f;
    }
    for (int c = c0; c < c1; ++c) {
      const float Dc = sm.anc[c + 1] - sm.anc[c];
      const float Ac = exp2_acc(-b * Dc);
      const float lr = sm.encR[c * M + j];
      const float ls = LEARN ? sm.encS[c * M + j] : 0.f;
      sm.encR[c * M + j] = R;
      if (LEARN) sm.encS[c * M + j] = S;
      if (LEARN) S = fmaf(Ac, fmaf(Dc, R, S), ls);
      R = fmaf(Ac, R, lr);
    }
    if (lane == 31) {  // every chunk composed: the state at T_span
      sm.endR[j] = r;
      if (LEARN) sm.endS[j] = s;
    }
  }
}

// Pass 2 for chunk c: lnL (log2 units, Kahan), d/dmu, d/dalpha, d/dbeta.
template <int M, int SPL, int BM, bool LEARN, typename EV>
__device__ __forceinline__ void pass2_chunk(int c, int s, int b0, int b1, float a0, const EV &ev,
                                            const Sm<M> &sm, float &Ls, float &Lc,
                                            float (&gbl)[LEARN ? M / SPL : 1], float *r_out) {
  constexpr int MS = M / SPL;
  constexpr int NQ = MS / 4;
  constexpr int AP = M + 4;
  constexpr bool PRIV = UsePriv<M>::value;
  const int tid = threadIdx.x;
  const int NT = blockDim.x;
  const int lane = tid & 31;
  const unsigned gmask = (SPL >= 32) ? 0xffffffffu : (((1u << SPL) - 1u) << (lane & ~(SPL - 1)));
  Walker<MS, BM, LEARN> wk;
  wk.template load_beta<SPL>(sm.bl2, s);
#pragma unroll
  for (int jj = 0; jj < MS; ++jj) {
    wk.R[jj] = sm.encR[c * M + src_of<SPL>(s, jj)];
    if (LEARN) wk.S[jj] = sm.encS[c * M + src_of<SPL>(s, jj)];
  }
  float4 *gp = reinterpret_cast<float4 *>(sm.gpriv);
  ev.chunk_begin(c, s, b0, b1, gmask);  // streamed events: start this chunk's copies
  float tprev = a0;
  int gs = b0;
  int pu = 0;
  float pw = 0.f;
  for (int n = b0; n < b1; ++n) {
    float tn;
    int un;
    ev.next(n, tn, un);
    if (tn > tprev) {
      if (n - gs == 1) {
        wk.add(pu, pw);
      } else {
        for (int k = gs; k < n; ++k) wk.add(slot_of<SPL>(s, ev.id(k)), ev.wt(k));
      }
      wk.decay(tn - tprev);
      tprev = tn;
      gs = n;
    }
    pu = slot_of<SPL>(s, un);
    pw = ev.wt(n);
    const float *arow = sm.alpha + un * AP + 4 * s;  // group s + SPL q of the row at step q
    float4 av[NQ];
    float d0 = 0.f, d1 = 0.f;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      av[q] = *reinterpret_cast<const float4 *>(arow + 4 * SPL * q);
      d0 = fmaf(av[q].x, wk.R[4 * q + 0], d0);
      d1 = fmaf(av[q].y, wk.R[4 * q + 1], d1);
      d0 = fmaf(av[q].z, wk.R[4 * q + 2], d0);
      d1 = fmaf(av[q].w, wk.R[4 * q + 3], d1);
    }
    float dot = d0 + d1;
#pragma unroll
    for (int o = 1; o < SPL; o <<= 1) dot += __shfl_xor_sync(gmask, dot, o);
    const float lam = sm.mu[un] + dot;
    const float r = rcp_ftz(lam);
    if (s == 0) {
      kahan_add(Ls, Lc, lg2_ftz(lam));
      if (PRIV) sm.mpriv[un * (NT / SPL) + c] += r;
      else atomicAdd(&sm.gm[un], r);
      if (r_out) r_out[n] = r;
    }
    if (PRIV) {
      float4 *g = gp + (un * NQ) * NT + tid;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        float4 x = g[q * NT];
        x.x = fmaf(r, wk.R[4 * q + 0], x.x);
        x.y = fmaf(r, wk.R[4 * q + 1], x.y);
        x.z = fmaf(r, wk.R[4 * q + 2], x.z);
        x.w = fmaf(r, wk.R[4 * q + 3], x.w);
        g[q * NT] = x;
      }
    } else {
      float *grow = sm.ga + un * ga_pitch(M);
#pragma unroll
      for (int jj = 0; jj < MS; ++jj) atomicAdd(&grow[ga_col(src_of<SPL>(s, jj))], r * wk.R[jj]);
    }
    if (LEARN) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        gbl[4 * q + 0] = fmaf(-r * av[q].x, wk.S[4 * q + 0], gbl[4 * q + 0]);
        gbl[4 * q + 1] = fmaf(-r * av[q].y, wk.S[4 * q + 1], gbl[4 * q + 1]);
        gbl[4 * q + 2] = fmaf(-r * av[q].z, wk.S[4 * q + 2], gbl[4 * q + 2]);
        gbl[4 * q + 3] = fmaf(-r * av[q].w, wk.S[4 * q + 3], gbl[4 * q + 3]);
      }
    }
  }
  ev.chunk_end();
}

// ---------------------------------------------------------------------------
// Window-level phases
// ---------------------------------------------------------------------------

// Stage (optional) and validate the window; counts and weight sums per type.
// Returns the window status (uniform across the CTA).
template <int M, bool STAGE>
__device__ int stage_and_validate(const float *tg, const int16_t *ug, const float *wg, int N,
                                  float T, int Mrt, Sm<M> &sm) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) sm.ctl[0] = 0x7fffffff;
  for (int j = tid; j < M; j += nt) {
    sm.cnt[j] = 0;
    sm.W[j] = 0.0;
  }
  __syncthreads();
  int code = 0x7fffffff;
  if (tid == 0 && (!(T >= 0.f) || !isfinite(T))) code = kE_TIME_RANGE;
#pragma unroll 4
  for (int n = tid; n < N; n += nt) {
    const float tv = tg[n];
    const int uv = (int)ug[n];
    const float wv = wg ? wg[n] : 1.f;
    if (!isfinite(tv) || !isfinite(wv)) code = min(code, (int)kE_NONFINITE);
    if (tv < 0.f || tv > T) code = min(code, (int)kE_TIME_RANGE);
    if (uv < 0 || uv >= Mrt) code = min(code, (int)kE_ID_RANGE);
    if (n > 0 && tv < tg[n - 1]) code = min(code, (int)kE_UNSORTED);
    if (STAGE) {
      sm.ev_t[n] = tv;
      sm.ev_u[n] = (uint16_t)uv;
      if (wg) sm.ev_w[n] = wv;
    }
    if (uv >= 0 && uv < Mrt) {
      atomicAdd(&sm.cnt[uv], 1);
      if (wg) atomicAdd(&sm.W[uv], (double)wv);
    }
  }
  if (code != 0x7fffffff) atomicMin(&sm.ctl[0], code);
  __syncthreads();
  // W_j becomes a double-float in place (the same 8 bytes), so the compensator
  // constants of every iteration need no FP64 arithmetic
  for (int j = tid; j < M; j += nt) {
    const double w = wg ? sm.W[j] : (double)sm.cnt[j];
    const float hi = (float)w;
    reinterpret_cast<float2 *>(sm.W)[j] = make_float2(hi, (float)(w - (double)hi));
  }
  __syncthreads();
  const int st = sm.ctl[0];
  return st == 0x7fffffff ? kOK : st;
}

// Chunk boundaries and anchors (a_c = first time of chunk c, T for an empty tail).
template <typename EV>
__device__ void setup_chunks(int NC, int N, float T, const EV &ev, int *bnd, float *anc) {
  for (int c = threadIdx.x; c <= NC; c += blockDim.x) {
    const int b = chunk_begin(c, NC, N, ev);
    bnd[c] = b;
    anc[c] = (c < NC && b < N) ? ev.time(b) : T;
  }
  __syncthreads();
}

// Pass 1 + scan + compensator constants.  Leaves C, dC, endR, endS in smem.
template <int M, int SPL, int BM, bool LEARN, typename EV>
__device__ void prepare_states(int NC, const EV &ev, int Mrt, Sm<M> &sm) {
  const int tid = threadIdx.x;
  const int c = tid / SPL, s = tid % SPL;
  if (c < NC) {
    pass1_chunk<M, SPL, BM, LEARN>(c, s, sm.bnd[c], sm.bnd[c + 1], sm.anc[c], sm.anc[c + 1], ev,
                                   sm);
  }
  __syncthreads();
  scan_chunks<M, BM, LEARN>(NC, sm);
  __syncthreads();
  for (int j = tid; j < M; j += blockDim.x) {
    if (j < Mrt) {
      // C_j = (W_j - R_j(T)) / beta_j and dC_j = (S_j(T) - C_j) / beta_j in
      // double-float: W_j - R_j(T) cancels for windows that end on a burst
      const float b = sm.beta[BM == 0 ? 0 : j];
      const float2 w = reinterpret_cast<const float2 *>(sm.W)[j];
      const FF Cj = ff_div(ff_add(FF{w.x, w.y}, FF{-sm.endR[j], 0.f}), b);
      sm.C[j] = Cj.hi + Cj.lo;
      if (LEARN) {
        const FF e = ff_add(FF{sm.endS[j], 0.f}, FF{-Cj.hi, -Cj.lo});
        sm.dC[j] = (e.hi + e.lo) / b;
      } else {
        sm.dC[j] = 0.f;
      }
    } else {
      sm.C[j] = 0.f;
      sm.dC[j] = 0.f;
    }
  }
  __syncthreads();
}

// Clear the accumulators pass 2 writes (own private slots, or the shared copy).
template <int M, int SPL>
__device__ __forceinline__ void clear_accumulators(Sm<M> &sm) {
  constexpr int NQ = M / SPL / 4;
  const int tid = threadIdx.x, NT = blockDim.x;
  if (UsePriv<M>::value) {
    float4 *gp = reinterpret_cast<float4 *>(sm.gpriv);
    for (int u = 0; u < M; ++u) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) gp[(u * NQ + q) * NT + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int p = tid; p < M * (NT / SPL); p += NT) sm.mpriv[p] = 0.f;
  } else {
    for (int p = tid; p < M * ga_pitch(M); p += NT) sm.ga[p] = 0.f;
    for (int j = tid; j < M; j += NT) sm.gm[j] = 0.f;
  }
  for (int j = tid; j < M; j += NT) sm.gb[j] = 0.f;
}

// Fixed scalar beta, staged events: replace each staged time by the decay
// factor from the previous event, exp(-beta (t_n - t_{n-1})), and mark the
// first event of every tie group in bit 15 of its id.  One thread per chunk;
// a chunk's first event starts from the entering state and needs no factor.
// Runs once per window, after pass 1 (which still needs the times).
template <int M, int SPL>
__device__ void to_decays(int NC, Sm<M> &sm) {
  const int tid = threadIdx.x;
  const int c = tid / SPL, s = tid % SPL;
  if (c < NC && s == 0) {
    const int b0 = sm.bnd[c], b1 = sm.bnd[c + 1];
    const float b2 = sm.bl2[0];
    float tprev = (b0 < b1) ? sm.ev_t[b0] : 0.f;
    for (int n = b0; n < b1; ++n) {
      const float tn = sm.ev_t[n];
      const float dt = tn - tprev;
      sm.ev_t[n] = exp2_acc(-b2 * dt);
      if (dt > 0.f) sm.ev_u[n] = (uint16_t)(sm.ev_u[n] | 0x8000u);
      tprev = tn;
    }
  }
  __syncthreads();
}

// Pass 2 with precomputed decay factors (fixed scalar beta, staged events).
template <int M, int SPL>
__device__ __forceinline__ void pass2_fixed(int c, int s, int b0, int b1, const float *w,
                                            const Sm<M> &sm, float &Ls, float &Lc, float *r_out) {
  constexpr int MS = M / SPL;
  constexpr int NQ = MS / 4;
  constexpr int AP = M + 4;
  constexpr bool PRIV = UsePriv<M>::value;
  const int tid = threadIdx.x;
  const int NT = blockDim.x;
  const int lane = tid & 31;
  const unsigned gmask = (SPL >= 32) ? 0xffffffffu : (((1u << SPL) - 1u) << (lane & ~(SPL - 1)));
  const float *A = sm.ev_t;
  const uint16_t *U = sm.ev_u;
  Walker<MS, 0, false> wk;
#pragma unroll
  for (int jj = 0; jj < MS; ++jj) wk.R[jj] = sm.encR[c * M + src_of<SPL>(s, jj)];
  float4 *gp = reinterpret_cast<float4 *>(sm.gpriv);
  int gs = b0;
  int pu = 0;
  float pw = 0.f;
  for (int n = b0; n < b1; ++n) {
    const float an = A[n];
    const int cd = (int)U[n];
    const int un = cd & 0x7fff;
    if (cd & 0x8000) {
      if (n - gs == 1) {
        wk.add(pu, pw);
      } else {
        for (int k = gs; k < n; ++k) wk.add(slot_of<SPL>(s, (int)U[k] & 0x7fff), w ? w[k] : 1.f);
      }
#pragma unroll
      for (int jj = 0; jj < MS; ++jj) wk.R[jj] *= an;
      gs = n;
    }
    pu = slot_of<SPL>(s, un);
    pw = w ? w[n] : 1.f;
    const float *arow = sm.alpha + un * AP + 4 * s;  // group s + SPL q of the row at step q
    float d0 = 0.f, d1 = 0.f;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const float4 av = *reinterpret_cast<const float4 *>(arow + 4 * SPL * q);
      d0 = fmaf(av.x, wk.R[4 * q + 0], d0);
      d1 = fmaf(av.y, wk.R[4 * q + 1], d1);
      d0 = fmaf(av.z, wk.R[4 * q + 2], d0);
      d1 = fmaf(av.w, wk.R[4 * q + 3], d1);
    }
    float dot = d0 + d1;
#pragma unroll
    for (int o = 1; o < SPL; o <<= 1) dot += __shfl_xor_sync(gmask, dot, o);
    const float lam = sm.mu[un] + dot;
    const float r = rcp_ftz(lam);
    if (s == 0) {
      kahan_add(Ls, Lc, lg2_ftz(lam));
      if (PRIV) sm.mpriv[un * (NT / SPL) + c] += r;
      else atomicAdd(&sm.gm[un], r);
      if (r_out) r_out[n] = r;
    }
    if (PRIV) {
      float4 *g = gp + (un * NQ) * NT + tid;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        float4 x = g[q * NT];
        x.x = fmaf(r, wk.R[4 * q + 0], x.x);
        x.y = fmaf(r, wk.R[4 * q + 1], x.y);
        x.z = fmaf(r, wk.R[4 * q + 2], x.z);
        x.w = fmaf(r, wk.R[4 * q + 3], x.w);
        g[q * NT] = x;
      }
    } else {
      float *grow = sm.ga + un * ga_pitch(M);
#pragma unroll
      for (int jj = 0; jj < MS; ++jj) atomicAdd(&grow[ga_col(src_of<SPL>(s, jj))], r * wk.R[jj]);
    }
  }
}

// Error-free sum of two floats added into a (hi, lo) pair.
__device__ __forceinline__ void pair_add(float &hi, float &lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (x - bp);
  hi = s;
}

// One lnL + gradient evaluation at the parameters in smem.  The accumulators
// must be clear.  On return (after a barrier) the event sums are complete and
// each warp's compensated partial sums of Part1 (log2 units) and of Part2 +
// Part3 sit in red as float4 (hi1, lo1, hi23, lo23); lnl_total() adds them up.
// FIXED: staged events already converted by to_decays (fixed scalar beta).
template <int M, int SPL, int BM, bool LEARN, bool FIXED, typename EV>
__device__ void evaluate(int NC, const EV &ev, float T, int Mrt, Sm<M> &sm, float *r_out) {
  constexpr int MS = M / SPL;
  constexpr int AP = M + 4;
  const int tid = threadIdx.x;
  const int c = tid / SPL, s = tid % SPL;
  float Ls = 0.f, Lc = 0.f;
  float gbl[LEARN ? MS : 1];
#pragma unroll
  for (int jj = 0; jj < (LEARN ? MS : 1); ++jj) gbl[jj] = 0.f;
  if (c < NC) {
    if (FIXED) {
      pass2_fixed<M, SPL>(c, s, sm.bnd[c], sm.bnd[c + 1], ev.w, sm, Ls, Lc, r_out);
    } else {
      pass2_chunk<M, SPL, BM, LEARN>(c, s, sm.bnd[c], sm.bnd[c + 1], sm.anc[c], ev, sm, Ls, Lc, gbl,
                                     r_out);
    }
    if (LEARN) {
      if (BM == 0) {
        float acc = 0.f;
#pragma unroll
        for (int jj = 0; jj < MS; ++jj) acc += gbl[jj];
        atomicAdd(&sm.gb[0], acc);
      } else {
#pragma unroll
        for (int jj = 0; jj < MS; ++jj) atomicAdd(&sm.gb[src_of<SPL>(s, jj)], gbl[jj]);
      }
    }
  }
  // Part2 and Part3 terms for this thread's share of the parameters
  float Ps = 0.f, Pc = 0.f;
  for (int p = tid; p < Mrt + Mrt * Mrt; p += blockDim.x) {
    if (p < Mrt) {
      kahan_add(Ps, Pc, -T * sm.mu[p]);
    } else {
      const int q = p - Mrt, i = q / Mrt, j = q % Mrt;
      kahan_add(Ps, Pc, -sm.alpha[i * AP + j] * sm.C[j]);
    }
  }
  float h1 = Ls, l1 = -Lc, h2 = Ps, l2 = -Pc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float a = __shfl_xor_sync(0xffffffffu, h1, o), b = __shfl_xor_sync(0xffffffffu, l1, o);
    const float cc = __shfl_xor_sync(0xffffffffu, h2, o), d = __shfl_xor_sync(0xffffffffu, l2, o);
    pair_add(h1, l1, a);
    l1 += b;
    pair_add(h2, l2, cc);
    l2 += d;
  }
  if ((tid & 31) == 0) reinterpret_cast<float4 *>(sm.red)[tid >> 5] = make_float4(h1, l1, h2, l2);
  __syncthreads();
}

// lnL from the per-warp partials (FP64: the only double arithmetic per evaluation).
// lnL from the per-warp partials (Part1 in log2 units, Part2+3) as a double-float.
template <int M>
__device__ __forceinline__ FF lnl_total_ff(const Sm<M> &sm) {
  const int nw = (blockDim.x + 31) >> 5;
  const float4 *r4 = reinterpret_cast<const float4 *>(sm.red);
  FF p1{0.f, 0.f}, p23{0.f, 0.f};
  for (int w = 0; w < nw; ++w) {
    const float4 v = r4[w];
    p1 = ff_add(p1, FF{v.x, v.y});
    p23 = ff_add(p23, FF{v.z, v.w});
  }
  return ff_add(ff_mul(p1, kLn2Hi, kLn2Lo), p23);
}

// The same total formed by one warp: lane l < nw takes warp l's partials and
// four shuffle rounds add them as a tree; lane 0 holds the total (nw <= 16).
__device__ __forceinline__ FF lnl_total_ff_warp(const double *red, int nw) {
  const int lane = threadIdx.x & 31;
  FF p1{0.f, 0.f}, p23{0.f, 0.f};
  if (lane < nw) {
    const float4 v = reinterpret_cast<const float4 *>(red)[lane];
    p1 = FF{v.x, v.y};
    p23 = FF{v.z, v.w};
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    const FF q1{__shfl_down_sync(0xffffffffu, p1.hi, o), __shfl_down_sync(0xffffffffu, p1.lo, o)};
    const FF q23{__shfl_down_sync(0xffffffffu, p23.hi, o), __shfl_down_sync(0xffffffffu, p23.lo, o)};
    p1 = ff_add(p1, q1);
    p23 = ff_add(p23, q23);
  }
  return ff_add(ff_mul(p1, kLn2Hi, kLn2Lo), p23);
}

// The stopping rule |lnL_k - lnL_{k-1}| <= tol |lnL_k| on double-floats.
__device__ __forceinline__ bool ff_small_change(FF cur, FF prev, float tol) {
  const float d = (cur.hi - prev.hi) + (cur.lo - prev.lo);
  return fabsf(d) <= tol * fabsf(cur.hi);
}

template <int M>
__device__ __forceinline__ double lnl_total(const Sm<M> &sm) {
  const int nw = (blockDim.x + 31) >> 5;
  const float4 *r4 = reinterpret_cast<const float4 *>(sm.red);
  double p1 = 0.0, p23 = 0.0;
  for (int w = 0; w < nw; ++w) {
    const float4 v = r4[w];
    p1 += (double)v.x + (double)v.y;
    p23 += (double)v.z + (double)v.w;
  }
  return p1 * kLn2 + p23;
}

// Event sum of d/dalpha_ij (over the private slots, or the shared copy).
template <int M, int SPL>
__device__ __forceinline__ float alpha_event_sum(int i, int j, const Sm<M> &sm) {
  if (UsePriv<M>::value) {
    constexpr int MS = M / SPL;
    constexpr int NQ = MS / 4;
    const int NT = blockDim.x, NC = NT / SPL;
    const int g = j >> 2, s = g % SPL, q = g / SPL, e = j & 3;  // j = src_of(s, 4 q + e)
    const float *base = sm.gpriv + ((i * NQ + q) * NT) * 4 + e;
    float acc = 0.f;
    for (int c = 0; c < NC; ++c) acc += base[(c * SPL + s) * 4];
    return acc;
  }
  return sm.ga[i * ga_pitch(M) + ga_col(j)];
}

template <int M, int SPL>
__device__ __forceinline__ float mu_event_sum(int i, const Sm<M> &sm) {
  if (UsePriv<M>::value) {
    const int NC = blockDim.x / SPL;
    float acc = 0.f;
    for (int c = 0; c < NC; ++c) acc += sm.mpriv[i * NC + c];
    return acc;
  }
  return sm.gm[i];
}

// Final gradient of parameter p (compact index: mu | alpha | beta).
template <int M, int SPL, int BM, bool LEARN>
__device__ __forceinline__ float grad_of(int p, int Mrt, float T, const Sm<M> &sm) {
  constexpr int AP = M + 4;
  if (p < Mrt) return mu_event_sum<M, SPL>(p, sm) - T;
  const int q = p - Mrt;
  if (q < Mrt * Mrt) {
    const int i = q / Mrt, j = q % Mrt;
    return alpha_event_sum<M, SPL>(i, j, sm) - sm.C[j];
  }
  if (!LEARN) return 0.f;
  const int jb = q - Mrt * Mrt;
  if (BM == 0) {
    float acc = sm.gb[0];
    for (int j = 0; j < Mrt; ++j) {
      float col = 0.f;
      for (int i = 0; i < Mrt; ++i) col += sm.alpha[i * AP + j];
      acc -= col * sm.dC[j];
    }
    return acc;
  }
  float col = 0.f;
  for (int i = 0; i < Mrt; ++i) col += sm.alpha[i * AP + jb];
  return sm.gb[jb] - col * sm.dC[jb];
}

template <int M>
__device__ __forceinline__ float &param_ref(int p, int Mrt, Sm<M> &sm) {
  constexpr int AP = M + 4;
  if (p < Mrt) return sm.mu[p];
  const int q = p - Mrt;
  if (q < Mrt * Mrt) return sm.alpha[(q / Mrt) * AP + (q % Mrt)];
  return sm.beta[q - Mrt * Mrt];
}

}  // namespace mdhp
