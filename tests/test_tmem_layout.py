"""Index arithmetic of the tensor-memory feature store, checked on the host.

Replays the formulas of the decoupled fit with feature store 1-3: the host's
sizing in mdhp_fit_batch (csrc/mdhp_api.cu: columns per CTA from the
occupancy, the shared-memory tier from what the carve leaves) and the
kernel's mapping in k_fit_x (csrc/mdhp_fitx.cuh: lane = thread mod 128 in
its warp's quarter, threads sharing a lane split its columns, steps of M
columns, the global scratch slot of (xcap + 768) rows in step-major order).
It checks that every access stays inside what was allocated and that no
two threads touch the same tensor-memory cell, for every block size the
kernel is built for and every occupancy the host could see."""
import pytest

M = 32  # the template width the tensor-memory kernels are built for
SMEM_SM = 233472  # shared memory per SM on sm_100-class parts (bytes)
MAX_DYN = 232448  # largest dynamic shared memory per CTA (bytes)


def host_sizing(nt, occ, carve, store):
    """mdhp_fit_batch: (tmem_cols, smem_steps, dynamic smem) or None if rejected."""
    cols = 512
    while cols > 32 and cols * max(occ, 1) > 512:
        cols >>= 1
    sets = max(nt // 128, 1)
    if cols * max(occ, 1) > 512 or cols // sets < M:
        return None
    dyn = carve
    steps = 0
    if store >= 2:
        step_bytes = M * 4 * nt
        room = min(SMEM_SM // max(occ, 1) - 1024, MAX_DYN) - dyn
        steps = max(0, min(room // step_bytes, 64))
        dyn += steps * step_bytes
    return cols, steps, dyn


def kernel_rows(nt, cols):
    """k_fit_x: per thread (lane, first column, steps in tensor memory)."""
    share = cols // (nt // 128) // M * M if nt > 128 else cols
    rows = []
    for tid in range(nt):
        warp, lane_in_warp = tid >> 5, tid & 31
        lane = 32 * (warp & 3) + lane_in_warp
        rows.append((lane, (tid >> 7) * share, share // M))
    return rows


@pytest.mark.parametrize("nt", [128, 256, 384])
@pytest.mark.parametrize("occ", [1, 2, 3, 4])
@pytest.mark.parametrize("store", [1, 2, 3])
def test_tensor_memory_cells_are_private_and_allocated(nt, occ, store):
    carve = 100 * 1024 if nt <= 256 else 136 * 1024
    if occ * (carve + 1024) > SMEM_SM:
        return  # the occupancy calculator never reports more CTAs than the carve allows
    sized = host_sizing(nt, occ, carve, store)
    if sized is None:
        return  # the host reports MDHP_E_UNSUPPORTED and launches nothing
    cols, steps, dyn = sized
    assert cols in (32, 64, 128, 256, 512) and cols * occ <= 512
    assert dyn <= MAX_DYN and dyn + 1024 <= SMEM_SM // occ  # the occupancy holds
    owner = {}
    for tid, (lane, c0, tsteps) in enumerate(kernel_rows(nt, cols)):
        assert 0 <= lane < 128
        # a warp touches only the lanes of its quarter
        assert lane // 32 == (tid >> 5) % 4
        assert tsteps >= 1
        for k in range(tsteps):
            first = c0 + k * M
            assert first % M == 0 or nt <= 128  # steps start on a step boundary
            for col in range(first, first + M):
                assert 0 <= col < cols, (tid, col, cols)
                assert (lane, col) not in owner, ((lane, col), owner.get((lane, col)), tid)
                owner[(lane, col)] = tid


@pytest.mark.parametrize("nt", [64, 128, 256, 384])
def test_scratch_slot_holds_every_step(nt):
    """Thread t's step k of a window of N events sits at ((k NQ + q) NT + t)
    in a slot of (xcap + 768) rows of NQ float4: the odd step count L
    (ceil(N / NT) | 1) never runs past the slot, for windows up to xcap."""
    nq = M // 4
    for xcap in (100, 1000, 10000, 100000):
        for n in sorted(set([0, 1, nt - 1, nt, nt + 1, xcap // 2, xcap - 1, xcap])):
            if n > xcap:
                continue
            L = max(((n + nt - 1) // nt) | 1, 1)
            last = ((L - 1) * nq + nq - 1) * nt + nt - 1
            assert last < (xcap + 768) * nq, (nt, xcap, n)


def test_store3_keeps_fewer_but_more_threads():
    """The 384-thread kernel (store 3) gets 5 steps per thread from 512 columns
    shared by three threads per lane; the 256-thread one gets 8."""
    r384 = kernel_rows(384, 512)
    r256 = kernel_rows(256, 512)
    assert {s for _, _, s in r384} == {5}
    assert {s for _, _, s in r256} == {8}
    assert max(c0 for _, c0, _ in r384) + 5 * M <= 512
