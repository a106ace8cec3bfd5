"""Tensor-core BF16 GEMM (mdhp_gemm_bf16, tcgen05.mma with accumulators in
tensor memory; engine 0: operands loaded by the tensor-memory accelerator
when both are K-contiguous, engine 2: per-thread 16-byte copies) against an
FP64 product of the same BF16 operands.

Bound: FP32 accumulation of K products in any order is within
K * 2^-24 * sum_k |a_mk b_kn| of the exact sum (each partial sum rounds once);
the test allows twice that, plus the final BF16 rounding (2^-8 relative) for
the BF16 output.  Covered: one tile with one K-block, N not a multiple of the
256 tile width (column tiles of 144), rows not a multiple of 128, every pair
of operand majors, the K split (partial tiles added with atomics, then bias,
ReLU and the BF16 copy; with TMA operands the split CTAs form a cluster that
sums the partial tiles through distributed shared memory, clusters of 3 to 8;
pairs of row tiles that share each weight box by multicast, with a padding
row tile when their count is odd),
accumulation into C, agreement with the warp-level
MMA engine, the initializer's largest layer (4096 x 256 x 8256), and the
unsupported layouts that are refused."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mdhp():
    import paper_2411_10258_gb300 as m
    from paper_2411_10258_gb300 import api

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return api


def _operands(M, N, K, a_mn, b_mn, seed):
    g = torch.Generator().manual_seed(seed)
    A = (torch.rand(M, K, generator=g) * 2 - 1).to(torch.bfloat16)
    B = (torch.rand(N, K, generator=g) * 2 - 1).to(torch.bfloat16)
    Ad = (A.t().contiguous() if a_mn else A).cuda()
    Bd = (B.t().contiguous() if b_mn else B).cuda()
    return A, B, Ad, Bd


def _ref(A, B):
    a, b = A.double(), B.double()
    return a @ b.t(), a.abs() @ b.abs().t()


def _check(C, ref, mag, K, extra=0.0):
    err = (C.double().cpu() - ref).abs()
    bound = 2.0 * K * 2.0 ** -24 * mag + extra * ref.abs() + 1e-30
    bad = err > bound
    assert not bool(bad.any()), (int(bad.sum()), float((err / (mag + 1e-30)).max()))


def _gemm(mdhp, Ad, Bd, M, N, K, a_mn, b_mn, engine=0, **kw):
    C = torch.full((M, N), float("nan"), device="cuda")
    mdhp.gemm_bf16(Ad, Bd, M, N, K, a_mn=a_mn, b_mn=b_mn, C=C, engine=engine, **kw)
    assert mdhp.gemm_check() == 0
    return C


@pytest.mark.parametrize("engine", [2, 0])
def test_tc_smallest_tile(mdhp, engine):
    """One CTA, one K-block of 64, N = 16: the descriptors and the tensor-memory round trip."""
    M, N, K = 128, 16, 64
    A, B, Ad, Bd = _operands(M, N, K, False, False, 1)
    C = _gemm(mdhp, Ad, Bd, M, N, K, False, False, engine=engine)
    ref, mag = _ref(A, B)
    _check(C, ref, mag, K)


@pytest.mark.parametrize("engine", [0, 2])
@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (256, 256, 512), (300, 272, 1000), (64, 48, 8),
                                   (130, 40, 200), (384, 256, 512)])
def test_tc_shapes(mdhp, M, N, K, engine):
    A, B, Ad, Bd = _operands(M, N, K, False, False, M + N + K)
    C = _gemm(mdhp, Ad, Bd, M, N, K, False, False, engine=engine)
    ref, mag = _ref(A, B)
    _check(C, ref, mag, K)


@pytest.mark.parametrize("a_mn,b_mn", [(0, 1), (1, 0), (1, 1)])
def test_tc_operand_majors(mdhp, a_mn, b_mn):
    M, N, K = 256, 144, 320
    A, B, Ad, Bd = _operands(M, N, K, a_mn, b_mn, 7 + 2 * a_mn + b_mn)
    C = _gemm(mdhp, Ad, Bd, M, N, K, a_mn, b_mn)
    ref, mag = _ref(A, B)
    _check(C, ref, mag, K)


@pytest.mark.parametrize("engine", [0, 2])
def test_tc_split_k_bias_relu_bf16(mdhp, engine):
    """Few tiles and a long K: the product is split over CTAs (atomics into C),
    then bias, ReLU and the BF16 copy."""
    M, N, K = 256, 256, 4096
    A, B, Ad, Bd = _operands(M, N, K, False, False, 11)
    bias = (torch.rand(N) - 0.5).float().cuda()
    C = torch.empty(M, N, device="cuda")
    Cb = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    mdhp.gemm_bf16(Ad, Bd, M, N, K, bias=bias, relu=True, C=C, C_bf16=Cb, engine=engine)
    assert mdhp.gemm_check() == 0
    ref, mag = _ref(A, B)
    ref = torch.clamp(ref + bias.double().cpu(), min=0.0)
    _check(C, ref, mag, K)
    _check(Cb.float(), ref, mag, K, extra=2.0 ** -8)


@pytest.mark.parametrize("M,N,K", [(128, 272, 128), (256, 256, 4096)])
def test_tc_accumulate_kmajor(mdhp, M, N, K):
    """Accumulation into C, TMA operands: without a split, and with K split
    over a cluster that sums its partial tiles before adding them."""
    A, B, Ad, Bd = _operands(M, N, K, False, False, 15)
    C0 = (torch.rand(M, N) - 0.5).float()
    C = C0.clone().cuda()
    mdhp.gemm_bf16(Ad, Bd, M, N, K, C=C, accumulate=True, engine=0)
    assert mdhp.gemm_check() == 0
    ref, mag = _ref(A, B)
    _check(C, ref + C0.double(), mag + C0.double().abs(), K)


def test_tc_accumulate(mdhp):
    M, N, K = 144, 272, 512
    A, B, Ad, Bd = _operands(M, N, K, True, True, 12)
    C0 = (torch.rand(M, N) - 0.5).float()
    C = C0.clone().cuda()
    mdhp.gemm_bf16(Ad, Bd, M, N, K, a_mn=True, b_mn=True, C=C, accumulate=True, engine=0)
    assert mdhp.gemm_check() == 0
    ref, mag = _ref(A, B)
    _check(C, ref + C0.double(), mag + C0.double().abs(), K)


def test_tc_matches_mma_engine(mdhp):
    M, N, K = 512, 256, 1024
    A, B, Ad, Bd = _operands(M, N, K, False, False, 13)
    ref, mag = _ref(A, B)
    for engine in (0, 1, 2):
        _check(_gemm(mdhp, Ad, Bd, M, N, K, False, False, engine=engine), ref, mag, K)


def test_tc_largest_initializer_layer(mdhp):
    """4096 windows x 8256 features -> 256 hidden units (M = 16 initializer's first layer)."""
    M, N, K = 4096, 256, 8256
    A, B, Ad, Bd = _operands(M, N, K, False, False, 14)
    C = _gemm(mdhp, Ad, Bd, M, N, K, False, False)
    rows = torch.arange(0, M, 37)
    ref, mag = _ref(A[rows], B)
    _check(C[rows.cuda()], ref, mag, K)


def test_tc_refuses_unsupported_layouts(mdhp):
    from paper_2411_10258_gb300 import _lib

    A = torch.zeros(128, 12, dtype=torch.bfloat16, device="cuda")
    B = torch.zeros(16, 12, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(128, 16, device="cuda")
    with pytest.raises(_lib.MdhpError):  # K = 12 is not a multiple of 8
        mdhp.gemm_bf16(A, B, 128, 16, 12, C=C, engine=0)
    # the warp-level MMA engine takes it
    mdhp.gemm_bf16(A, B, 128, 16, 12, C=C, engine=1)
    torch.cuda.synchronize()
    assert float(C.abs().max()) == 0.0
