// Learned warm start for MDHP-GDS: per-window features, a 4-layer BF16 MLP
// (FP32 accumulate) trained on the GPU by the kernels below, and a head that
// maps its output to a starting point (mu, alpha) for the fit.  The paper has
// no initializer; the fit it starts is the paper's (Sec. IV-B).
//
// Features of a window (K = M + 32 M^2 + 3 values, zero-padded to K0):
//   N_i / N                          event share of each type
//   h_ij[b], b = 0..31               for every event of type i, the gap to the
//                                    last earlier event of type j (strictly
//                                    earlier: a tie group does not see
//                                    itself), as bin floor(log2(gap N / T)) + 16
//                                    clamped to [0, 31]; each (i, j) histogram
//                                    divided by its total
//   log N, log T, beta
// Network: X [B, K0] -> 4 layers (ReLU between) -> Y [B, M + M^2].
// Head:    mu_i = mu_cold_i exp(clamp(y_i, -6, 6)), alpha_ij = (beta / M) softplus(y_ij),
//          mu_cold the fit's cold start 0.5 max(N_i, 1) / T.
// Loss (training, per window): sum_i (y_i - clamp(log(mu*_i / mu_cold_i), -6, 6))^2 +
//          sum_ij (softplus(y_ij) - alpha*_ij M / beta)^2, averaged over windows.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "mdhp.h"
#include "mdhp_dispatch.h"

namespace mdhp {

constexpr int kBins = 32;

// tensor-core GEMM (mdhp_gemm_tc.cu)
bool gemm_tc_supported(const void *A, int64_t lda, int a_mn, const void *B, int64_t ldb, int b_mn, int Mm,
                       int Nn, int Kk);
// staging 0: TMA boxes for K-major operands (else per-thread 16-byte copies); 1: always the copies
mdhp_status gemm_tc(const __nv_bfloat16 *A, int64_t lda, int a_mn, const __nv_bfloat16 *B, int64_t ldb,
                    int b_mn, int Mm, int Nn, int Kk, const float *bias, int relu, float *Cf,
                    __nv_bfloat16 *Cb, int64_t ldc, int accumulate, int split, cudaStream_t st,
                    int staging);
int gemm_tc_launches(int Mm, int Nn, int Kk, int accumulate, int split, int a_mn, int b_mn, int staging);

__host__ __device__ inline int init_k0(int M) {
  const int K = M + kBins * M * M + 3;
  return (K + 63) / 64 * 64;
}

// ---------------------------------------------------------------------------
// Features.  One CTA per window, NT threads = NT chunks of the window.
// PACK: two 16-bit bin counters per 32-bit word (half the shared memory, so
// two CTAs of 256 threads fit an SM at M = 32); taken when the batch states
// max_events < 65,536, since no bin then exceeds 65,535 counts.  A window
// longer than that bound gets an all-zero histogram block (its shares, log N,
// log T and beta are still set).
// ---------------------------------------------------------------------------
constexpr int kFeatThreads = 256;

template <int M, bool PACK>
__device__ __forceinline__ int hist_count(const uint32_t *hist, int q) {
  return PACK ? (int)((hist[q >> 1] >> ((q & 1) * 16)) & 0xFFFFu) : (int)hist[q];
}

template <int M, bool PACK>
__global__ void __launch_bounds__(kFeatThreads) k_features(const int64_t *offsets, const float *t,
                                                           const int16_t *id, const float *Tspan,
                                                           const float *beta, int beta_stride, int Mrt,
                                                           int K0, __nv_bfloat16 *X, float *aux) {
  static_assert((M & (M - 1)) == 0 && kBins == 32, "power-of-two M, 32 bins");
  constexpr int kWords = PACK ? M * M * kBins / 2 : M * M * kBins;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *hist = reinterpret_cast<uint32_t *>(smem);                 // [M][M][kBins] counts
  float *lastc = reinterpret_cast<float *>(hist + kWords);             // [NT][M]
  int *cnt = reinterpret_cast<int *>(lastc + blockDim.x * M);          // [M]
  float *invtot = reinterpret_cast<float *>(cnt + M);                  // [M][M]
  const int b = blockIdx.x, tid = threadIdx.x, NT = blockDim.x;
  const int64_t o0 = offsets[b];
  const int N = (int)(offsets[b + 1] - o0);
  const float T = Tspan[b];
  const float *tt = t + o0;
  const int16_t *uu = id + o0;
  const bool hist_on = !PACK || N < 65536;
  for (int p = tid; p < kWords / 4; p += NT) reinterpret_cast<uint4 *>(hist)[p] = make_uint4(0, 0, 0, 0);
  for (int j = tid; j < M; j += NT) cnt[j] = 0;
  __syncthreads();
  // chunk c = [b0, b1), boundaries moved past tie groups
  const int c = tid;
  int b0 = (int)(((long long)c * N) / NT), b1 = (int)(((long long)(c + 1) * N) / NT);
  while (b0 > 0 && b0 < N && tt[b0] == tt[b0 - 1]) ++b0;
  while (b1 > 0 && b1 < N && tt[b1] == tt[b1 - 1]) ++b1;
  if (c == NT - 1) b1 = N;
  // last time of each type inside the chunk
  float lt[M];
#pragma unroll
  for (int j = 0; j < M; ++j) lt[j] = -INFINITY;
  for (int n = b0; n < b1; ++n) {
    const int u = (int)uu[n];
    if (u >= 0 && u < Mrt) {
#pragma unroll
      for (int j = 0; j < M; ++j) lt[j] = (j == u) ? tt[n] : lt[j];
      atomicAdd(&cnt[u], 1);
    }
  }
#pragma unroll
  for (int j = 0; j < M; ++j) lastc[c * M + j] = lt[j];
  __syncthreads();
  if (tid < M) {  // exclusive running max over chunks
    float run = -INFINITY;
    for (int cc = 0; cc < NT; ++cc) {
      const float v = lastc[cc * M + tid];
      lastc[cc * M + tid] = run;
      run = fmaxf(run, v);
    }
  }
  __syncthreads();
  // histogram walk: gaps to the last earlier event of every type
#pragma unroll
  for (int j = 0; j < M; ++j) lt[j] = lastc[c * M + j];
  const float scale = (T > 0.f && N > 0) ? (float)N / T : 1.f;
  int gs = b0;
  float tcur = (b0 < b1) ? tt[b0] : 0.f;
  for (int n = hist_on ? b0 : b1; n < b1; ++n) {
    const float tn = tt[n];
    if (tn > tcur) {  // the previous tie group becomes history
      for (int k = gs; k < n; ++k) {
        const int u = (int)uu[k];
#pragma unroll
        for (int j = 0; j < M; ++j) lt[j] = (j == u) ? tt[k] : lt[j];
      }
      tcur = tn;
      gs = n;
    }
    const int i = (int)uu[n];
    if (i < 0 || i >= Mrt) continue;
#pragma unroll
    for (int j = 0; j < M; ++j) {
      if (j < Mrt && lt[j] > -INFINITY) {
        const float gap = (tn - lt[j]) * scale;
        // floor(log2(gap)) of a positive float is its exponent (subnormals
        // and the clamp below both land in bin 0)
        int bin = gap > 0.f ? ((__float_as_int(gap) >> 23) & 0xff) - 127 + kBins / 2 : 0;
        bin = bin < 0 ? 0 : (bin >= kBins ? kBins - 1 : bin);
        const int q = (i * M + j) * kBins + bin;
        if (PACK) atomicAdd(&hist[q >> 1], 1u << ((q & 1) * 16));
        else atomicAdd(&hist[q], 1u);
      }
    }
  }
  __syncthreads();
  for (int pair = tid; pair < M * M; pair += NT) {  // row totals of each histogram, once
    int tot = 0;
    for (int k = 0; k < kBins; ++k) tot += hist_count<M, PACK>(hist, pair * kBins + k);
    invtot[pair] = tot > 0 ? 1.f / (float)tot : 0.f;
  }
  __syncthreads();
  // the row, eight BF16 values (one 16-byte store) per step; K0 % 64 == 0
  uint4 *row = reinterpret_cast<uint4 *>(X + (size_t)b * K0);
  const float invN = N > 0 ? 1.f / (float)N : 0.f;
  constexpr int kHist0 = M, kHist1 = M + M * M * kBins;
  for (int v8 = tid; v8 < K0 / 8; v8 += NT) {
    uint32_t packed[4];
#pragma unroll
    for (int e2 = 0; e2 < 4; ++e2) {
      float two[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = v8 * 8 + e2 * 2 + h;
        float v = 0.f;
        if (p < Mrt) {
          v = (float)cnt[p] * invN;
        } else if (p >= kHist0 && p < kHist1) {
          const int q = p - kHist0, pair = q / kBins;
          const int i = pair / M, j = pair % M;
          if (i < Mrt && j < Mrt) v = (float)hist_count<M, PACK>(hist, q) * invtot[pair];
        } else if (p == kHist1) {
          v = logf((float)(N > 0 ? N : 1));
        } else if (p == kHist1 + 1) {
          v = logf(T > 0.f ? T : 1.f);
        } else if (p == kHist1 + 2) {
          v = beta[(int64_t)b * beta_stride];
        }
        two[h] = v;
      }
      const __nv_bfloat162 bb = __floats2bfloat162_rn(two[0], two[1]);
      packed[e2] = *reinterpret_cast<const uint32_t *>(&bb);
    }
    row[v8] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
  }
  for (int i = tid; i < Mrt; i += NT) aux[(int64_t)b * Mrt + i] = 0.5f * (float)max(cnt[i], 1) / T;
}

// ---------------------------------------------------------------------------
// BF16 GEMM on the tensor cores (mma.sync m16n8k16, FP32 accumulate).
// C[m][n] = sum_k A(m,k) B(k,n), A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn].
// CTA tile 64 x 64 x 32, 4 warps of 32 x 32.  Epilogue: + bias[n], ReLU,
// FP32 and/or BF16 output (row-major, ldc), or accumulate into FP32.
// ---------------------------------------------------------------------------
struct GemmArgs {
  const __nv_bfloat16 *A, *B;
  int64_t sam, sak, sbk, sbn;
  int Mm, Nn, Kk;
  const float *bias;
  int relu, accumulate;
  int vec_a, vec_b;  // k contiguous and 8-aligned: vectorised tile loads
  float *Cf;
  __nv_bfloat16 *Cb;
  int64_t ldc;
};

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4],
                                               const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Epilogue of a warp's 32 x 32 accumulator block at (mb, nb).
__device__ __forceinline__ void gemm_epilogue(const GemmArgs &g, const float (&acc)[2][4][4],
                                              int mb, int nb, int grp, int tig) {
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = mb + a * 16 + grp + h * 8;
        if (m >= g.Mm) continue;
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const int n = nb + b * 8 + tig * 2 + cc;
          if (n >= g.Nn) continue;
          float v = acc[a][b][h * 2 + cc];
          const int64_t o = (int64_t)m * g.ldc + n;
          if (g.accumulate) {
            g.Cf[o] += v;
            continue;
          }
          if (g.bias) v += g.bias[n];
          if (g.relu) v = fmaxf(v, 0.f);
          if (g.Cf) g.Cf[o] = v;
          if (g.Cb) g.Cb[o] = __float2bfloat16(v);
        }
      }
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? 16 : 0;  // 0 source bytes: the 16 bytes are zero-filled
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

// Both operands k-contiguous (A [m][k], B [n][k], rows 16-byte aligned, K a
// multiple of 8): 64 x 64 x 64 tiles, a 3-stage cp.async pipeline (loads for
// tile t + 2 in flight while tile t is multiplied), fragments by ldmatrix.
constexpr int kGemmStages = 3, kGemmBK = 64, kGemmPad = 8;
constexpr int kGemmRow = kGemmBK + kGemmPad;  // bf16 per shared row (144 bytes: conflict-free ldmatrix)
constexpr int kGemmSmem = kGemmStages * 2 * 64 * kGemmRow * 2;

__global__ void __launch_bounds__(128) k_gemm_bf16_kk(GemmArgs g) {
  extern __shared__ __align__(16) unsigned char gsm[];
  __nv_bfloat16 *As = reinterpret_cast<__nv_bfloat16 *>(gsm);     // [stage][64][kGemmRow]
  __nv_bfloat16 *Bs = As + kGemmStages * 64 * kGemmRow;            // [stage][64][kGemmRow]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int grp = lane >> 2, tig = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  const int nk = (g.Kk + kGemmBK - 1) / kGemmBK;
  auto load_tile = [&](int t, int stage) {
    const int k0 = t * kGemmBK;
    __nv_bfloat16 *as = As + stage * 64 * kGemmRow, *bs = Bs + stage * 64 * kGemmRow;
#pragma unroll
    for (int e = tid; e < 64 * kGemmBK / 8; e += 128) {  // 4 chunks of 16 bytes per thread
      const int r = e >> 3, kk = (e & 7) * 8;
      const int k = k0 + kk, m = m0 + r, n = n0 + r;
      const bool va = m < g.Mm && k < g.Kk, vb = n < g.Nn && k < g.Kk;
      cp_async16(as + r * kGemmRow + kk, va ? g.A + (int64_t)m * g.sam + k : g.A, va);
      cp_async16(bs + r * kGemmRow + kk, vb ? g.B + (int64_t)n * g.sbn + k : g.B, vb);
    }
  };
#pragma unroll
  for (int st = 0; st < kGemmStages - 1; ++st) {
    if (st < nk) load_tile(st, st);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  for (int t = 0; t < nk; ++t) {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kGemmStages - 2) : "memory");
    __syncthreads();  // tile t landed for every thread; tile t - 1's buffer is free
    if (t + kGemmStages - 1 < nk) load_tile(t + kGemmStages - 1, (t + kGemmStages - 1) % kGemmStages);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    const __nv_bfloat16 *as = As + (t % kGemmStages) * 64 * kGemmRow;
    const __nv_bfloat16 *bs = Bs + (t % kGemmStages) * 64 * kGemmRow;
#pragma unroll
    for (int ks = 0; ks < kGemmBK; ks += 16) {
      uint32_t af[2][4], bq[2][4];
#pragma unroll
      for (int a = 0; a < 2; ++a)  // rows wm + 16a .. +15, k ks .. ks + 15
        ldsm_x4(af[a], as + (wm + a * 16 + (lane & 7) + ((lane >> 3) & 1) * 8) * kGemmRow + ks +
                           (lane >> 4) * 8);
#pragma unroll
      for (int bb = 0; bb < 2; ++bb)  // n wn + 16bb .. +15 as two n8 tiles, k ks .. ks + 15
        ldsm_x4(bq[bb], bs + (wn + bb * 16 + (lane & 7) + (lane >> 4) * 8) * kGemmRow + ks +
                            ((lane >> 3) & 1) * 8);
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const uint32_t bf[2] = {bq[b >> 1][(b & 1) * 2], bq[b >> 1][(b & 1) * 2 + 1]};
          mma_bf16_16816(acc[a][b], af[a], bf);
        }
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  gemm_epilogue(g, acc, m0 + wm, n0 + wn, grp, tig);
}

__global__ void __launch_bounds__(128) k_gemm_bf16(GemmArgs g) {
  constexpr int BM = 64, BN = 64, BK = 32, PAD = 8;
  __shared__ __align__(16) __nv_bfloat16 As[BM][BK + PAD];
  __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + PAD];  // [n][k]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int grp = lane >> 2, tig = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  const __nv_bfloat16 zero = __float2bfloat16(0.f);
  // 16-byte loads when k is the contiguous dimension (8 bf16 per load); the
  // host only sets vec_* when strides and sizes are multiples of 8
  for (int k0 = 0; k0 < g.Kk; k0 += BK) {
    if (g.vec_a) {
      for (int e = tid; e < BM * BK / 8; e += 128) {
        const int r = e / (BK / 8), kk = (e % (BK / 8)) * 8;
        const int m = m0 + r, k = k0 + kk;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (m < g.Mm && k < g.Kk) v = *reinterpret_cast<const uint4 *>(g.A + (int64_t)m * g.sam + k);
        *reinterpret_cast<uint4 *>(&As[r][kk]) = v;
      }
    } else {
      for (int e = tid; e < BM * BK; e += 128) {
        const int r = e / BK, kk = e % BK;
        const int m = m0 + r, k = k0 + kk;
        As[r][kk] = (m < g.Mm && k < g.Kk) ? g.A[(int64_t)m * g.sam + (int64_t)k * g.sak] : zero;
      }
    }
    if (g.vec_b) {
      for (int e = tid; e < BN * BK / 8; e += 128) {
        const int r = e / (BK / 8), kk = (e % (BK / 8)) * 8;
        const int n = n0 + r, k = k0 + kk;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (n < g.Nn && k < g.Kk) v = *reinterpret_cast<const uint4 *>(g.B + (int64_t)n * g.sbn + k);
        *reinterpret_cast<uint4 *>(&Bs[r][kk]) = v;
      }
    } else {
      for (int e = tid; e < BN * BK; e += 128) {
        const int r = e / BK, kk = e % BK;
        const int n = n0 + r, k = k0 + kk;
        Bs[r][kk] = (n < g.Nn && k < g.Kk) ? g.B[(int64_t)k * g.sbk + (int64_t)n * g.sbn] : zero;
      }
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < BK; ks += 16) {
      uint32_t af[2][4], bfr[4][2];
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int r = wm + a * 16 + grp;
        af[a][0] = *reinterpret_cast<const uint32_t *>(&As[r][ks + tig * 2]);
        af[a][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][ks + tig * 2]);
        af[a][2] = *reinterpret_cast<const uint32_t *>(&As[r][ks + tig * 2 + 8]);
        af[a][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][ks + tig * 2 + 8]);
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int n = wn + b * 8 + grp;
        bfr[b][0] = *reinterpret_cast<const uint32_t *>(&Bs[n][ks + tig * 2]);
        bfr[b][1] = *reinterpret_cast<const uint32_t *>(&Bs[n][ks + tig * 2 + 8]);
      }
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) mma_bf16_16816(acc[a][b], af[a], bfr[b]);
    }
    __syncthreads();
  }
  gemm_epilogue(g, acc, m0 + wm, n0 + wn, grp, tig);
}

// ---------------------------------------------------------------------------
// Small kernels of the training step
// ---------------------------------------------------------------------------
__device__ __forceinline__ float softplusf(float x) { return x > 20.f ? x : log1pf(expf(x)); }
__device__ __forceinline__ float sigmoidf_(float x) { return 1.f / (1.f + expf(-x)); }

// Head: y [B, O] -> mu [B, M], alpha [B, M, M].
__global__ void k_init_head(const float *Y, int O, const float *aux, const float *beta,
                            int beta_stride, int Mrt, int Bn, float *mu, float *alpha) {
  const int b = blockIdx.x;
  if (b >= Bn) return;
  const float *y = Y + (size_t)b * O;
  for (int i = threadIdx.x; i < Mrt; i += blockDim.x) {
    const float z = fminf(fmaxf(y[i], -6.f), 6.f);
    mu[(int64_t)b * Mrt + i] = aux[(int64_t)b * Mrt + i] * expf(z);
  }
  for (int p = threadIdx.x; p < Mrt * Mrt; p += blockDim.x) {
    const int j = p % Mrt;
    const float bj = beta[(int64_t)b * beta_stride + (beta_stride == 1 ? 0 : j)];
    alpha[(int64_t)b * Mrt * Mrt + p] = bj / (float)Mrt * softplusf(y[Mrt + p]);
  }
}

// Loss and dL/dY (FP32 and BF16 copies); loss summed into *loss (atomic).
__global__ void k_init_loss(const float *Y, int O, const float *aux, const float *beta,
                            int beta_stride, int Mrt, int Bn, const float *mu_t,
                            const float *alpha_t, float *dY, __nv_bfloat16 *dYb, float *loss) {
  const int b = blockIdx.x;
  if (b >= Bn) return;
  const float inv = 1.f / (float)Bn;
  float acc = 0.f;
  for (int p = threadIdx.x; p < O; p += blockDim.x) {
    float d = 0.f;
    const float y = Y[(size_t)b * O + p];
    if (p < Mrt) {
      const float z = fminf(fmaxf(logf(fmaxf(mu_t[(int64_t)b * Mrt + p], 1e-20f) / aux[(int64_t)b * Mrt + p]),
                                  -6.f), 6.f);
      const float e = y - z;
      acc += e * e;
      d = 2.f * e * inv;
    } else if (p < Mrt + Mrt * Mrt) {
      const int q = p - Mrt, j = q % Mrt;
      const float bj = beta[(int64_t)b * beta_stride + (beta_stride == 1 ? 0 : j)];
      const float a = alpha_t[(int64_t)b * Mrt * Mrt + q] * (float)Mrt / bj;
      const float e = softplusf(y) - a;
      acc += e * e;
      d = 2.f * e * sigmoidf_(y) * inv;
    }
    dY[(size_t)b * O + p] = d;
    dYb[(size_t)b * O + p] = __float2bfloat16(d);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc * inv);
}

// dH = dH * (H > 0) in place (FP32) plus a BF16 copy.
__global__ void k_relu_bwd(float *dH, const float *H, __nv_bfloat16 *dHb, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const float v = H[i] > 0.f ? dH[i] : 0.f;
    dH[i] = v;
    dHb[i] = __float2bfloat16(v);
  }
}

// db[n] += sum_b dY[b][n]
__global__ void k_bias_grad(const float *dY, int Bn, int O, float *db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < O) {
    float s = 0.f;
    for (int b = 0; b < Bn; ++b) s += dY[(size_t)b * O + n];
    db[n] += s;
  }
}

// AdamW on the FP32 master weights, refreshing the BF16 copy of the matrices.
__global__ void k_adamw(float *w, const float *g, float *m, float *v, __nv_bfloat16 *wb,
                        const int *is_matrix, int64_t n, float lr, float b1, float b2, float eps,
                        float wd, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float wi = w[i];
    if (is_matrix[i >> 8]) wi -= lr * wd * wi;  // decoupled decay on matrices only
    wi -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16(wi);
  }
}

__global__ void k_f32_to_bf16(const float *w, __nv_bfloat16 *wb, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) wb[i] = __float2bfloat16(w[i]);
}

__global__ void k_init_uniform(float *w, __nv_bfloat16 *wb, int64_t n, float bound, uint64_t seed,
                               uint64_t stream) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    // SplitMix64 of (seed, stream, i) -> uniform in [-bound, bound)
    uint64_t z = seed + 0x9e3779b97f4a7c15ULL * (uint64_t)(i + 1) + (stream << 40);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z ^= z >> 31;
    const float u = (float)(z >> 40) * (1.f / 16777216.f);
    const float v = bound * (2.f * u - 1.f);
    w[i] = v;
    wb[i] = __float2bfloat16(v);
  }
}

}  // namespace mdhp

using namespace mdhp;

struct mdhp_init_model {
  int M, K0, H, O, max_batch, layers = 4;
  int64_t off_w[4], off_b[4], nparams;
  int din[4], dout[4];
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // FP32 master / grad / moments
  __nv_bfloat16 *wb = nullptr;                                    // BF16 copy
  int *is_matrix = nullptr;                                       // per 256-element block
  __nv_bfloat16 *X = nullptr, *hb[4] = {};
  float *h[4] = {}, *dh[4] = {}, *aux = nullptr, *loss = nullptr;
  __nv_bfloat16 *dhb[4] = {};
  int64_t step = 0;
  int gemm_engine = 0;  // 0: tensor cores (tcgen05) where the layouts allow; 1: mma.sync
};

static mdhp_status init_fail(mdhp_status s, const char *msg) {
  record_error(msg);
  return s;
}

static int grid1(int64_t n, int t = 256) { return (int)((n + t - 1) / t); }

// The warp-level MMA path (mma.sync), any strides.
static void launch_gemm_mma(const __nv_bfloat16 *A, int64_t sam, int64_t sak, const __nv_bfloat16 *B,
                            int64_t sbk, int64_t sbn, int Mm, int Nn, int Kk, const float *bias,
                            int relu, float *Cf, __nv_bfloat16 *Cb, int64_t ldc, int accumulate,
                            cudaStream_t st) {
  const int va = (sak == 1 && sam % 8 == 0 && Kk % 8 == 0 && ((uintptr_t)A & 15) == 0) ? 1 : 0;
  const int vb = (sbk == 1 && sbn % 8 == 0 && Kk % 8 == 0 && ((uintptr_t)B & 15) == 0) ? 1 : 0;
  GemmArgs g{A, B, sam, sak, sbk, sbn, Mm, Nn, Kk, bias, relu, accumulate, va, vb, Cf, Cb, ldc};
  dim3 grid((Nn + 63) / 64, (Mm + 63) / 64);
  if (va && vb) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_gemm_bf16_kk, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
      attr = true;
    }
    k_gemm_bf16_kk<<<grid, 128, kGemmSmem, st>>>(g);
    return;
  }
  k_gemm_bf16<<<grid, 128, 0, st>>>(g);
}

// Whether a product given by strides (A(m,k) = A[m*sam + k*sak], B(k,n) =
// B[k*sbk + n*sbn]) runs on the tensor cores (tcgen05): engine 0, one of the
// two strides of each operand 1, a supported layout, and an FP32 output when
// the K split needs one.  Fills the major flags and pitches.
struct TcRoute {
  bool use;
  int a_mn, b_mn;
  int64_t lda, ldb;
};
static TcRoute tc_route(int engine, const __nv_bfloat16 *A, int64_t sam, int64_t sak,
                        const __nv_bfloat16 *B, int64_t sbk, int64_t sbn, int Mm, int Nn, int Kk,
                        const float *Cf, int accumulate) {
  TcRoute r{false, 0, 0, 0, 0};
  if (engine != 0 || !((sak == 1 || sam == 1) && (sbk == 1 || sbn == 1))) return r;
  r.a_mn = sak == 1 ? 0 : 1;
  r.b_mn = sbk == 1 ? 0 : 1;
  r.lda = r.a_mn ? sak : sam;
  r.ldb = r.b_mn ? sbk : sbn;
  const bool out_ok = Cf != nullptr || gemm_tc_launches(Mm, Nn, Kk, accumulate, 0, r.a_mn, r.b_mn, 0) == 1;
  r.use = out_ok && gemm_tc_supported(A, r.lda, r.a_mn, B, r.ldb, r.b_mn, Mm, Nn, Kk);
  return r;
}

// Kernel launches of one product (for the launch counts the library reports).
static int gemm_launches(int engine, const __nv_bfloat16 *A, int64_t sam, int64_t sak,
                         const __nv_bfloat16 *B, int64_t sbk, int64_t sbn, int Mm, int Nn, int Kk,
                         const float *Cf, int accumulate) {
  const TcRoute r = tc_route(engine, A, sam, sak, B, sbk, sbn, Mm, Nn, Kk, Cf, accumulate);
  return r.use ? gemm_tc_launches(Mm, Nn, Kk, accumulate, 0, r.a_mn, r.b_mn, 0) : 1;
}

// A product on the tensor cores (tcgen05) when tc_route allows it, else on
// the warp-level MMA path.
static mdhp_status launch_gemm(int engine, const __nv_bfloat16 *A, int64_t sam, int64_t sak,
                               const __nv_bfloat16 *B, int64_t sbk, int64_t sbn, int Mm, int Nn, int Kk,
                               const float *bias, int relu, float *Cf, __nv_bfloat16 *Cb, int64_t ldc,
                               int accumulate, cudaStream_t st) {
  const TcRoute r = tc_route(engine, A, sam, sak, B, sbk, sbn, Mm, Nn, Kk, Cf, accumulate);
  if (r.use)
    return gemm_tc(A, r.lda, r.a_mn, B, r.ldb, r.b_mn, Mm, Nn, Kk, bias, relu, Cf, Cb, ldc, accumulate,
                   0, st, 0);
  launch_gemm_mma(A, sam, sak, B, sbk, sbn, Mm, Nn, Kk, bias, relu, Cf, Cb, ldc, accumulate, st);
  return MDHP_OK;
}

extern "C" {

mdhp_status mdhp_init_model_create(mdhp_init_model **out, int32_t M, int32_t hidden,
                                   int32_t max_batch, uint64_t seed) {
  if (!out) return init_fail(MDHP_E_ARG, "mdhp_init_model_create: out NULL");
  *out = nullptr;
  if (M < 1 || M > 32) return init_fail(MDHP_E_ARG, "mdhp_init_model_create: M must be 1..32");
  if (hidden < 64 || hidden > 4096 || hidden % 64)
    return init_fail(MDHP_E_ARG, "mdhp_init_model_create: hidden must be a multiple of 64 in [64, 4096]");
  if (max_batch < 1 || max_batch > 65536)
    return init_fail(MDHP_E_ARG, "mdhp_init_model_create: max_batch must be 1..65536");
  mdhp_init_model *p = new mdhp_init_model();
  p->M = M;
  p->K0 = init_k0(M);
  p->H = hidden;
  p->O = M + M * M;
  p->max_batch = max_batch;
  const int dims[5] = {p->K0, hidden, hidden, hidden, p->O};
  int64_t off = 0;
  for (int l = 0; l < 4; ++l) {
    p->din[l] = dims[l];
    p->dout[l] = dims[l + 1];
    p->off_w[l] = off;
    off += (int64_t)dims[l] * dims[l + 1];
    off = (off + 255) / 256 * 256;
    p->off_b[l] = off;
    off += dims[l + 1];
    off = (off + 255) / 256 * 256;
  }
  p->nparams = off;
  bool ok = true;
  ok &= cudaMalloc(&p->w, off * 4) == cudaSuccess;
  ok &= cudaMalloc(&p->g, off * 4) == cudaSuccess;
  ok &= cudaMalloc(&p->m, off * 4) == cudaSuccess;
  ok &= cudaMalloc(&p->v, off * 4) == cudaSuccess;
  ok &= cudaMalloc(&p->wb, off * 2) == cudaSuccess;
  ok &= cudaMalloc(&p->is_matrix, (off / 256) * 4) == cudaSuccess;
  ok &= cudaMalloc(&p->X, (size_t)max_batch * p->K0 * 2) == cudaSuccess;
  ok &= cudaMalloc(&p->aux, (size_t)max_batch * M * 4) == cudaSuccess;
  ok &= cudaMalloc(&p->loss, 4) == cudaSuccess;
  for (int l = 0; l < 4; ++l) {
    ok &= cudaMalloc(&p->h[l], (size_t)max_batch * p->dout[l] * 4) == cudaSuccess;
    ok &= cudaMalloc(&p->hb[l], (size_t)max_batch * p->dout[l] * 2) == cudaSuccess;
    ok &= cudaMalloc(&p->dh[l], (size_t)max_batch * p->dout[l] * 4) == cudaSuccess;
    ok &= cudaMalloc(&p->dhb[l], (size_t)max_batch * p->dout[l] * 2) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    mdhp_init_model_destroy(p);
    return init_fail(MDHP_E_NOMEM, "mdhp_init_model_create: allocation failed");
  }
  std::vector<int> mat(off / 256, 0);
  for (int l = 0; l < 4; ++l)
    for (int64_t e = p->off_w[l] / 256; e < (p->off_w[l] + (int64_t)p->din[l] * p->dout[l] + 255) / 256; ++e)
      mat[e] = 1;
  cudaMemcpy(p->is_matrix, mat.data(), mat.size() * 4, cudaMemcpyHostToDevice);
  cudaMemset(p->w, 0, off * 4);
  cudaMemset(p->wb, 0, off * 2);
  cudaMemset(p->m, 0, off * 4);
  cudaMemset(p->v, 0, off * 4);
  for (int l = 0; l < 4; ++l) {  // U(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases
    const int64_t n = (int64_t)p->din[l] * p->dout[l];
    k_init_uniform<<<grid1(n), 256>>>(p->w + p->off_w[l], p->wb + p->off_w[l], n,
                                      1.f / sqrtf((float)p->din[l]), seed, (uint64_t)l);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    mdhp_init_model_destroy(p);
    return init_fail(MDHP_E_CUDA, "mdhp_init_model_create: initialisation failed");
  }
  *out = p;
  return MDHP_OK;
}

void mdhp_init_model_destroy(mdhp_init_model *p) {
  if (!p) return;
  cudaFree(p->w); cudaFree(p->g); cudaFree(p->m); cudaFree(p->v); cudaFree(p->wb);
  cudaFree(p->is_matrix); cudaFree(p->X); cudaFree(p->aux); cudaFree(p->loss);
  for (int l = 0; l < 4; ++l) {
    cudaFree(p->h[l]); cudaFree(p->hb[l]); cudaFree(p->dh[l]); cudaFree(p->dhb[l]);
  }
  delete p;
}

mdhp_status mdhp_init_model_info(const mdhp_init_model *p, int32_t *feature_dim, int32_t *out_dim,
                                 int64_t *num_params) {
  if (!p) return init_fail(MDHP_E_ARG, "mdhp_init_model_info: model NULL");
  if (feature_dim) *feature_dim = p->K0;
  if (out_dim) *out_dim = p->O;
  if (num_params) *num_params = p->nparams;
  return MDHP_OK;
}

mdhp_status mdhp_init_model_get(const mdhp_init_model *p, int32_t what, float *dst, void *stream) {
  if (!p || !dst || (what != 0 && what != 1)) return init_fail(MDHP_E_ARG, "mdhp_init_model_get: bad argument");
  if (cudaMemcpyAsync(dst, what == 0 ? p->w : p->g, p->nparams * 4, cudaMemcpyDeviceToDevice,
                      (cudaStream_t)stream) != cudaSuccess)
    return init_fail(MDHP_E_CUDA, cudaGetErrorString(cudaGetLastError()));
  return MDHP_OK;
}

mdhp_status mdhp_init_model_set_params(mdhp_init_model *p, const float *src, void *stream) {
  if (!p || !src) return init_fail(MDHP_E_ARG, "mdhp_init_model_set_params: NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(p->w, src, p->nparams * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return init_fail(MDHP_E_CUDA, cudaGetErrorString(cudaGetLastError()));
  k_f32_to_bf16<<<grid1(p->nparams), 256, 0, st>>>(p->w, p->wb, p->nparams);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return init_fail(MDHP_E_CUDA, cudaGetErrorString(e));
  return MDHP_OK;
}

mdhp_status mdhp_init_features(const mdhp_batch *batch, const float *beta, void *features_bf16,
                               float *mu_cold, void *stream) {
  if (!batch || !beta || !features_bf16 || !mu_cold)
    return init_fail(MDHP_E_ARG, "mdhp_init_features: NULL argument");
  if (batch->M < 1 || batch->M > 32) return init_fail(MDHP_E_ARG, "mdhp_init_features: M must be 1..32");
  if (batch->B <= 0) return MDHP_OK;
  const int M = batch->M, Mt = M <= 4 ? 4 : M <= 8 ? 8 : M <= 16 ? 16 : 32;
  const int K0 = init_k0(M);
  const int nt = kFeatThreads;
  const bool pack = batch->max_events > 0 && batch->max_events < 65536;
  const int words = pack ? Mt * Mt * kBins / 2 : Mt * Mt * kBins;
  const int smem = (words + nt * Mt + Mt + Mt * Mt) * 4;
  const int bstride = batch->beta_mode == MDHP_BETA_SCALAR ? 1 : M;
  cudaStream_t st = (cudaStream_t)stream;
#define MDHP_FEAT_P(MV, PK)                                                                       \
  {                                                                                               \
    if (smem > 48 * 1024)                                                                         \
      cudaFuncSetAttribute(k_features<MV, PK>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
    k_features<MV, PK><<<batch->B, nt, smem, st>>>(batch->offsets, batch->t, batch->id,           \
                                                   batch->T_span, beta, bstride, M, K0,           \
                                                   (__nv_bfloat16 *)features_bf16, mu_cold);      \
  }
#define MDHP_FEAT(MV)                  \
  case MV:                             \
    if (pack) MDHP_FEAT_P(MV, true)    \
    else MDHP_FEAT_P(MV, false)        \
    break;
  switch (Mt) {
    MDHP_FEAT(4)
    MDHP_FEAT(8)
    MDHP_FEAT(16)
    MDHP_FEAT(32)
  }
#undef MDHP_FEAT_P
#undef MDHP_FEAT
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return init_fail(MDHP_E_CUDA, cudaGetErrorString(e));
  return MDHP_OK;
}

// Forward over rows [0, Bn) of X (BF16 [Bn][K0]); leaves Y in h[3] (FP32).
static mdhp_status init_forward(mdhp_init_model *p, const __nv_bfloat16 *X, int Bn, cudaStream_t st) {
  const __nv_bfloat16 *in = X;
  for (int l = 0; l < 4; ++l) {
    const int din = p->din[l], dout = p->dout[l];
    const mdhp_status s = launch_gemm(p->gemm_engine, in, din, 1, p->wb + p->off_w[l], 1, din, Bn, dout,
                                      din, p->w + p->off_b[l], l < 3 ? 1 : 0, p->h[l], p->hb[l], dout, 0,
                                      st);
    if (s != MDHP_OK) return s;
    in = p->hb[l];
  }
  return MDHP_OK;
}

// kernel launches of init_forward over Bn rows
static int init_forward_launches(const mdhp_init_model *p, const __nv_bfloat16 *X, int Bn) {
  int n = 0;
  const __nv_bfloat16 *in = X;
  for (int l = 0; l < 4; ++l) {
    const int din = p->din[l], dout = p->dout[l];
    n += gemm_launches(p->gemm_engine, in, din, 1, p->wb + p->off_w[l], 1, din, Bn, dout, din, p->h[l], 0);
    in = p->hb[l];
  }
  return n;
}

mdhp_status mdhp_init_forward(mdhp_init_model *p, const void *features_bf16, int32_t B, float *out,
                              void *stream) {
  if (!p || !features_bf16 || !out) return init_fail(MDHP_E_ARG, "mdhp_init_forward: NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  for (int b0 = 0; b0 < B; b0 += p->max_batch) {
    const int n = B - b0 < p->max_batch ? B - b0 : p->max_batch;
    const mdhp_status s = init_forward(p, (const __nv_bfloat16 *)features_bf16 + (size_t)b0 * p->K0, n, st);
    if (s != MDHP_OK) return s;
    cudaMemcpyAsync(out + (size_t)b0 * p->O, p->h[3], (size_t)n * p->O * 4, cudaMemcpyDeviceToDevice, st);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return init_fail(MDHP_E_CUDA, cudaGetErrorString(e));
  return MDHP_OK;
}

}  // extern "C"

namespace mdhp {
// per chunk of max_batch windows: the features, the four layers' products
// (one or two launches each) and the head
int init_predict_launches(const mdhp_init_model *p, int B) {
  if (!p || B <= 0) return 0;
  int n = 0;
  for (int b0 = 0; b0 < B; b0 += p->max_batch) {
    const int rows = B - b0 < p->max_batch ? B - b0 : p->max_batch;
    n += 2 + init_forward_launches(p, p->X, rows);
  }
  return n;
}
}  // namespace mdhp

extern "C" {

mdhp_status mdhp_init_predict(mdhp_init_model *p, const mdhp_batch *batch, const float *beta,
                              float *mu, float *alpha, void *stream) {
  if (!p || !batch || !beta || !mu || !alpha) return init_fail(MDHP_E_ARG, "mdhp_init_predict: NULL argument");
  if (batch->M != p->M) return init_fail(MDHP_E_ARG, "mdhp_init_predict: batch M differs from the model's");
  cudaStream_t st = (cudaStream_t)stream;
  const int bstride = batch->beta_mode == MDHP_BETA_SCALAR ? 1 : batch->M;
  for (int b0 = 0; b0 < batch->B; b0 += p->max_batch) {
    const int n = batch->B - b0 < p->max_batch ? batch->B - b0 : p->max_batch;
    mdhp_batch sub = *batch;
    sub.B = n;
    sub.offsets = batch->offsets + b0;
    sub.T_span = batch->T_span + b0;
    const float *bsub = beta + (int64_t)b0 * bstride;
    mdhp_status s = mdhp_init_features(&sub, bsub, p->X, p->aux, stream);
    if (s != MDHP_OK) return s;
    if ((s = init_forward(p, p->X, n, st)) != MDHP_OK) return s;
    k_init_head<<<n, 128, 0, st>>>(p->h[3], p->O, p->aux, bsub, bstride, p->M, n,
                                   mu + (int64_t)b0 * p->M, alpha + (int64_t)b0 * p->M * p->M);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return init_fail(MDHP_E_CUDA, cudaGetErrorString(e));
  return MDHP_OK;
}

mdhp_status mdhp_init_backward(mdhp_init_model *p, const void *features_bf16,
                               const float *mu_cold, const float *beta, int32_t beta_stride,
                               const float *mu_target, const float *alpha_target, int32_t B,
                               float *loss_out, void *stream) {
  if (!p || !features_bf16 || !mu_cold || !beta || !mu_target || !alpha_target)
    return init_fail(MDHP_E_ARG, "mdhp_init_backward: NULL argument");
  if (B < 1 || B > p->max_batch) return init_fail(MDHP_E_ARG, "mdhp_init_backward: B outside 1..max_batch");
  if (beta_stride != 1 && beta_stride != p->M) return init_fail(MDHP_E_ARG, "mdhp_init_backward: beta_stride");
  cudaStream_t st = (cudaStream_t)stream;
  const __nv_bfloat16 *X = (const __nv_bfloat16 *)features_bf16;
  mdhp_status s = init_forward(p, X, B, st);
  if (s != MDHP_OK) return s;
  cudaMemsetAsync(p->loss, 0, 4, st);
  cudaMemsetAsync(p->g, 0, p->nparams * 4, st);
  k_init_loss<<<B, 128, 0, st>>>(p->h[3], p->O, mu_cold, beta, beta_stride, p->M, B, mu_target,
                                 alpha_target, p->dh[3], p->dhb[3], p->loss);
  for (int l = 3; l >= 0; --l) {
    const int din = p->din[l], dout = p->dout[l];
    const __nv_bfloat16 *in = l > 0 ? p->hb[l - 1] : X;
    // dW[dout][din] = dY^T [dout][B] x In [B][din]
    if ((s = launch_gemm(p->gemm_engine, p->dhb[l], 1, dout, in, din, 1, dout, din, B, nullptr, 0,
                         p->g + p->off_w[l], nullptr, din, 1, st)) != MDHP_OK)
      return s;
    k_bias_grad<<<grid1(dout), 256, 0, st>>>(p->dh[l], B, dout, p->g + p->off_b[l]);
    if (l > 0) {
      // dIn[B][din] = dY [B][dout] x W [dout][din]; then the ReLU of layer l-1
      if ((s = launch_gemm(p->gemm_engine, p->dhb[l], dout, 1, p->wb + p->off_w[l], din, 1, B, din, dout,
                           nullptr, 0, p->dh[l - 1], nullptr, din, 0, st)) != MDHP_OK)
        return s;
      const int64_t n = (int64_t)B * din;
      k_relu_bwd<<<grid1(n), 256, 0, st>>>(p->dh[l - 1], p->h[l - 1], p->dhb[l - 1], n);
    }
  }
  if (loss_out) cudaMemcpyAsync(loss_out, p->loss, 4, cudaMemcpyDeviceToDevice, st);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return init_fail(MDHP_E_CUDA, cudaGetErrorString(e));
  return MDHP_OK;
}

mdhp_status mdhp_init_set_grads(mdhp_init_model *p, const float *src, void *stream) {
  if (!p || !src) return init_fail(MDHP_E_ARG, "mdhp_init_set_grads: NULL argument");
  if (cudaMemcpyAsync(p->g, src, (size_t)p->nparams * 4, cudaMemcpyDeviceToDevice,
                      (cudaStream_t)stream) != cudaSuccess)
    return init_fail(MDHP_E_CUDA, cudaGetErrorString(cudaGetLastError()));
  return MDHP_OK;
}

mdhp_status mdhp_init_apply(mdhp_init_model *p, float lr, float weight_decay, void *stream) {
  if (!p) return init_fail(MDHP_E_ARG, "mdhp_init_apply: NULL model");
  cudaStream_t st = (cudaStream_t)stream;
  p->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)p->step), c2 = 1.f - powf(b2, (float)p->step);
  k_adamw<<<grid1(p->nparams), 256, 0, st>>>(p->w, p->g, p->m, p->v, p->wb, p->is_matrix,
                                              p->nparams, lr, b1, b2, 1e-8f, weight_decay, c1, c2);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return init_fail(MDHP_E_CUDA, cudaGetErrorString(e));
  return MDHP_OK;
}

mdhp_status mdhp_init_train_step(mdhp_init_model *p, const void *features_bf16,
                                 const float *mu_cold, const float *beta, int32_t beta_stride,
                                 const float *mu_target, const float *alpha_target, int32_t B,
                                 float lr, float weight_decay, float *loss_out, void *stream) {
  const mdhp_status s = mdhp_init_backward(p, features_bf16, mu_cold, beta, beta_stride, mu_target,
                                           alpha_target, B, loss_out, stream);
  if (s != MDHP_OK) return s;
  return mdhp_init_apply(p, lr, weight_decay, stream);
}

mdhp_status mdhp_init_model_set_gemm(mdhp_init_model *p, int32_t engine) {
  if (!p || engine < 0 || engine > 1) return init_fail(MDHP_E_ARG, "mdhp_init_model_set_gemm: bad argument");
  p->gemm_engine = engine;
  return MDHP_OK;
}

mdhp_status mdhp_gemm_bf16(const void *A, int64_t lda, int32_t a_mn, const void *B, int64_t ldb,
                           int32_t b_mn, int32_t M, int32_t N, int32_t K, const float *bias,
                           int32_t relu, float *C, void *C_bf16, int64_t ldc, int32_t accumulate,
                           int32_t engine, void *stream) {
  if (!A || !B || M < 1 || N < 1 || K < 1 || engine < 0 || engine > 2 || (!C && (accumulate || !C_bf16)))
    return init_fail(MDHP_E_ARG, "mdhp_gemm_bf16: bad argument");
  const __nv_bfloat16 *a = (const __nv_bfloat16 *)A, *b = (const __nv_bfloat16 *)B;
  __nv_bfloat16 *cb = accumulate ? nullptr : (__nv_bfloat16 *)C_bf16;
  cudaStream_t st = (cudaStream_t)stream;
  if (engine == 0 || engine == 2) {
    if (!gemm_tc_supported(A, lda, a_mn, B, ldb, b_mn, M, N, K))
      return init_fail(MDHP_E_UNSUPPORTED, "mdhp_gemm_bf16: layout not supported by the tensor-core GEMM");
    if (!C && gemm_tc_launches(M, N, K, accumulate, 0, a_mn, b_mn, engine == 2 ? 1 : 0) > 1)
      return init_fail(MDHP_E_ARG, "mdhp_gemm_bf16: this shape splits K and needs the FP32 output");
    return gemm_tc(a, lda, a_mn, b, ldb, b_mn, M, N, K, bias, relu, C, cb, ldc, accumulate, 0, st,
                   engine == 2 ? 1 : 0);
  }
  const int64_t sam = a_mn ? 1 : lda, sak = a_mn ? lda : 1;
  const int64_t sbk = b_mn ? ldb : 1, sbn = b_mn ? 1 : ldb;
  launch_gemm_mma(a, sam, sak, b, sbk, sbn, M, N, K, accumulate ? nullptr : bias, accumulate ? 0 : relu, C,
                  cb, ldc, accumulate, st);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return init_fail(MDHP_E_CUDA, cudaGetErrorString(e));
  return MDHP_OK;
}

}  // extern "C"
