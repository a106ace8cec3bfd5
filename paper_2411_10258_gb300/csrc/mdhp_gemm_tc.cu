// BF16 GEMM on the fifth-generation tensor cores (tcgen05.mma, FP32
// accumulators in tensor memory) for the learned initializer's layers:
//   C[m][n] (+)= sum_k A(m,k) B(k,n)   (+ bias[n], ReLU; FP32 and/or BF16 out)
// A is [M][K] with K contiguous (a_mn = 0) or [K][M] with M contiguous
// (a_mn = 1); B is [N][K] with K contiguous (b_mn = 0) or [K][N] with N
// contiguous (b_mn = 1).  Both majors are native operand layouts of the MMA,
// so the transposes of the backward pass need no copies.
//
// One CTA computes a 128 x BN tile (BN <= 256, a multiple of 16) over a range
// of K (split-K across blockIdx.z).  128 threads:
//   * all threads stage K-blocks of 64 with cp.async (16-byte chunks) into a
//     4-deep ring of shared-memory stages, in the no-swizzle canonical layout
//     of the MMA: 8 x 16-byte "core matrices", core matrix (g, kg) of an
//     operand (g = row group of 8 along M or N, kg = group of 8 along K) at
//     byte (g * 8 + kg) * 128, its 8 rows 16 bytes apart (rows run along M/N
//     for a K-major operand and along K for an M/N-major one);
//   * thread 0 issues the stage's four 128 x BN x 16 MMAs and commits them to
//     the stage's mbarrier; a stage is refilled after that barrier completes;
//   * the accumulator tile (128 lanes x BN columns of FP32) lives in tensor
//     memory, allocated per CTA; the epilogue reads it back with tcgen05.ld
//     (warp w owns lanes 32w..32w+31 = tile rows) and applies bias and ReLU,
//     or adds into C with atomics when K is split.
// No cluster, no multicast: every CTA reads its own tiles.  Every wait is
// bounded; a wait that gives up counts a timeout (mdhp_gemm_check), waits
// (bounded) for the MMAs in flight, frees the tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "mdhp.h"
#include "mdhp_async.cuh"

namespace mdhp {

void record_error(const char *msg);  // mdhp_api.cu

namespace tc {

constexpr int kBM = 128, kBK = 64, kStages = 4, kThreads = 128, kMaxBN = 256;
constexpr int kAStage = kBM * kBK * 2;     // 16 KB
constexpr int kBStage = kMaxBN * kBK * 2;  // 32 KB
constexpr int kTmemCols = 256;
// stages, then mbarriers and the tensor-memory address; 1 KB of slack to
// align the stages to 1 KB
constexpr int kSmem = kStages * (kAStage + kBStage) + 128 + 1024;

struct Args {
  const __nv_bfloat16 *A, *B;
  int64_t lda, ldb;      // row pitch of the stored arrays (elements)
  int a_mn, b_mn;        // 1: M (resp. N) is the contiguous dimension
  int Mm, Nn, Kk;
  int BN;                // tile width (multiple of 16, <= 256)
  int kb_per_split;      // K-blocks of 64 per blockIdx.z
  const float *bias;
  int relu;
  int atomic;            // add the tile into Cf with atomics (split K)
  int accumulate;        // add the tile into Cf (one CTA per element)
  float *Cf;
  __nv_bfloat16 *Cb;
  int64_t ldc;
};

__device__ int g_timeouts;

// Shared-memory matrix descriptor (tcgen05), no swizzle: start address,
// leading byte offset (between core matrices along K), stride byte offset
// (between core matrices along M/N), all in 16-byte units; bits 46-47 hold
// the descriptor version 1; base offset, LBO mode and swizzle mode 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9 = 1, 10-12 = 1), majors (bit 15: A, bit 16: B; 0 = K),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ __forceinline__ uint32_t instr_desc(int M, int N, int a_mn, int b_mn) {
  uint32_t d = 0;
  d |= 1u << 4;
  d |= 1u << 7;
  d |= 1u << 10;
  d |= (uint32_t)(a_mn & 1) << 15;
  d |= (uint32_t)(b_mn & 1) << 16;
  d |= (uint32_t)((N >> 3) & 0x3F) << 17;
  d |= (uint32_t)((M >> 4) & 0x1F) << 24;
  return d;
}

__device__ __forceinline__ void cp16(uint32_t dst, const void *src, bool valid) {
  const int n = valid ? 16 : 0;  // 0 source bytes: the chunk is zero-filled
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(n)
               : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_saddr, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_saddr),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// the mbarrier arrives once all earlier tcgen05 operations of this thread completed
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}

// 16 consecutive FP32 columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of 16-byte chunk e of a stage (rows = 8-wide groups along M/N
// for K-major data, along K for M/N-major data) and the element it starts at.
// K-major: a warp's 32 chunks are 8 rows x 4 consecutive K chunks, so the
// global reads are 64 contiguous bytes per row and the shared writes fill
// four whole core matrices.  M/N-major: 8 K rows x 4 consecutive 8-wide
// groups along M/N.
struct Chunk {
  int off;  // byte offset in the stage
  int mn;   // first M/N index (relative to the tile)
  int k;    // first K index (relative to the K-block)
};
__host__ __device__ __forceinline__ Chunk chunk_kmajor(int e) {
  const int r = e & 7, kc_lo = (e >> 3) & 3, q = e >> 5;
  const int g = q >> 1, kc = ((q & 1) << 2) | kc_lo;
  return {(g * 8 + kc) * 128 + r * 16, g * 8 + r, kc * 8};
}
__host__ __device__ __forceinline__ Chunk chunk_mnmajor(int e, int rows) {
  const int r = e & 7, a = e >> 3;
  const int g = a % (rows / 8), kg = a / (rows / 8);
  return {(g * 8 + kg) * 128 + r * 16, g * 8, kg * 8 + r};
}

// one operand's K-block (rows x 64) into a stage
__device__ __forceinline__ void load_operand(uint32_t sbase, const __nv_bfloat16 *X, int64_t ld, int mn_major,
                                             int rows, int r0, int rlim, int k0, int klim) {
  const int nchunks = rows * 8;
  for (int e = threadIdx.x; e < nchunks; e += kThreads) {
    if (!mn_major) {
      const Chunk c = chunk_kmajor(e);
      const int r = r0 + c.mn, k = k0 + c.k;
      const bool v = r < rlim && k < klim;
      cp16(sbase + c.off, v ? X + (int64_t)r * ld + k : X, v);
    } else {
      const Chunk c = chunk_mnmajor(e, rows);
      const int r = r0 + c.mn, k = k0 + c.k;
      const bool v = r < rlim && k < klim;
      cp16(sbase + c.off, v ? X + (int64_t)k * ld + r : X, v);
    }
  }
}

__global__ void __launch_bounds__(kThreads, 1) k_gemm_tc(Args g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // 1 KB-aligned stages
  const uint32_t raw = smem_addr(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  unsigned char *base = smem_raw + pad;
  const uint32_t sA = raw + pad;
  const uint32_t sB = sA + kStages * kAStage;
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + kStages * (kAStage + kBStage));
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + kStages);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * g.BN;
  const int nkb = (g.Kk + kBK - 1) / kBK;
  const int kb0 = blockIdx.z * g.kb_per_split;
  const int kb1 = min(nkb, kb0 + g.kb_per_split);
  const int n = kb1 - kb0;  // K-blocks of this CTA (>= 1 by construction)

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(bars + s, 1);
    mbar_init_fence();
  }
  if (warp == 0) {
    tmem_alloc(smem_addr(tslot), kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  const uint32_t idesc = instr_desc(kBM, g.BN, g.a_mn, g.b_mn);
  bool ok = true;
  int last = -1;  // last K-block whose MMAs were committed (uniform)
  auto load = [&](int i) {  // K-block kb0 + i into stage i % kStages
    const int st = i % kStages, k0 = (kb0 + i) * kBK;
    load_operand(sA + st * kAStage, g.A, g.lda, g.a_mn, kBM, m0, g.Mm, k0, g.Kk);
    load_operand(sB + st * kBStage, g.B, g.ldb, g.b_mn, g.BN, n0, g.Nn, k0, g.Kk);
  };
#pragma unroll
  for (int i = 0; i < kStages - 1; ++i) {
    if (i < n) load(i);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  for (int i = 0; i < n; ++i) {
    const int st = i % kStages;
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kStages - 2) : "memory");
    fence_proxy_async_shared();  // this thread's staged chunks -> the MMA's reads
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int s = 0; s < kBK / 16; ++s) {
        const uint64_t ad = smem_desc(sA + st * kAStage + s * 256, 128, 1024);
        const uint64_t bd = smem_desc(sB + st * kBStage + s * 256, 128, 1024);
        mma_bf16(tmem, ad, bd, idesc, (i > 0 || s > 0) ? 1u : 0u);
      }
      mma_commit(bars + st);
    }
    last = i;
    // the next load goes into the stage of K-block i - 1: its MMAs must be done
    const int nx = i + kStages - 1;
    if (nx < n) {
      if (i >= 1) {
        const int sp = (i - 1) % kStages;
        if (!mbar_wait(bars + sp, (uint32_t)(((i - 1) / kStages) & 1))) ok = false;
        if (__syncthreads_or(!ok)) break;
      }
      load(nx);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  // the last commit covers every MMA of this CTA (also after a wait gave up)
  {
    const bool done = mbar_wait(bars + (last % kStages), (uint32_t)((last / kStages) & 1));
    if (__syncthreads_or(!ok || !done)) {
      if (tid == 0) atomicAdd(&g_timeouts, 1);
      ok = false;
    }
  }
  tc_fence_after();
  if (ok) {
    const int m = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < g.BN; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (m < g.Mm) {
        const int64_t row = (int64_t)m * g.ldc;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int nn = n0 + c0 + j;
          if (nn >= g.Nn) break;
          float x = v[j];
          if (g.atomic) {
            atomicAdd(g.Cf + row + nn, x);
            continue;
          }
          if (g.accumulate) {
            g.Cf[row + nn] += x;
            continue;
          }
          if (g.bias) x += g.bias[nn];
          if (g.relu) x = fmaxf(x, 0.f);
          if (g.Cf) g.Cf[row + nn] = x;
          if (g.Cb) g.Cb[row + nn] = __float2bfloat16(x);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// split K: bias, ReLU and the BF16 copy once the partial tiles are summed
__global__ void k_gemm_finish(float *Cf, __nv_bfloat16 *Cb, int64_t ldc, int Mm, int Nn, const float *bias,
                              int relu) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)Mm * Nn) return;
  const int m = (int)(i / Nn), nn = (int)(i % Nn);
  const int64_t o = (int64_t)m * ldc + nn;
  float x = Cf[o];
  if (bias) x += bias[nn];
  if (relu) x = fmaxf(x, 0.f);
  Cf[o] = x;
  if (Cb) Cb[o] = __float2bfloat16(x);
}

}  // namespace tc

static int tc_num_sms() {
  static int v = -1;
  if (v < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  }
  return v;
}

// Launch plan of one product; split = 0 picks the K split from the tile count.
struct TcPlan {
  int BN, tiles_n, tiles_m, nkb, kb_per_split, splits;
};
static TcPlan tc_plan(int Mm, int Nn, int Kk, int split) {
  TcPlan p{};
  p.tiles_n = (Nn + tc::kMaxBN - 1) / tc::kMaxBN;
  p.BN = ((Nn + p.tiles_n - 1) / p.tiles_n + 15) / 16 * 16;
  p.tiles_m = (Mm + tc::kBM - 1) / tc::kBM;
  p.nkb = (Kk + tc::kBK - 1) / tc::kBK;
  int s = split;
  if (s <= 0) {  // fill the SMs, at least 4 K-blocks per CTA
    const int tiles = p.tiles_m * p.tiles_n;
    s = tc_num_sms() / (tiles > 0 ? tiles : 1);
    const int cap = p.nkb / 4;
    if (s > cap) s = cap;
  }
  if (s < 1) s = 1;
  if (s > p.nkb) s = p.nkb;
  p.kb_per_split = (p.nkb + s - 1) / s;
  p.splits = (p.nkb + p.kb_per_split - 1) / p.kb_per_split;  // every split has >= 1 K-block
  return p;
}

// Operand layouts the kernel takes: 16-byte aligned bases and pitches, K a
// multiple of 8, and for an M/N-major operand M (N) a multiple of 8.
bool gemm_tc_supported(const void *A, int64_t lda, int a_mn, const void *B, int64_t ldb, int b_mn, int Mm,
                       int Nn, int Kk) {
  if (Mm < 1 || Nn < 1 || Kk < 8 || Kk % 8) return false;
  if (((uintptr_t)A & 15) || ((uintptr_t)B & 15) || lda % 8 || ldb % 8) return false;
  if (a_mn && Mm % 8) return false;
  if (b_mn && Nn % 8) return false;
  return true;
}

// C (+)= A B on the tensor cores.  accumulate = 1: Cf += A B (no bias, ReLU
// or BF16 output).  Otherwise Cf and/or Cb receive A B + bias, ReLU'd; with a
// K split Cf is required (it holds the partial sums).  split = 0: automatic.
mdhp_status gemm_tc(const __nv_bfloat16 *A, int64_t lda, int a_mn, const __nv_bfloat16 *B, int64_t ldb,
                    int b_mn, int Mm, int Nn, int Kk, const float *bias, int relu, float *Cf,
                    __nv_bfloat16 *Cb, int64_t ldc, int accumulate, int split, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(tc::k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmem) !=
        cudaSuccess) {
      cudaGetLastError();
      record_error("gemm_tc: shared memory attribute");
      return MDHP_E_CUDA;
    }
    attr = true;
  }
  const TcPlan p = tc_plan(Mm, Nn, Kk, split);
  tc::Args g{};
  g.A = A; g.B = B; g.lda = lda; g.ldb = ldb; g.a_mn = a_mn; g.b_mn = b_mn;
  g.Mm = Mm; g.Nn = Nn; g.Kk = Kk; g.BN = p.BN; g.kb_per_split = p.kb_per_split;
  g.ldc = ldc;
  const bool finish = p.splits > 1 && !accumulate;
  if (accumulate || p.splits > 1) {
    if (!Cf) {
      record_error("gemm_tc: a K split or accumulation needs the FP32 output");
      return MDHP_E_ARG;
    }
    g.atomic = p.splits > 1 ? 1 : 0;
    g.accumulate = p.splits > 1 ? 0 : 1;
    g.Cf = Cf;
    if (finish && cudaMemset2DAsync(Cf, (size_t)ldc * 4, 0, (size_t)Nn * 4, (size_t)Mm, st) != cudaSuccess) {
      cudaGetLastError();
      record_error("gemm_tc: clearing the output failed");
      return MDHP_E_CUDA;
    }
  } else {
    g.bias = bias; g.relu = relu; g.Cf = Cf; g.Cb = Cb;
  }
  dim3 grid(p.tiles_n, p.tiles_m, p.splits);
  tc::k_gemm_tc<<<grid, tc::kThreads, tc::kSmem, st>>>(g);
  if (finish) {
    const int64_t tot = (int64_t)Mm * Nn;
    tc::k_gemm_finish<<<(int)((tot + 255) / 256), 256, 0, st>>>(Cf, Cb, ldc, Mm, Nn, bias, relu);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    char buf[160];
    snprintf(buf, sizeof(buf), "gemm_tc: %s", cudaGetErrorString(e));
    record_error(buf);
    return MDHP_E_CUDA;
  }
  return MDHP_OK;
}

int gemm_tc_launches(int Mm, int Nn, int Kk, int accumulate, int split) {
  const TcPlan p = tc_plan(Mm, Nn, Kk, split);
  return 1 + ((p.splits > 1 && !accumulate) ? 1 : 0);
}

}  // namespace mdhp

extern "C" mdhp_status mdhp_gemm_check(int32_t *timeouts) {
  if (!timeouts) {
    mdhp::record_error("mdhp_gemm_check: NULL argument");
    return MDHP_E_ARG;
  }
  int v = 0;
  const int zero = 0;
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpyFromSymbol(&v, mdhp::tc::g_timeouts, sizeof(int)) != cudaSuccess ||
      cudaMemcpyToSymbol(mdhp::tc::g_timeouts, &zero, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    mdhp::record_error("mdhp_gemm_check: device query failed");
    return MDHP_E_CUDA;
  }
  *timeouts = v;
  return MDHP_OK;
}
