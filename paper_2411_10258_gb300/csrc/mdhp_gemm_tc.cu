// BF16 GEMM on the fifth-generation tensor cores (tcgen05.mma, FP32
// accumulators in tensor memory) for the learned initializer's layers:
//   C[m][n] (+)= sum_k A(m,k) B(k,n)   (+ bias[n], ReLU; FP32 and/or BF16 out)
// A is [M][K] with K contiguous (a_mn = 0) or [K][M] with M contiguous
// (a_mn = 1); B is [N][K] with K contiguous (b_mn = 0) or [K][N] with N
// contiguous (b_mn = 1).  Both majors are native operand layouts of the MMA,
// so the transposes of the backward pass need no copies.
//
// Two kernels compute 128 x BN output tiles (BN <= 256, a multiple of 16),
// each over a range of K (split-K across blockIdx.z):
//
// k_gemm_tma (both operands K-contiguous: every forward layer).  Warp-
// specialised: one thread issues TMA box loads (128-byte swizzle) into a ring
// of stages on full/empty mbarrier pairs, one thread issues the MMAs, four
// warps run the epilogue; no block-wide barrier in the main loop.  The K
// splits of a tile form a thread-block cluster whose CTAs sum their partial
// tiles through distributed shared memory (no atomics, no second launch);
// with small clusters two row tiles also share each weight box by multicast.
//
// k_gemm_tc (any operand majors, e.g. the backward products): 128 threads
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
//     (warp w owns lanes 32w..32w+31 = tile rows) into shared memory, then
//     writes it row by row (coalesced), with bias and ReLU, or adds it into
//     C with atomics when K is split (then a finishing launch applies bias,
//     ReLU and the BF16 copy).
// Every mbarrier wait is bounded; a wait that gives up counts a timeout
// (mdhp_gemm_check), waits (bounded) for the copies and MMAs in flight, frees
// the tensor memory and leaves the tile unwritten.
#include <cuda.h>  // CUtensorMap and its encoding enums (the encoder is fetched at run time)
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
// align the stages to 1 KB.  The epilogue reuses the stages for the output
// tile (128 rows of up to 256 + 4 floats).
constexpr int kSmem = kStages * (kAStage + kBStage) + 256 + 1024;
static_assert(kBM * (kMaxBN + 4) * 4 <= kStages * (kAStage + kBStage), "output tile fits the stages");

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
    // accumulator tile -> shared memory (the stages are free: every MMA and
    // copy has completed), rows padded by 4 floats so that a warp's 16-byte
    // stores of 32 different rows spread over the banks
    float *tile = reinterpret_cast<float *>(base);
    const int pitch = g.BN + 4;
    const int r = warp * 32 + lane;
    for (int c0 = 0; c0 < g.BN; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      float4 *dst = reinterpret_cast<float4 *>(tile + r * pitch + c0);
#pragma unroll
      for (int q = 0; q < 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
    __syncthreads();
    // out row by row, a warp's lanes on consecutive columns (coalesced)
    const int rows = min(kBM, g.Mm - m0), cols = min(g.BN, g.Nn - n0);
    for (int rr = warp; rr < rows; rr += kThreads / 32) {
      const float *src = tile + rr * pitch;
      const int64_t o = (int64_t)(m0 + rr) * g.ldc + n0;
      for (int cc = lane; cc < cols; cc += 32) {
        float x = src[cc];
        if (g.atomic) {
          atomicAdd(g.Cf + o + cc, x);
          continue;
        }
        if (g.accumulate) {
          g.Cf[o + cc] += x;
          continue;
        }
        if (g.bias) x += g.bias[n0 + cc];
        if (g.relu) x = fmaxf(x, 0.f);
        if (g.Cf) g.Cf[o + cc] = x;
        if (g.Cb) g.Cb[o + cc] = __float2bfloat16(x);
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


// ---------------------------------------------------------------------------
// K-major x K-major products (every forward layer): the same tile and
// accumulator, with the operands brought in by the tensor-memory accelerator.
// Each stage holds one 128 x 64 box of A and one BN x 64 box of B, written by
// TMA in the 128-byte-swizzled layout (rows of 128 bytes, the 16-byte chunks
// of row r XOR-permuted by r mod 8, 8-row groups 1 KB apart), which is also a
// canonical operand layout of the MMA.  Warp roles (192 threads):
//   warp 0, one thread: producer; waits for a stage's "empty" barrier, then
//     issues its two box loads, completing on the stage's "full" barrier;
//   warp 1, one thread: waits for "full", issues the stage's four MMAs and
//     commits them to "empty"; after the last stage commits to "accum";
//     warp 1 also allocates and frees the tensor memory;
//   warps 2-5: the epilogue (warp w reads TMEM lanes 32 (w mod 4) ..).
// No block-wide barrier in the main loop.
// ---------------------------------------------------------------------------
constexpr int kTmaThreads = 192;
constexpr int kTmaMaxStages = 8;

struct TmaArgs {
  int Mm, Nn, Kk, BN, kb_per_split;
  int splits;       // CTAs per tile along K (1..8); the cluster sums the partial tiles
  int cm;           // 1 or 2 row tiles per cluster sharing each B box (multicast halves)
  int stages;       // ring depth: as many stages of (A box + B box) as fit the stage area
  int stage_bytes;  // 16 KB of A + BN x 128 bytes of B (a multiple of 1 KB)
  uint32_t tmem_cols;  // power of two >= BN (at least 32)
  const float *bias;
  int relu, accumulate;
  float *Cf;
  __nv_bfloat16 *Cb;
  int64_t ldc;
};

// descriptor of a K-major operand in the 128-byte-swizzled layout: 8-row
// groups 1024 bytes apart (SBO); the leading offset is not used by this
// layout (set to 16 bytes); swizzle mode 2 (128 bytes) in bits 61-63
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// one box into the same shared-memory offset of every CTA in `mask` (cluster
// ranks), completing on the mbarrier at the same offset in each
__device__ __forceinline__ void tma_load_2d_mc(uint32_t dst, const CUtensorMap *map, int x, int y,
                                               uint64_t *bar, uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.multicast::cluster"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar)), "h"(mask)
      : "memory");
}
// arrive on the mbarrier at the same offset in every CTA of `mask` once this
// thread's earlier tcgen05 operations completed
__device__ __forceinline__ void mma_commit_mc(uint64_t *bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_addr(bar)),
      "h"(mask)
      : "memory");
}

// thread-block cluster: barrier over every thread of every CTA, this CTA's
// rank, and loads from a peer CTA's shared memory (DSMEM)
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t map_peer(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ float ld_peer(uint32_t addr) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ float4 ld_peer_v4(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr)
               : "memory");
  return v;
}
__device__ __forceinline__ int ld_peer_int(uint32_t addr) {
  int v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

__global__ void __launch_bounds__(kTmaThreads, 1)
    k_gemm_tma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TmaArgs g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t raw = smem_addr(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  unsigned char *base = smem_raw + pad;
  const uint32_t sA = raw + pad;  // stage s: A box at sA + s * stage_bytes, B box 16 KB further
  const int S = g.stages;
  const uint32_t SB = (uint32_t)g.stage_bytes;
  uint64_t *full = reinterpret_cast<uint64_t *>(base + kStages * (kAStage + kBStage));
  uint64_t *empty = full + kTmaMaxStages;
  uint64_t *accum = empty + kTmaMaxStages;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(accum + 1);
  int *flags = reinterpret_cast<int *>(tslot + 1);  // [0] error, [1] fills issued, [2] fills consumed
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * g.BN;
  const int nkb = (g.Kk + kBK - 1) / kBK;
  const int kb0 = blockIdx.z * g.kb_per_split;
  const int n = min(nkb, kb0 + g.kb_per_split) - kb0;  // >= 1 by construction
  const uint32_t bytes = (uint32_t)(kBM + g.BN) * (uint32_t)(kBK * 2);
  // cluster (1, cm, splits): rank = ym + cm z; the cm row tiles of one split
  // share each B box, every CTA loading 1/cm of it for all of them
  const bool clustered = g.cm > 1 || g.splits > 1;
  const int ym = g.cm > 1 ? (int)(blockIdx.y & 1) : 0;
  const int zs = (int)blockIdx.z;
  const uint16_t bmask = (uint16_t)(((1u << g.cm) - 1u) << (g.cm * zs));
  const int bn_part = g.BN / g.cm;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, (uint32_t)g.cm);  // the MMA threads of every CTA sharing the stage's B box
    }
    mbar_init(accum, 1);
    mbar_init_fence();
    flags[0] = (clustered && cluster_rank() != (uint32_t)(ym + g.cm * zs)) ? 1 : 0;
    flags[1] = 0;
    flags[2] = 0;
  }
  if (warp == 1) {
    tmem_alloc(smem_addr(tslot), g.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  if (clustered) cluster_sync();  // every CTA's barriers initialised before any multicast reaches them
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0) {  // producer
    int i = 0;
    for (; i < n; ++i) {
      const int s = i % S;
      if (i >= S && !mbar_wait(empty + s, (uint32_t)(((i / S) - 1) & 1))) {
        flags[0] = 1;
        break;
      }
      mbar_expect_tx(full + s, bytes);  // A + the whole B box (its cm parts from cm CTAs)
      const int k0 = (kb0 + i) * kBK;
      tma_load_2d(sA + s * SB, &tmA, k0, m0, full + s);
      if (g.cm > 1)
        tma_load_2d_mc(sA + s * SB + kAStage + (uint32_t)(ym * bn_part * kBK * 2), &tmB, k0, n0 + ym * bn_part,
                       full + s, bmask);
      else
        tma_load_2d(sA + s * SB + kAStage, &tmB, k0, n0, full + s);
    }
    flags[1] = i;
  } else if (warp == 1 && lane == 0) {  // MMA issuer
    const uint32_t idesc = instr_desc(kBM, g.BN, 0, 0);
    int i = 0;
    for (; i < n; ++i) {
      const int s = i % S;
      if (!mbar_wait(full + s, (uint32_t)((i / S) & 1))) {
        flags[0] = 1;
        break;
      }
      tc_fence_after();
      const uint32_t a_s = sA + s * SB, b_s = a_s + kAStage;
#pragma unroll
      for (int k = 0; k < kBK / 16; ++k)  // 16 K-elements = 32 bytes further along each row
        mma_bf16(tmem, smem_desc_sw128(a_s + k * 32), smem_desc_sw128(b_s + k * 32), idesc,
                 (i > 0 || k > 0) ? 1u : 0u);
      if (g.cm > 1)
        mma_commit_mc(empty + s, bmask);  // the stage is free in every CTA only when all have read it
      else
        mma_commit(empty + s);
    }
    flags[2] = i;
    mma_commit(accum);  // every MMA issued above
  }
  bool ok = true;
  if (warp >= 2) {  // epilogue: accumulators -> shared memory tile
    if (!mbar_wait(accum, 0)) ok = false;
    tc_fence_after();
    float *tile = reinterpret_cast<float *>(base);
    const int pitch = g.BN + 4;
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int r = q * 32 + lane;
    if (ok) {
      for (int c0 = 0; c0 < g.BN; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
        float4 *dst = reinterpret_cast<float4 *>(tile + r * pitch + c0);
#pragma unroll
        for (int j = 0; j < 4; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
      }
    } else {
      flags[0] = 1;
    }
  }
  tc_fence_before();
  __syncthreads();  // tile in shared memory; every role's flags visible
  bool good = flags[0] == 0;
  const int rows = max(0, min(kBM, g.Mm - m0)), cols = min(g.BN, g.Nn - n0);  // 0: a padding row tile
  const int pitch = g.BN + 4;
  // rows this CTA writes: all of them, or with K split over the cluster its
  // share, summed over the cluster's partial tiles read from shared memory
  int r0 = 0, r1 = rows;
  uint32_t peer_tile[8] = {};
  if (g.splits > 1) {
    cluster_sync();  // every partial tile and error flag of the cluster is in place
    const int share = (rows + g.splits - 1) / g.splits;
    r0 = min(rows, zs * share);
    r1 = min(rows, r0 + share);
#pragma unroll
    for (int z = 0; z < 8; ++z) {
      if (z < g.splits) {
        const uint32_t pr = (uint32_t)(ym + g.cm * z);  // same row tile, split z
        peer_tile[z] = map_peer(smem_addr(base), pr);
        if (ld_peer_int(map_peer(smem_addr(flags), pr)) != 0) good = false;
      }
    }
  }
  if (g.splits > 1 && good) {
    // the cluster's sum of this CTA's rows: every thread takes 4 consecutive
    // columns (16-byte loads from each CTA's tile; this CTA's own from local
    // shared memory), four items at a time so that 4 x splits loads are in
    // flight; then bias, ReLU and the outputs
    constexpr int kItems = 4;
    const int c4n = (cols + 3) / 4;
    const int items = (r1 - r0) * c4n;
    const float *own = reinterpret_cast<const float *>(base);
    for (int it = tid; it < items; it += kItems * kTmaThreads) {
      float4 acc[kItems];
      int rr[kItems], c4[kItems];
#pragma unroll
      for (int h = 0; h < kItems; ++h) {
        const int k = it + h * kTmaThreads;
        rr[h] = k < items ? r0 + k / c4n : -1;
        c4[h] = k < items ? k % c4n : 0;
        acc[h] = rr[h] >= 0 ? *reinterpret_cast<const float4 *>(own + rr[h] * pitch + 4 * c4[h])
                            : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int z = 0; z < 8; ++z) {
        if (z < g.splits && z != zs) {
#pragma unroll
          for (int h = 0; h < kItems; ++h) {
            if (rr[h] >= 0) {
              const float4 v = ld_peer_v4(peer_tile[z] + (uint32_t)((rr[h] * pitch + 4 * c4[h]) * 4));
              acc[h].x += v.x;
              acc[h].y += v.y;
              acc[h].z += v.z;
              acc[h].w += v.w;
            }
          }
        }
      }
#pragma unroll
      for (int h = 0; h < kItems; ++h) {
        if (rr[h] < 0) continue;
        const float a4[4] = {acc[h].x, acc[h].y, acc[h].z, acc[h].w};
        const int64_t o = (int64_t)(m0 + rr[h]) * g.ldc + n0 + 4 * c4[h];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int cc = 4 * c4[h] + e;
          if (cc >= cols) break;
          float x = a4[e];
          if (g.accumulate) {
            g.Cf[o + e] += x;
            continue;
          }
          if (g.bias) x += g.bias[n0 + cc];
          if (g.relu) x = fmaxf(x, 0.f);
          if (g.Cf) g.Cf[o + e] = x;
          if (g.Cb) g.Cb[o + e] = __float2bfloat16(x);
        }
      }
    }
  } else if (warp >= 2 && good) {  // coalesced out, row by row
    const float *tile = reinterpret_cast<const float *>(base);
    for (int rr = r0 + warp - 2; rr < r1; rr += 4) {
      const int64_t o = (int64_t)(m0 + rr) * g.ldc + n0;
      for (int cc = lane; cc < cols; cc += 32) {
        float x = tile[rr * pitch + cc];
        if (g.accumulate) {
          g.Cf[o + cc] += x;
          continue;
        }
        if (g.bias) x += g.bias[n0 + cc];
        if (g.relu) x = fmaxf(x, 0.f);
        if (g.Cf) g.Cf[o + cc] = x;
        if (g.Cb) g.Cb[o + cc] = __float2bfloat16(x);
      }
    }
  }
  // the peers have read this CTA's tile, and every multicast write or
  // commit arrival aimed at this CTA has landed (all MMAs of the cluster done)
  if (clustered) cluster_sync();
  if (flags[0] != 0 && tid == 0) {
    atomicAdd(&g_timeouts, 1);
    // box loads issued and not consumed by an MMA land before the CTA's
    // shared memory is released; the MMAs issued finish before the tensor
    // memory is freed
    for (int i = flags[2]; i < flags[1]; ++i)
      mbar_wait(full + (i % S), (uint32_t)((i / S) & 1));
    mbar_wait(accum, 0);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, g.tmem_cols);
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

// Launch plan of one product.
// Copy-staged kernel: 256-column tiles (split evenly), K split over enough
// CTAs to fill the SMs (at least 4 K-blocks each), the partial tiles added
// into C with atomics.  TMA kernel: K split over at most 8 CTAs, a cluster
// that sums its partial tiles itself; the widest tile (256, 128 or 64
// columns) whose tiles x splits occupy three quarters of the SMs, else the
// tiling with the most CTAs.  split > 0 forces that split (256-column tiles).
struct TcPlan {
  int BN, tiles_n, tiles_m, nkb, kb_per_split, splits;
};
static void tc_split(TcPlan &p, int s) {
  if (s < 1) s = 1;
  if (s > p.nkb) s = p.nkb;
  p.kb_per_split = (p.nkb + s - 1) / s;
  p.splits = (p.nkb + p.kb_per_split - 1) / p.kb_per_split;  // every split has >= 1 K-block
}
static void tc_width(TcPlan &p, int Nn, int width) {
  p.tiles_n = (Nn + width - 1) / width;
  p.BN = ((Nn + p.tiles_n - 1) / p.tiles_n + 15) / 16 * 16;
}
static TcPlan tc_plan(int Mm, int Nn, int Kk, int split, bool tma) {
  TcPlan p{};
  const int sms = tc_num_sms();
  p.tiles_m = (Mm + tc::kBM - 1) / tc::kBM;
  p.nkb = (Kk + tc::kBK - 1) / tc::kBK;
  if (split > 0 || !tma) {
    tc_width(p, Nn, tc::kMaxBN);
    int s = split;
    if (s <= 0) {
      const int tiles = p.tiles_m * p.tiles_n;
      s = sms / (tiles > 0 ? tiles : 1);
      if (s > p.nkb / 4) s = p.nkb / 4;
    }
    if (tma && s > 8) s = 8;
    tc_split(p, s);
    return p;
  }
  TcPlan best{};
  int best_ctas = -1;
  for (int w = tc::kMaxBN; w >= 64; w /= 2) {
    TcPlan q = p;
    tc_width(q, Nn, w);
    const int tiles = q.tiles_m * q.tiles_n;
    int s = sms / (tiles > 0 ? tiles : 1);
    if (s > 8) s = 8;
    if (s > q.nkb / 4) s = q.nkb / 4;
    tc_split(q, s);
    const int ctas = tiles * q.splits;
    if (ctas * 4 >= sms * 3) return q;
    if (ctas > best_ctas) {
      best = q;
      best_ctas = ctas;
    }
  }
  return best;
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
// cuTensorMapEncodeTiled, fetched from the driver once (no link against libcuda)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    cudaDriverEntryPointQueryResult q{};
    void *f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)f;
    cudaGetLastError();
    looked_up = true;
  }
  return fn;
}

// 2-D map of a K-major [rows][K] BF16 operand with pitch ld elements: boxes of
// 64 K-elements (128 bytes) x box_rows, 128-byte swizzle, zero fill outside
static bool encode_kmajor(CUtensorMap *map, const void *base, int64_t ld, int rows, int Kk, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)Kk, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)tc::kBK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

mdhp_status gemm_tc(const __nv_bfloat16 *A, int64_t lda, int a_mn, const __nv_bfloat16 *B, int64_t ldb,
                    int b_mn, int Mm, int Nn, int Kk, const float *bias, int relu, float *Cf,
                    __nv_bfloat16 *Cb, int64_t ldc, int accumulate, int split, cudaStream_t st,
                    int staging) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(tc::k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(tc::k_gemm_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmem) !=
            cudaSuccess) {
      cudaGetLastError();
      record_error("gemm_tc: shared memory attribute");
      return MDHP_E_CUDA;
    }
    attr = true;
  }
  // K-major operands: boxes by the tensor-memory accelerator (staging 0);
  // otherwise, or staging 1, 16-byte copies by every thread
  CUtensorMap mA, mB;
  bool tma = staging == 0 && !a_mn && !b_mn && encode_fn() != nullptr;
  TcPlan p = tc_plan(Mm, Nn, Kk, split, tma);
  // two row tiles per cluster share each B box when the cluster stays within
  // 4 CTAs (the row-tile count is then padded to even); clusters of 8 CTAs
  // of this size do not all fit on the GPU at once (measured: 15 of 16)
  const int cm = (tma && p.tiles_m >= 2 && 2 * p.splits <= 4) ? 2 : 1;
  if (tma && !(encode_kmajor(&mA, A, lda, Mm, Kk, tc::kBM) && encode_kmajor(&mB, B, ldb, Nn, Kk, p.BN / cm))) {
    tma = false;
    p = tc_plan(Mm, Nn, Kk, split, false);
  }
  if ((accumulate || (!tma && p.splits > 1)) && !Cf) {
    record_error("gemm_tc: a K split or accumulation needs the FP32 output");
    return MDHP_E_ARG;
  }
  dim3 grid(p.tiles_n, tma ? (p.tiles_m + cm - 1) / cm * cm : p.tiles_m, p.splits);
  const bool finish = !tma && p.splits > 1 && !accumulate;
  if (tma) {
    tc::TmaArgs t{};
    t.Mm = Mm; t.Nn = Nn; t.Kk = Kk; t.BN = p.BN; t.kb_per_split = p.kb_per_split;
    t.splits = p.splits;
    t.cm = cm;
    t.stage_bytes = tc::kAStage + p.BN * tc::kBK * 2;
    t.stages = tc::kStages * (tc::kAStage + tc::kBStage) / t.stage_bytes;
    if (t.stages > tc::kTmaMaxStages) t.stages = tc::kTmaMaxStages;
    t.tmem_cols = p.BN <= 32 ? 32u : p.BN <= 64 ? 64u : p.BN <= 128 ? 128u : 256u;
    t.accumulate = accumulate ? 1 : 0;
    t.Cf = Cf;
    t.ldc = ldc;
    if (!accumulate) {
      t.bias = bias; t.relu = relu; t.Cb = Cb;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(tc::kTmaThreads, 1, 1);
    cfg.dynamicSmemBytes = tc::kSmem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1;
    at[0].val.clusterDim.y = (unsigned)cm;        // row tiles sharing each B box
    at[0].val.clusterDim.z = (unsigned)p.splits;  // the K splits of one tile
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, tc::k_gemm_tma, mA, mB, t) != cudaSuccess) {
      char buf[160];
      snprintf(buf, sizeof(buf), "gemm_tc: cluster launch: %s", cudaGetErrorString(cudaGetLastError()));
      record_error(buf);
      return MDHP_E_CUDA;
    }
  } else {
    tc::Args g{};
    g.A = A; g.B = B; g.lda = lda; g.ldb = ldb; g.a_mn = a_mn; g.b_mn = b_mn;
    g.Mm = Mm; g.Nn = Nn; g.Kk = Kk; g.BN = p.BN; g.kb_per_split = p.kb_per_split;
    g.ldc = ldc;
    if (accumulate || p.splits > 1) {
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
    tc::k_gemm_tc<<<grid, tc::kThreads, tc::kSmem, st>>>(g);
  }
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

// launches of one product (the TMA kernel sums its K split in the cluster;
// the copy-staged one adds a finishing launch)
int gemm_tc_launches(int Mm, int Nn, int Kk, int accumulate, int split, int a_mn, int b_mn, int staging) {
  const bool tma = staging == 0 && !a_mn && !b_mn && encode_fn() != nullptr;
  const TcPlan p = tc_plan(Mm, Nn, Kk, split, tma);
  return 1 + ((!tma && p.splits > 1 && !accumulate) ? 1 : 0);
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
