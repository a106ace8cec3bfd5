// mdhp_fit_batch_noalloc: batched fitting for callers that may not allocate
// device memory.  The plan-based entry point (mdhp_fit_batch) keeps its work
// queue, length order and sort workspace in memory the plan allocated with
// cudaMalloc.  Some callers cannot do that: a process whose device memory is
// all owned by a pooling allocator of another framework, an embedded or
// safety-critical deployment that forbids allocation after start-up (an
// in-vehicle detector running this fit on every window, for instance), or a
// host thread that must not risk the device-wide synchronisation cudaMalloc
// can imply.  This variant keeps the same scratch in one fixed array that is
// part of the library's device image instead.
//
// The array lives at file scope in device memory; every GPU that loads the
// library holds it until the process exits.  Host code may not use its name
// as a device address: the address is taken once per device with
// cudaGetSymbolAddress while that device is current, cached with the id of
// the context it belongs to (taken again in a new context, e.g. after
// cudaDeviceReset), and passed to the kernels.  All calls share the array, so calls that overlap on the GPU
// (two streams, or two host threads on one device) race on it.
#include <cuda.h>

#include <cstdio>
#include <mutex>

#include "mdhp.h"
#include "mdhp_dispatch.h"

namespace mdhp {

// Layout (int32): [0..31] per-bucket counts, [32..63] per-bucket cursors,
// [64] work-queue counter, [65..66] work range, [128, 128 + B) window order.
constexpr int kNaHead = 128;
static __device__ __align__(256) int g_noalloc_scratch[kNaHead + MDHP_NOALLOC_MAX_WINDOWS];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
int *g_na_ptr[kMaxDevices] = {};
unsigned long long g_na_ctx[kMaxDevices] = {};  // id of the context the address belongs to

// Unique id of the calling thread's current CUDA context (0 if unknown).
// Context ids are never reused within a process, so an address taken in a
// context that cudaDeviceReset has since destroyed is never mistaken for one
// of the new context.  The driver functions are reached through the
// runtime's entry-point query, so the library needs no link to libcuda.
unsigned long long current_ctx_id() {
  using GetCur = CUresult (*)(CUcontext *);
  using GetId = CUresult (*)(CUcontext, unsigned long long *);
  static GetCur get_cur = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    cudaDriverEntryPointQueryResult q1{}, q2{};
    void *f1 = nullptr, *f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) ==
            cudaSuccess && q1 == cudaDriverEntryPointSuccess)
      get_cur = (GetCur)f1;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess && q2 == cudaDriverEntryPointSuccess)
      get_id = (GetId)f2;
    cudaGetLastError();
    looked_up = true;
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_cur && get_id && get_cur(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS)
    return id;
  return 0;
}

// Address of the scratch array on the current device, taken once per device
// and context (the first call after a cudaDeviceReset takes it again).
int *na_scratch(mdhp_status *st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    *st = MDHP_E_CUDA;
    record_error("mdhp_fit_batch_noalloc: no current CUDA device");
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_na_mutex);
  // an address taken in another context (or with no context current, as
  // after a cudaDeviceReset before the runtime re-creates it) is taken again
  if (g_na_ptr[dev] && current_ctx_id() != g_na_ctx[dev]) g_na_ptr[dev] = nullptr;
  if (!g_na_ptr[dev]) {
    int *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      char buf[256];
      snprintf(buf, sizeof(buf), "mdhp_fit_batch_noalloc: cudaGetSymbolAddress: %s",
               cudaGetErrorString(e));
      record_error(buf);
      *st = MDHP_E_CUDA;
      return nullptr;
    }
    g_na_ptr[dev] = p;
    g_na_ctx[dev] = current_ctx_id();
  }
  return g_na_ptr[dev];
}

// Length buckets (floor(log2(N + 1)), 0..31) give a longest-first order
// without a sort workspace: count, scan (descending buckets), scatter.
__global__ void k_na_clear(int *s) {
  const int i = threadIdx.x;
  if (i < kNaHead) s[i] = 0;
}

__device__ __forceinline__ int na_bucket(const int64_t *offsets, int b) {
  const int64_t n = offsets[b + 1] - offsets[b];
  const unsigned long long v = (unsigned long long)(n < 0 ? 0 : n) + 1ull;
  const int lg = 63 - __clzll((long long)v);
  return lg > 31 ? 31 : lg;
}

__global__ void k_na_count(const int64_t *offsets, int B, int *s) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) atomicAdd(&s[na_bucket(offsets, b)], 1);
}

__global__ void k_na_scan(int B, int *s) {
  if (threadIdx.x == 0) {
    int run = 0;
    for (int k = 31; k >= 0; --k) {  // longest bucket first
      s[32 + k] = run;
      run += s[k];
    }
    s[64] = 0;
    s[65] = 0;
    s[66] = B;
  }
}

__global__ void k_na_scatter(const int64_t *offsets, int B, int *s) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) {
    const int pos = atomicAdd(&s[32 + na_bucket(offsets, b)], 1);
    s[kNaHead + pos] = b;
  }
}

}  // namespace
}  // namespace mdhp

using namespace mdhp;

extern "C" mdhp_status mdhp_fit_batch_noalloc(const mdhp_batch *batch, const mdhp_fit_opts *o,
                                              float *mu, float *alpha, float *beta,
                                              double *loglik, int32_t *iters,
                                              int32_t *win_status, void *stream) {
  char msg[256];
  if (!batch || !o) {
    record_error("mdhp_fit_batch_noalloc: batch/opts NULL");
    return MDHP_E_ARG;
  }
  if (batch->B < 0 || batch->M < 1 || batch->M > 64 || batch->n_events < 0) {
    record_error("mdhp_fit_batch_noalloc: bad batch sizes (B >= 0, 1 <= M <= 64)");
    return MDHP_E_ARG;
  }
  if (batch->B > MDHP_NOALLOC_MAX_WINDOWS) {
    snprintf(msg, sizeof(msg),
             "mdhp_fit_batch_noalloc: B = %d exceeds the fixed scratch capacity of %d windows "
             "(split the batch, or use mdhp_fit_batch with a plan)",
             batch->B, MDHP_NOALLOC_MAX_WINDOWS);
    record_error(msg);
    return MDHP_E_ARG;
  }
  if (batch->beta_mode != MDHP_BETA_SCALAR && batch->beta_mode != MDHP_BETA_PER_SOURCE) {
    record_error("mdhp_fit_batch_noalloc: beta_mode must be scalar or per-source");
    return batch->beta_mode == MDHP_BETA_MATRIX ? MDHP_E_UNSUPPORTED : MDHP_E_ARG;
  }
  if ((batch->B > 0 && (!batch->offsets || !batch->T_span)) ||
      (batch->n_events > 0 && (!batch->t || !batch->id)) || !mu || !alpha || !beta ||
      !loglik || !iters || !win_status || batch->max_events < 0) {
    record_error("mdhp_fit_batch_noalloc: NULL pointer or negative max_events");
    return MDHP_E_ARG;
  }
  if (o->max_iters < 1 || (o->optimizer != 0 && o->optimizer != 1) || o->patience < 1 ||
      o->init < 0 || o->init > 1) {
    record_error("mdhp_fit_batch_noalloc: bad options (init must be 0 or 1)");
    return MDHP_E_ARG;
  }
  mdhp_status st = MDHP_OK;
  int *s = na_scratch(&st);
  if (!s) return st;
  const int B = batch->B;
  if (B == 0) return MDHP_OK;
  cudaStream_t cs = (cudaStream_t)stream;

  // shape: the plan-based entry point's default shape for this width
  const int M = batch->M;
  const int Mt = M <= 4 ? 4 : M <= 8 ? 8 : M <= 16 ? 16 : M <= 32 ? 32 : 64;
  const Shape shape = default_shape(Mt);
  const int nt = shape.nt, spl = shape.spl, cutoff = shape.cutoff;
  const bool learn = o->fit_beta != 0;
  const bool stage = batch->max_events > 0 && batch->max_events <= cutoff;
  FitFn fn = get_fit(Mt, spl, batch->beta_mode, learn, stage);
  if (!fn) {
    record_error("mdhp_fit_batch_noalloc: no kernel for this shape");
    return MDHP_E_UNSUPPORTED;
  }

  k_na_clear<<<1, kNaHead, 0, cs>>>(s);
  k_na_count<<<(B + 255) / 256, 256, 0, cs>>>(batch->offsets, B, s);
  k_na_scan<<<1, 32, 0, cs>>>(B, s);
  k_na_scatter<<<(B + 255) / 256, 256, 0, cs>>>(batch->offsets, B, s);

  FitArgs a{};
  a.offsets = batch->offsets; a.t = batch->t; a.id = batch->id; a.T = batch->T_span;
  a.w = batch->weights; a.mu = mu; a.alpha = alpha; a.beta = beta; a.loglik = loglik;
  a.iters = iters; a.status = win_status;
  a.order = s + kNaHead;
  a.queue = s + 64;
  a.range = s + 65;
  a.Mrt = M; a.NC = nt / spl;
  a.ev_cap = stage ? batch->max_events : 0;
  a.optimizer = o->optimizer; a.max_iters = o->max_iters; a.fit_beta = o->fit_beta;
  a.patience = o->patience; a.init = o->init; a.lr = o->lr; a.mu_floor = o->mu_floor;
  a.alpha_floor = o->alpha_floor; a.beta_floor = o->beta_floor; a.b1 = o->adam_b1;
  a.b2 = o->adam_b2; a.eps = o->adam_eps; a.tol = o->tol;
  a.xbuf = nullptr;
  a.carve = make_carve(Mt, nt, spl, a.ev_cap, batch->weights != nullptr, learn, o->optimizer == 1,
                       true, Mt <= 32);
  int dev = 0, optin = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (a.carve.total > optin) {
    snprintf(msg, sizeof(msg), "mdhp_fit_batch_noalloc: shared memory %d > %d (lower max_events)",
             a.carve.total, optin);
    record_error(msg);
    return MDHP_E_ARG;
  }
  if (a.carve.total > 48 * 1024 &&
      cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           a.carve.total) != cudaSuccess) {
    cudaGetLastError();
    record_error("mdhp_fit_batch_noalloc: cudaFuncSetAttribute failed");
    return MDHP_E_CUDA;
  }
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, nt, a.carve.total);
  int grid = sms * (occ > 0 ? occ : 1);
  if (grid > B) grid = B;
  fn<<<grid, nt, a.carve.total, cs>>>(a);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "mdhp_fit_batch_noalloc: launch: %s", cudaGetErrorString(e));
    record_error(msg);
    return MDHP_E_CUDA;
  }
  return MDHP_OK;
}
