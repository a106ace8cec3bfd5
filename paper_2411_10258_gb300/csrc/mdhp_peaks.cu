// Throughput probes of the arithmetic pipes the fit kernels use: FP32 FMA
// and the multi-function unit's approximate ex2, lg2 and reciprocal.  They
// give the rooflines of the benchmark a measured denominator on the GPU at
// hand instead of a datasheet figure.
//
// Each probe fills every SM to its thread limit with CTAs whose threads run
// independent dependency chains of one operation (enough chains per warp and
// warps per scheduler to hide the pipe's latency), times the launch with CUDA
// events on the caller's stream, and reports operations per second.  The
// chains are bounded maps (contractions towards a fixed point) so values stay
// normal, and their results feed a conditional store that never fires but
// keeps the compiler from removing the work.
#include <cuda_runtime.h>

#include <cstdio>

#include "mdhp.h"

namespace mdhp {

void record_error(const char *msg);  // mdhp_api.cu

static __device__ float g_probe_sink;

namespace {

constexpr int kProbeThreads = 256;

// x <- x b + c, fixed point c / (1 - b); kChains independent chains per thread
template <int kChains>
__global__ void __launch_bounds__(kProbeThreads) k_probe_fma(int iters, float b, float c) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 0.001f * (float)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], b, c);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == -1.f) g_probe_sink = s;
}

__device__ __forceinline__ float mufu(int op, float x) {
  float y;
  if (op == 0) {
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  } else if (op == 1) {
    asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  } else {
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  }
  return y;
}

// op 0: x <- 2^(-x) on (0, 1]; op 1: x <- log2(x + 2) on [1, 2];
// op 2: x <- 1 / (x + 1) on (0, 1].  One FP32 add or negation per MUFU op,
// which runs on the FMA pipe and is not the bound (the MUFU issue rate is a
// fraction of the FMA rate).
template <int OP, int kChains>
__global__ void __launch_bounds__(kProbeThreads) k_probe_mufu(int iters) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 0.25f + 0.001f * (float)((threadIdx.x + k) & 255);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) {
        if (OP == 0) x[k] = mufu(0, -x[k]);
        else if (OP == 1) x[k] = mufu(1, x[k] + 2.f);
        else x[k] = mufu(2, x[k] + 1.f);
      }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == -1.f) g_probe_sink = s;
}

template <typename F>
mdhp_status time_launch(F launch, cudaStream_t st, float *best_ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    record_error("mdhp_probe_peak: cudaEventCreate failed");
    cudaGetLastError();
    return MDHP_E_CUDA;
  }
  float best = -1.f;
  mdhp_status s = MDHP_OK;
  for (int rep = 0; rep < 4; ++rep) {  // the first run warms up
    cudaEventRecord(e0, st);
    launch();
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      char buf[256];
      snprintf(buf, sizeof(buf), "mdhp_probe_peak: %s", cudaGetErrorString(cudaGetLastError()));
      record_error(buf);
      s = MDHP_E_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best < 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *best_ms = best;
  return s;
}

}  // namespace
}  // namespace mdhp

using namespace mdhp;

extern "C" mdhp_status mdhp_probe_peak(int32_t what, double *ops_per_s, float *ms, void *stream) {
  if (!ops_per_s || what < 0 || what > 3) {
    record_error("mdhp_probe_peak: bad argument");
    return MDHP_E_ARG;
  }
  int dev = 0, sms = 0, thr = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&thr, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess) {
    cudaGetLastError();
    record_error("mdhp_probe_peak: no CUDA device");
    return MDHP_E_CUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int grid = sms * (thr / kProbeThreads);
  const double threads = (double)grid * kProbeThreads;
  float best = -1.f;
  double ops = 0.0;
  mdhp_status s;
  if (what == 0) {
    constexpr int kChains = 8;
    const int iters = 16384;  // 16 x 8 FMA per trip
    s = time_launch([&] { k_probe_fma<kChains><<<grid, kProbeThreads, 0, st>>>(iters, 0.999f, 0.001f); },
                    st, &best);
    ops = threads * iters * 16.0 * kChains * 2.0;  // an FMA is 2 floating-point operations
  } else {
    constexpr int kChains = 4;
    const int iters = 8192;  // 8 x 4 MUFU ops per trip
    if (what == 1)
      s = time_launch([&] { k_probe_mufu<0, kChains><<<grid, kProbeThreads, 0, st>>>(iters); }, st, &best);
    else if (what == 2)
      s = time_launch([&] { k_probe_mufu<1, kChains><<<grid, kProbeThreads, 0, st>>>(iters); }, st, &best);
    else
      s = time_launch([&] { k_probe_mufu<2, kChains><<<grid, kProbeThreads, 0, st>>>(iters); }, st, &best);
    ops = threads * iters * 8.0 * kChains;
  }
  if (s != MDHP_OK) return s;
  if (best <= 0.f) {
    record_error("mdhp_probe_peak: no timing");
    return MDHP_E_CUDA;
  }
  *ops_per_s = ops / (best * 1e-3);
  if (ms) *ms = best;
  return MDHP_OK;
}
