// mdhp_simulate: bulk simulation of exponential-kernel MDHP windows on the GPU
// (training and test data for the learned initializer and the fits).
//
// Ogata's thinning (Ogata, IEEE Trans. Inf. Theory 27(1), 1981) for the
// intensity of Sec. II, lambda_i(t) = mu_i + sum_j alpha_ij sum_{t_k < t, u_k = j}
// exp(-beta_j (t - t_k)), with the superposition split: the total intensity
// Lambda = sum_i mu_i + sum_j c_j R_j (c_j = sum_i alpha_ij) only decays between
// events, so its value just after the current time bounds it until the next
// event; an accepted point goes to the background (type i with probability
// mu_i / sum mu) or to source j (probability c_j R_j), then to target i with
// probability alpha_ij / c_j.  The type is therefore drawn from lambda_i / Lambda.
//
// One thread per window, in FP64: the thinning loop is a long serial chain per
// window, and GB300's FP64 pipe is narrow, so lanes that each run a different
// window (no per-window reductions, no replicated scalar work) use it best.
// The per-source states R_j, their column sums c_j and decays beta_j sit in
// shared memory, [j][thread], so a warp's accesses to one j are conflict-free.
// With a scalar beta all states decay by one factor, computed once per
// candidate.  Windows are taken in the caller's order (longest first keeps the
// lanes of a warp busy for similar times).
//
// Random numbers: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) as a counter-
// based generator, u_k = mix(key + k * 0x9e3779b97f4a7c15) >> 11 scaled to
// [0, 1), one key per window derived from (seed, stream id, window index).
// Uniforms are drawn in a fixed order per candidate (gap, acceptance, then on
// acceptance the component and, for an excitation, the target), so a window's
// events depend only on its key and parameters, not on the launch.
#include <cstdint>
#include <cstdio>

#include "mdhp.h"
#include "mdhp_dispatch.h"

namespace mdhp {
namespace {

constexpr int kSimThreads = 64;

__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double sm64_u01(uint64_t key, uint64_t &ctr) {
  ctr += 1;
  const uint64_t z = sm64_mix(key + ctr * 0x9e3779b97f4a7c15ull);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ uint64_t sim_key(uint64_t seed, uint64_t stream_id, uint64_t w) {
  return sm64_mix(sm64_mix(sm64_mix(seed) ^ (stream_id + 0x632be59bd9b4e019ull)) ^ (w + 1));
}

struct SimArgs {
  int M, mode, B;
  const double *mu, *alpha, *beta;
  const int64_t *offsets;
  const int32_t *order;
  uint64_t seed, stream_id, first_window;
  float *t;
  int16_t *id;
  float *T;
  int32_t *status;
};

__device__ __forceinline__ bool finite_nonneg(double x) { return x >= 0.0 && x <= 1.79e308; }

__global__ void __launch_bounds__(kSimThreads) k_simulate(SimArgs a) {
  extern __shared__ double sh[];
  const int tid = threadIdx.x;
  const int64_t r = (int64_t)blockIdx.x * kSimThreads + tid;
  if (r >= a.B) return;
  const int b = a.order ? a.order[r] : (int)r;
  if (b < 0 || b >= a.B) return;
  const int M = a.M;
  const int nb = a.mode == 0 ? 1 : M;
  double *R = sh + tid;                        // R_j   at R[j * kSimThreads]
  double *C = sh + M * kSimThreads + tid;      // c_j
  double *D = sh + 2 * M * kSimThreads + tid;  // beta_j (per-source mode)
  const double *mu = a.mu + (int64_t)b * M;
  const double *al = a.alpha + (int64_t)b * M * M;
  const double *be = a.beta + (int64_t)b * nb;
  const int64_t o = a.offsets[b];
  const int64_t n_target = a.offsets[b + 1] - o;

  bool ok = n_target >= 0;
  double mu_tot = 0.0;
  for (int i = 0; i < M; ++i) {
    const double m = mu[i];
    ok &= finite_nonneg(m);
    mu_tot += m;
  }
  for (int j = 0; j < M; ++j) {
    double c = 0.0;
    for (int i = 0; i < M; ++i) {
      const double x = al[(int64_t)i * M + j];
      ok &= finite_nonneg(x);
      c += x;
    }
    C[j * kSimThreads] = c;
    R[j * kSimThreads] = 0.0;
  }
  for (int j = 0; j < nb; ++j) {
    const double x = be[j];
    ok &= x > 0.0 && x <= 1.79e308;
    if (a.mode == 1) D[j * kSimThreads] = x;
  }
  if (!ok) {
    a.status[b] = MDHP_E_ARG;
    a.T[b] = 0.0f;
    return;
  }
  const double beta0 = be[0];
  const uint64_t key = sim_key(a.seed, a.stream_id, a.first_window + (uint64_t)b);
  uint64_t ctr = 0;

  double t = 0.0, lam_bar = mu_tot, T_span = 0.0;  // no excitation yet
  int64_t n = 0, cand = 0;
  const int64_t cand_cap = 256 * (n_target + 16);
  int st = MDHP_OK;
  float t_last = 0.0f;
  for (;;) {
    if (!(lam_bar > 0.0)) {  // no intensity left: the window cannot be completed
      T_span = t;
      if (n < n_target) st = MDHP_E_SIM_STALLED;
      break;
    }
    if (++cand > cand_cap) {
      T_span = t;
      st = MDHP_E_SIM_STALLED;
      break;
    }
    const double e = -log1p(-sm64_u01(key, ctr));
    const double tc = t + e / lam_bar;
    const double dt = tc - t;
    double lam = mu_tot;
    if (a.mode == 0) {
      const double d = exp(-beta0 * dt);
      for (int j = 0; j < M; ++j) {
        const double rj = R[j * kSimThreads] * d;
        R[j * kSimThreads] = rj;
        lam += C[j * kSimThreads] * rj;
      }
    } else {
      for (int j = 0; j < M; ++j) {
        const double rj = R[j * kSimThreads] * exp(-D[j * kSimThreads] * dt);
        R[j * kSimThreads] = rj;
        lam += C[j * kSimThreads] * rj;
      }
    }
    t = tc;
    const double u = sm64_u01(key, ctr) * lam_bar;
    if (!(u <= lam)) {  // rejected: the intensity just after t bounds what follows
      lam_bar = lam;
      continue;
    }
    if (n == n_target) {  // the (N+1)-th point closes the observation window
      T_span = t;
      break;
    }
    double v = sm64_u01(key, ctr) * lam;
    int ty = -1;
    if (v < mu_tot) {
      for (int i = 0; i < M; ++i) {
        const double m = mu[i];
        if (v < m) { ty = i; break; }
        v -= m;
      }
      if (ty < 0) ty = M - 1;
    } else {
      v -= mu_tot;
      int src = -1;
      for (int j = 0; j < M; ++j) {
        const double q = C[j * kSimThreads] * R[j * kSimThreads];
        if (v < q) { src = j; break; }
        v -= q;
      }
      if (src < 0) src = M - 1;
      double v2 = sm64_u01(key, ctr) * C[src * kSimThreads];
      for (int i = 0; i < M; ++i) {
        const double x = al[(int64_t)i * M + src];
        if (v2 < x) { ty = i; break; }
        v2 -= x;
      }
      if (ty < 0) ty = M - 1;
    }
    t_last = (float)t;
    a.t[o + n] = t_last;
    a.id[o + n] = (int16_t)ty;
    ++n;
    R[ty * kSimThreads] += 1.0;
    lam_bar = mu_tot;  // intensity just after the new event, summed as above
    for (int j = 0; j < M; ++j) lam_bar += C[j * kSimThreads] * R[j * kSimThreads];
  }
  float Tf = (float)T_span;
  if (n > 0 && Tf < t_last) Tf = t_last;  // float rounding must not put T_span before the last event
  a.T[b] = Tf;
  a.status[b] = st;
}

}  // namespace
}  // namespace mdhp

using namespace mdhp;

extern "C" mdhp_status mdhp_simulate(int32_t M, int32_t beta_mode, int32_t B, const double *mu,
                                     const double *alpha, const double *beta,
                                     const int64_t *offsets, const int32_t *order, uint64_t seed,
                                     uint64_t stream_id, uint64_t first_window, float *t,
                                     int16_t *id, float *T_span, int32_t *win_status,
                                     void *stream) {
  if (M < 1 || M > 64) {
    record_error("mdhp_simulate: M must be 1..64");
    return MDHP_E_ARG;
  }
  if (beta_mode == MDHP_BETA_MATRIX) {
    record_error("mdhp_simulate: matrix-shaped beta is not supported");
    return MDHP_E_UNSUPPORTED;
  }
  if (beta_mode != MDHP_BETA_SCALAR && beta_mode != MDHP_BETA_PER_SOURCE) {
    record_error("mdhp_simulate: bad beta_mode");
    return MDHP_E_ARG;
  }
  if (B < 0) {
    record_error("mdhp_simulate: B < 0");
    return MDHP_E_ARG;
  }
  if (B == 0) return MDHP_OK;
  if (!mu || !alpha || !beta || !offsets || !t || !id || !T_span || !win_status) {
    record_error("mdhp_simulate: NULL argument");
    return MDHP_E_ARG;
  }
  SimArgs a{M, beta_mode, B, mu, alpha, beta, offsets, order, seed, stream_id, first_window,
            t, id, T_span, win_status};
  const size_t smem = (size_t)3 * M * kSimThreads * sizeof(double);
  static_assert(3 * 64 * kSimThreads * sizeof(double) <= 227 * 1024, "shared memory");
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k_simulate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess) {
    cudaGetLastError();
    record_error("mdhp_simulate: cannot raise the shared-memory limit");
    return MDHP_E_CUDA;
  }
  const int grid = (int)(((int64_t)B + kSimThreads - 1) / kSimThreads);
  k_simulate<<<grid, kSimThreads, smem, (cudaStream_t)stream>>>(a);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    char buf[256];
    snprintf(buf, sizeof(buf), "mdhp_simulate: launch: %s", cudaGetErrorString(e));
    record_error(buf);
    return MDHP_E_CUDA;
  }
  return MDHP_OK;
}
