// Kernels of the MDHP-GDS library (sm_103a).  See mdhp_solver.cuh for the
// recursion and the chunk decomposition.
#pragma once

#include <type_traits>

#include "mdhp_solver.cuh"

namespace mdhp {

struct LlgArgs {
  const int64_t *offsets;
  const float *t;
  const int16_t *id;
  const float *T;
  const float *w;
  const float *mu, *alpha, *beta;
  double *loglik;
  float *g_mu, *g_alpha, *g_beta, *r_out;
  int32_t *status;
  int B, Mrt, NC, ev_cap;
  Carve carve;
};

struct FitArgs {
  const int64_t *offsets;
  const float *t;
  const int16_t *id;
  const float *T;
  const float *w;
  float *mu, *alpha, *beta;  // in/out
  double *loglik;
  int32_t *iters, *status;
  const int *order;  // window order (length-sorted), nullptr = identity
  int *queue;        // work counter, zero at launch
  const int *range;  // device [begin, end) of order positions, or nullptr
  int qbegin, qend;
  int Mrt, NC, ev_cap;
  int optimizer, max_iters, fit_beta, patience, init;
  float lr, mu_floor, alpha_floor, beta_floor, b1, b2, eps;
  double tol;
  float4 *xbuf;  // decoupled fit: per-CTA feature scratch (global), or nullptr
  float *pbuf;   // recursion fit: per-CTA slot (pstride floats) for theta_{k-1}, or nullptr
  int pstride;   //   (nullptr: theta_{k-1} is kept in shared memory)
  int pipe_steps, pipe_stages;  // streamed features: bulk-copy ring (0 stages: register prefetch)
  // decoupled fit, two launches sharing one length-sorted range: qdir 1 takes
  // windows from the front (longest first), qdir 2 from the back; dq =
  // {claimed, front, back} counters; 0 = the single-ended queue `queue`
  int qdir;
  int *dq;
  int slot_base;  // first feature-scratch slot of this launch
  // recursion fit, streamed events: 1 = pass 2 reads them through the
  // bulk-copy ring (batch arrays 16-byte aligned, no weights); n_total =
  // events in the batch arrays (the copies are clamped to them)
  int ring;
  int64_t n_total;
  // bulk-copy rings (features, events): polls of a consumer's wait, 0 = the
  // default bound (kWaitPolls suspending polls)
  uint32_t wait_polls;
  // decoupled fit with tensor-memory feature rows (XM_TMEM): columns this CTA
  // allocates (a power of two, 32..512; the CTAs resident on one SM together
  // take at most 512)
  int tmem_cols;
  int smem_steps;  //   and steps per thread kept in shared memory after the carve
  Carve carve;
};

struct WgArgs {
  const int64_t *offsets;
  const float *t;
  const int16_t *id;
  const float *T;
  const float *alpha, *beta;
  const float *r;      // 1/lambda per event from the forward pass
  float *g_w;          // out
  const int32_t *status;
  int Mrt, NC;
};

// Load the window's parameters into shared memory (alpha padded with zeros).
template <int M, int BM>
__device__ void load_params(int b, int Mrt, const float *mu, const float *alpha, const float *beta,
                            Sm<M> &sm) {
  constexpr int AP = M + 4;
  const int nb = BM == 0 ? 1 : Mrt;
  for (int p = threadIdx.x; p < M * AP; p += blockDim.x) {
    const int i = p / AP, j = p % AP;
    sm.alpha[p] = (i < Mrt && j < Mrt) ? alpha[(int64_t)b * Mrt * Mrt + i * Mrt + j] : 0.f;
  }
  for (int j = threadIdx.x; j < M; j += blockDim.x) sm.mu[j] = j < Mrt ? mu[(int64_t)b * Mrt + j] : 0.f;
  if (BM == 2) {  // matrix beta [i][j] (pitch M in shared memory; 1 in padding)
    for (int p = threadIdx.x; p < M * M; p += blockDim.x) {
      const int i = p / M, j = p % M;
      const float bv = (i < Mrt && j < Mrt) ? beta[(int64_t)b * Mrt * Mrt + i * Mrt + j] : 1.f;
      sm.beta[p] = bv;
      sm.bl2[p] = bv * kLog2e;
    }
    return;
  }
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    const float bv = (j < nb) ? beta[(int64_t)b * nb + j] : 1.f;
    sm.beta[j] = bv;
    sm.bl2[j] = bv * kLog2e;
  }
}

template <int M, int SPL, int BM, bool LEARN, bool STAGE>
__global__ void __launch_bounds__(256, 2) k_loglik_grad(LlgArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  Sm<M> sm;
  sm.bind(smem, a.carve);
  constexpr int AP = M + 1;
  const int b = blockIdx.x;
  const int Mrt = a.Mrt;
  const int64_t o0 = a.offsets[b];
  const int N = (int)(a.offsets[b + 1] - o0);
  const float T = a.T[b];
  const float *tg = a.t + o0;
  const int16_t *ug = a.id + o0;
  const float *wg = a.w ? a.w + o0 : nullptr;
  int st;
  if (STAGE && N > a.ev_cap) {
    st = kE_ARG;
  } else {
    st = stage_and_validate<M, STAGE>(tg, ug, wg, N, T, Mrt, sm);
  }
  const int nb = BM == 0 ? 1 : Mrt;
  if (st != kOK) {
    if (threadIdx.x == 0) {
      a.status[b] = st;
      a.loglik[b] = __longlong_as_double(0x7ff8000000000000LL);
    }
    for (int p = threadIdx.x; p < Mrt * Mrt; p += blockDim.x) a.g_alpha[(int64_t)b * Mrt * Mrt + p] = 0.f;
    for (int p = threadIdx.x; p < Mrt; p += blockDim.x) a.g_mu[(int64_t)b * Mrt + p] = 0.f;
    if (a.g_beta)
      for (int p = threadIdx.x; p < nb; p += blockDim.x) a.g_beta[(int64_t)b * nb + p] = 0.f;
    return;
  }
  load_params<M, BM>(b, Mrt, a.mu, a.alpha, a.beta, sm);
  clear_accumulators<M, SPL>(sm);
  __syncthreads();
  constexpr bool FIXED = STAGE && !LEARN && BM == 0;
  if (STAGE) {
    const EvS ev{sm.ev_t, sm.ev_u, wg ? sm.ev_w : nullptr};
    setup_chunks(a.NC, N, T, ev, sm.bnd, sm.anc);
    prepare_states<M, SPL, BM, LEARN>(a.NC, ev, Mrt, sm);
    if (FIXED) to_decays<M, SPL>(a.NC, sm);
    evaluate<M, SPL, BM, LEARN, FIXED>(a.NC, ev, T, Mrt, sm, a.r_out ? a.r_out + o0 : nullptr);
  } else {
    const EvG ev{tg, ug, wg};
    setup_chunks(a.NC, N, T, ev, sm.bnd, sm.anc);
    prepare_states<M, SPL, BM, LEARN>(a.NC, ev, Mrt, sm);
    evaluate<M, SPL, BM, LEARN, false>(a.NC, ev, T, Mrt, sm, a.r_out ? a.r_out + o0 : nullptr);
  }
  double lnl = 0.0;
  int bad = 0;
  if (threadIdx.x == 0) {
    lnl = lnl_total(sm);
    bad = !isfinite(lnl);
  }
  const int np = Mrt + Mrt * Mrt + (LEARN ? nb : 0);
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    const float g = grad_of<M, SPL, BM, LEARN>(p, Mrt, T, sm);
    bad |= !isfinite(g);
    if (p < Mrt) {
      a.g_mu[(int64_t)b * Mrt + p] = g;
    } else if (p < Mrt + Mrt * Mrt) {
      a.g_alpha[(int64_t)b * Mrt * Mrt + (p - Mrt)] = g;
    } else if (a.g_beta) {
      a.g_beta[(int64_t)b * nb + (p - Mrt - Mrt * Mrt)] = g;
    }
  }
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    a.loglik[b] = lnl;
    a.status[b] = bad ? kE_NONFINITE : kOK;
  }
  (void)AP;
}

// Iterations of one window (events accessed through ev); returns nothing, writes
// the window's outputs.  See the header's description of the iteration.
template <int M, int SPL, int BM, bool LEARN, typename EV>
__device__ void fit_window(const FitArgs &a, int b, int N, float T, const EV &ev, Sm<M> &sm) {
  constexpr int AP = M + 4;
  const int Mrt = a.Mrt;
  const int nb = BM == 0 ? 1 : Mrt;
  const int np = Mrt + Mrt * Mrt + nb;
  const int nupd = a.fit_beta ? np : Mrt + Mrt * Mrt;
  const int tid = threadIdx.x;
  // theta_{k-1} (restored after a non-finite evaluation), the gradient
  // buffer and the Adam moments: the CTA's device slot (four blocks of
  // pstride / 4 floats) when the launch provides one, else shared memory
  float *slotp = a.pbuf ? a.pbuf + (size_t)blockIdx.x * a.pstride : nullptr;
  const int pq = a.pstride / 4;
  float *prevp = slotp ? slotp : sm.prev;
  float *gbp = slotp ? slotp + pq : sm.gbuf;
  float *amp = slotp ? slotp + 2 * pq : sm.am;
  float *avp = slotp ? slotp + 3 * pq : sm.av;
  if (a.optimizer == 1) {
    for (int p = tid; p < np; p += blockDim.x) {
      amp[p] = 0.f;
      avp[p] = 0.f;
    }
  }
  constexpr bool FIXED = std::is_same<EV, EvS>::value && !LEARN && BM == 0;
  setup_chunks(a.NC, N, T, ev, sm.bnd, sm.anc);
  if (!LEARN) prepare_states<M, SPL, BM, false>(a.NC, ev, Mrt, sm);
  if (FIXED) to_decays<M, SPL>(a.NC, sm);
  const float invN = 1.f / (float)max(N, 1);
  // convergence bookkeeping lives in thread 0; decisions go through ctl[2]
  FF lnl_prev{0.f, 0.f}, lnl_out{0.f, 0.f};
  const bool use_tol = a.tol > 0.0;
  const float tolf = (float)a.tol;
  int streak = 0, k = 0;
  int wst = a.tol > 0.0 ? kE_MAXITER : kOK;
  float b1t = 1.f, b2t = 1.f;
  for (k = 0; k < a.max_iters; ++k) {
    if (LEARN) prepare_states<M, SPL, BM, LEARN>(a.NC, ev, Mrt, sm);
    evaluate<M, SPL, BM, LEARN, FIXED>(a.NC, ev, T, Mrt, sm, nullptr);
    int bad = 0;
    if (tid == 0) {
      const FF val = lnl_total_ff(sm);
      bad = !isfinite(val.hi);
      int decision = 0;  // 0 update, 1 stop
      if (!bad) {
        if (k > 0 && use_tol && ff_small_change(val, lnl_prev, tolf)) ++streak;
        else streak = 0;
        lnl_prev = val;
        lnl_out = val;
        if (use_tol && streak >= a.patience) { wst = kOK; decision = 1; }
        else if (k == a.max_iters - 1) decision = 1;
      } else if (k == 0) {
        lnl_out = val;
      }
      sm.ctl[2] = decision;
    }
    for (int p = tid; p < np; p += blockDim.x) {
      const float g = grad_of<M, SPL, BM, LEARN>(p, Mrt, T, sm);
      bad |= !isfinite(g);
      gbp[p] = g;
    }
    bad = __syncthreads_or(bad);
    if (bad) {
      if (k > 0) {
        for (int p = tid; p < nupd; p += blockDim.x) param_ref<M>(p, Mrt, sm) = prevp[p];
      }
      wst = kE_NONFINITE;
      __syncthreads();
      break;
    }
    if (sm.ctl[2]) { ++k; break; }
    b1t *= a.b1;
    b2t *= a.b2;
    const float c1 = 1.f / (1.f - b1t), c2 = 1.f / (1.f - b2t);  // Adam bias corrections
    for (int p = tid; p < nupd; p += blockDim.x) {
      const float g = gbp[p] * invN;
      float &th = param_ref<M>(p, Mrt, sm);
      float step;
      if (a.optimizer == 1) {
        const float m1 = a.b1 * amp[p] + (1.f - a.b1) * g;
        const float m2 = a.b2 * avp[p] + (1.f - a.b2) * g * g;
        amp[p] = m1;
        avp[p] = m2;
        step = a.lr * (m1 * c1) * rcp_ftz(sqrt_ftz(m2 * c2) + a.eps);  // as in the decoupled fit
      } else {
        step = a.lr * g;
      }
      const float fl = p < Mrt ? a.mu_floor : (p < Mrt + Mrt * Mrt ? a.alpha_floor : a.beta_floor);
      prevp[p] = th;
      th = fmaxf(th + step, fl);
    }
    __syncthreads();  // the event sums were read; parameters updated
    clear_accumulators<M, SPL>(sm);
    if (LEARN) {
      for (int j = tid; j < M; j += blockDim.x) sm.bl2[j] = sm.beta[j] * kLog2e;
    }
    __syncthreads();
  }
  // write back the last evaluated point
  for (int p = tid; p < Mrt * Mrt; p += blockDim.x)
    a.alpha[(int64_t)b * Mrt * Mrt + p] = sm.alpha[(p / Mrt) * AP + (p % Mrt)];
  for (int i = tid; i < Mrt; i += blockDim.x) a.mu[(int64_t)b * Mrt + i] = sm.mu[i];
  for (int j = tid; j < nb; j += blockDim.x) a.beta[(int64_t)b * nb + j] = sm.beta[j];
  if (tid == 0) {
    a.loglik[b] = ff_to_double(lnl_out);
    a.iters[b] = k;
    a.status[b] = wst;
  }
  __syncthreads();
}

template <int M, int SPL, int BM, bool LEARN, bool STAGE>
__global__ void __launch_bounds__(256, 2) k_fit(FitArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  Sm<M> sm;
  sm.bind(smem, a.carve);
  constexpr int AP = M + 4;
  const int Mrt = a.Mrt;
  const int nb = BM == 0 ? 1 : Mrt;
  const int np = Mrt + Mrt * Mrt + nb;
  const int tid = threadIdx.x;
  if (!STAGE && a.ring) {  // the streamed events' ring: one mbarrier per chunk and stage
    if (tid == 0) {
      for (int q = 0; q < a.NC * kRingD; ++q) mbar_init(sm.rbar + q, 1);
      mbar_init_fence();
      sm.ctl[4] = 0;
    }
    for (int c = tid; c < a.NC; c += blockDim.x) sm.rfill[c] = 0;
    __syncthreads();
  }
  for (;;) {
    if (tid == 0) sm.ctl[1] = atomicAdd(a.queue, 1);
    __syncthreads();
    const int q = sm.ctl[1];
    const int qb = a.range ? a.range[0] : a.qbegin;
    const int qe = a.range ? a.range[1] : a.qend;
    __syncthreads();
    if (qb + q >= qe) break;
    const int b = a.order ? a.order[qb + q] : qb + q;
    const int64_t o0 = a.offsets[b];
    const int N = (int)(a.offsets[b + 1] - o0);
    const float T = a.T[b];
    const float *tg = a.t + o0;
    const int16_t *ug = a.id + o0;
    const float *wg = a.w ? a.w + o0 : nullptr;
    int st;
    if (STAGE && N > a.ev_cap) {
      st = kE_ARG;
    } else {
      st = stage_and_validate<M, STAGE>(tg, ug, wg, N, T, Mrt, sm);
    }
    if (st != kOK) {
      if (tid == 0) {
        a.status[b] = st;
        a.loglik[b] = __longlong_as_double(0x7ff8000000000000LL);
        a.iters[b] = 0;
      }
      __syncthreads();
      continue;
    }
    // starting point
    load_params<M, BM>(b, Mrt, a.mu, a.alpha, a.beta, sm);
    clear_accumulators<M, SPL>(sm);
    __syncthreads();
    if (a.init == 1) {  // cold start: mu_i = 0.5 max(N_i,1)/T, alpha_ij = 0.5 beta_ij / M
      for (int p = tid; p < Mrt * Mrt; p += blockDim.x) {
        const int i = p / Mrt, j = p % Mrt;
        sm.alpha[i * AP + j] = 0.5f * sm.beta[BM == 0 ? 0 : j] / (float)Mrt;
      }
      for (int i = tid; i < Mrt; i += blockDim.x)
        sm.mu[i] = 0.5f * (float)max(sm.cnt[i], 1) / T;
    }
    __syncthreads();
    if (STAGE) {
      const EvS ev{sm.ev_t, sm.ev_u, wg ? sm.ev_w : nullptr};
      fit_window<M, SPL, BM, LEARN>(a, b, N, T, ev, sm);
    } else if (a.ring) {
      const EvRing ev{tg, ug, nullptr, a.t, a.id, o0, a.n_total, sm.rt, sm.ru, sm.rbar, sm.rfill,
                      sm.ctl + 4, a.wait_polls};
      fit_window<M, SPL, BM, LEARN>(a, b, N, T, ev, sm);
    } else {
      const EvG ev{tg, ug, wg};
      fit_window<M, SPL, BM, LEARN>(a, b, N, T, ev, sm);
    }
  }
}

// d lnL / d w_k by the reverse-time recursion P_j(t) = sum_{n: t_n > t}
// r_n alpha_{u_n j} exp(-beta_j (t_n - t)):  g_k = P_{u_k}(t_k) -
// (sum_i alpha_{i u_k}) (1 - exp(-beta_{u_k} (T - t_k))) / beta_{u_k}.
// One thread per chunk (all M sources in registers), same chunking and tie
// rule as the forward pass, reverse scan over chunks.
template <int M, int BM>
__global__ void __launch_bounds__(256) k_weight_grad(WgArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int AP = M + 1;
  const int b = blockIdx.x;
  if (a.status && a.status[b] != kOK) return;
  const int NC = a.NC, Mrt = a.Mrt, tid = threadIdx.x;
  float *alpha = (float *)smem;
  float *bl2 = alpha + M * AP;
  float *betas = bl2 + M;
  float *col = betas + M;
  float *anc = col + M;
  int *bnd = (int *)(anc + NC + 1);
  float *enc = (float *)(bnd + NC + 1);
  const int64_t o0 = a.offsets[b];
  const int N = (int)(a.offsets[b + 1] - o0);
  const float T = a.T[b];
  const float *t = a.t + o0;
  const int16_t *u = a.id + o0;
  const float *r = a.r + o0;
  const int nb = BM == 0 ? 1 : Mrt;
  for (int p = tid; p < M * AP; p += blockDim.x) {
    const int i = p / AP, j = p % AP;
    alpha[p] = (i < Mrt && j < Mrt) ? a.alpha[(int64_t)b * Mrt * Mrt + i * Mrt + j] : 0.f;
  }
  for (int j = tid; j < M; j += blockDim.x) {
    const float bv = j < nb ? a.beta[(int64_t)b * nb + j] : 1.f;
    betas[j] = BM == 0 ? a.beta[b] : bv;
    bl2[j] = betas[j] * kLog2e;
  }
  __syncthreads();
  for (int j = tid; j < M; j += blockDim.x) {
    float s = 0.f;
    for (int i = 0; i < M; ++i) s += alpha[i * AP + j];
    col[j] = s;
  }
  setup_chunks(NC, N, T, EvG{t, u, nullptr}, bnd, anc);
  const int c = tid;
  float P[M];
  float b2[M];
#pragma unroll
  for (int j = 0; j < M; ++j) b2[j] = bl2[j];
  // reverse pass 1: effect of chunk c at its own anchor, from a zero state at a_{c+1}
  if (c < NC) {
    const int b0 = bnd[c], b1 = bnd[c + 1];
#pragma unroll
    for (int j = 0; j < M; ++j) P[j] = 0.f;
    float tcur = anc[c + 1];
    int n = b1 - 1;
    while (n >= b0) {
      const float tgp = t[n];
      int gs = n;
      while (gs > b0 && t[gs - 1] == tgp) --gs;
      const float dt = tcur - tgp;
      if (dt > 0.f) {
#pragma unroll
        for (int j = 0; j < M; ++j) P[j] *= exp2_acc(-b2[j] * dt);
      }
      tcur = tgp;
      for (int k = gs; k <= n; ++k) {
        const float rk = r[k];
        const float *arow = alpha + (int)u[k] * AP;
#pragma unroll
        for (int j = 0; j < M; ++j) P[j] = fmaf(rk, arow[j], P[j]);
      }
      n = gs - 1;
    }
    const float dt = tcur - anc[c];
    if (dt > 0.f) {
#pragma unroll
      for (int j = 0; j < M; ++j) P[j] *= exp2_acc(-b2[j] * dt);
    }
#pragma unroll
    for (int j = 0; j < M; ++j) enc[c * M + j] = P[j];
  }
  __syncthreads();
  // reverse scan: enc[c] <- state at a_{c+1} carrying every later event
  if (tid < M) {
    const int j = tid;
    float E = 0.f;
    for (int cc = NC - 1; cc >= 0; --cc) {
      const float loc = enc[cc * M + j];
      enc[cc * M + j] = E;
      const float D = anc[cc + 1] - anc[cc];
      E = fmaf(exp2_acc(-bl2[j] * D), E, loc);
    }
  }
  __syncthreads();
  // reverse pass 2
  if (c < NC) {
    const int b0 = bnd[c], b1 = bnd[c + 1];
#pragma unroll
    for (int j = 0; j < M; ++j) P[j] = enc[c * M + j];
    float tcur = anc[c + 1];
    int n = b1 - 1;
    while (n >= b0) {
      const float tgp = t[n];
      int gs = n;
      while (gs > b0 && t[gs - 1] == tgp) --gs;
      const float dt = tcur - tgp;
      if (dt > 0.f) {
#pragma unroll
        for (int j = 0; j < M; ++j) P[j] *= exp2_acc(-b2[j] * dt);
      }
      tcur = tgp;
      for (int k = gs; k <= n; ++k) {
        const int uk = (int)u[k];
        float pv = 0.f;
#pragma unroll
        for (int j = 0; j < M; ++j) pv = (j == uk) ? P[j] : pv;
        const float bj = betas[uk];
        const float comp = col[uk] * (-expm1f(-bj * (T - tgp))) / bj;
        a.g_w[o0 + k] = pv - comp;
      }
      for (int k = gs; k <= n; ++k) {
        const float rk = r[k];
        const float *arow = alpha + (int)u[k] * AP;
#pragma unroll
        for (int j = 0; j < M; ++j) P[j] = fmaf(rk, arow[j], P[j]);
      }
      n = gs - 1;
    }
  }
}

}  // namespace mdhp
