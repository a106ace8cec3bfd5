// Decoupled fixed-beta fit.
//
// With beta fixed, every state R_j(t_n) = sum_{k in j, t_k < t_n} w_k
// exp(-beta_j (t_n - t_k)) is independent of the parameters being fitted
// (mu, alpha): the paper's "decoupling" of Stage 1 (Sec. IV-B.3), which
// hoists everything parameter-free out of the descent loop.  This kernel
// computes the features x_n = R(t_n) once per window by the chunked recursion
// (pass 1 + scan + one feature walk), stores them grouped by event type
// (a stable counting sort: type-major, time order within a type), and then
// runs every iteration as a dense pass over the features:
//   lambda_n = mu_i + alpha_i . x_n,  r_n = 1 / lambda_n,
//   d/dalpha_i += r_n x_n,  d/dmu_i += r_n,  Part1 += ln lambda_n  (i = type of n)
// Each thread owns a contiguous range of the sorted features, so the row
// alpha_i and the sums d/dalpha_i stay in registers with static indices; a
// thread's partial sums of type i go to segment slot (thread + i), which is
// unique (ranges and types are both ordered), and the slots of a type are
// contiguous, so the block reduction needs no atomics.  Features live in
// shared memory (XS) or in a per-CTA global scratch slot read through L1/L2.
// Part2 + Part3 use the compensator constants of the state at T_span.
#pragma once

#include "mdhp_async.cuh"
#include "mdhp_solver.cuh"
#include "mdhp_tmem.cuh"

namespace mdhp {

// Feature layout.  Thread t owns sorted positions [t L, t L + L) and reads
// them in order, step k = pos - t L.  In shared memory the slices are planes
// [q][pos] (the lanes' positions are an odd stride L apart: distinct bank
// groups).  In global memory they are stored step-major, [k][q][t]: at each
// step a warp's 32 lanes read 512 contiguous bytes per float4 slice (4 cache
// lines), where a position-major layout would touch 32 lines per load.
struct XMap {
  int L, NT;
};
template <bool XS>
__device__ __forceinline__ int xidx(int q, int pos, int xcap, int NQ, XMap m) {
  if (XS) return q * xcap + pos;
  const int t = pos / m.L, k = pos - t * m.L;
  return (k * NQ + q) * m.NT + t;
}

// Counting sort of the window's events by type and the feature walk.
// Needs bnd/anc (NT chunks), encR (entering states), cnt (events per type).
// Writes X[q * xcap + pos] (float4 slices of x_n) and tstart[0..M].
template <int M, int BM, bool XS, typename EV, typename XP>
__device__ void build_features(int N, const EV &ev, int Mrt, Sm<M> &sm, XP X, int xcap, XMap m) {
  constexpr int AP = M + 4;
  constexpr int NQ = M / 4;
  const int tid = threadIdx.x, NT = blockDim.x, NC = NT;
  int *ctr = reinterpret_cast<int *>(sm.P);  // [type][chunk]
  for (int p = tid; p < M * NC; p += NT) ctr[p] = 0;
  if (tid == 0) {
    int acc = 0;
    for (int i = 0; i < M; ++i) {
      sm.tstart[i] = acc;
      acc += (i < Mrt) ? sm.cnt[i] : 0;
    }
    sm.tstart[M] = acc;
  }
  __syncthreads();
  const int c = tid;
  const int b0 = sm.bnd[c], b1 = sm.bnd[c + 1];
#pragma unroll 4
  for (int n = b0; n < b1; ++n) ctr[ev.id(n) * NC + c] += 1;
  __syncthreads();
  {  // exclusive scan over chunks, per type, from the type's start: one warp
     // per type, each lane a run of G chunks (G odd: the lanes' reads and
     // writes fall in distinct banks), the runs' totals scanned by shuffles
    const int lane = tid & 31, nw = NT >> 5;
    const int G = ((NC + 31) >> 5) | 1;
    const int c0 = min(lane * G, NC), c1 = min(c0 + G, NC);
    for (int i = tid >> 5; i < M; i += nw) {
      int *row = ctr + i * NC;
      int sum = 0;
      for (int cc = c0; cc < c1; ++cc) sum += row[cc];
      int incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      int run = sm.tstart[i] + incl - sum;
      for (int cc = c0; cc < c1; ++cc) {
        const int v = row[cc];
        row[cc] = run;
        run += v;
      }
    }
  }
  __syncthreads();
  // walk the chunk in time order from its entering state; x_n = state at t_n
  Walker<M, BM, false> wk;
  wk.template load_beta<1>(sm.bl2, 0);  // one thread holds every source: slot j = source j
#pragma unroll
  for (int j = 0; j < M; ++j) wk.R[j] = sm.encR[c * M + j];
  float tprev = sm.anc[c];
  int gs = b0;
  float tnx = 0.f;  // the next event, loaded one step ahead
  int unx = 0;
  if (b0 < b1) ev.get(b0, tnx, unx);
  for (int n = b0; n < b1; ++n) {
    const float tn = tnx;
    const int un = unx;
    if (n + 1 < b1) ev.get(n + 1, tnx, unx);
    if (tn > tprev) {
      for (int k = gs; k < n; ++k) wk.add(ev.id(k), ev.wt(k));
      wk.decay(tn - tprev);
      tprev = tn;
      gs = n;
    }
    const int pos = ctr[un * NC + c];
    ctr[un * NC + c] = pos + 1;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      X[xidx<XS>(q, pos, xcap, NQ, m)] =
          make_float4(wk.R[4 * q], wk.R[4 * q + 1], wk.R[4 * q + 2], wk.R[4 * q + 3]);
  }
  __syncthreads();
}

// Features for a fixed MATRIX beta (beta_ij per pair).  The row of an event n
// of type i is R_i.(t_n), R_ij(t) = sum_{k: t_k < t, u_k = j} w_k exp(-beta_ij
// (t - t_k)), so the iteration pass is the same as for the other beta shapes.
// One thread per (target row i, chunk c), NCm = NT / M chunks.  A row is kept
// lazily as S_j at an anchor time ta, R_ij(t) = 2^(-b_ij (t - ta)) S_j with
// b_ij = beta_ij log2(e): an event k of type j adds w_k 2^(+b_ij (t_k - ta))
// to S_j (one exponential per event and row); at an event of type i the row is
// materialised (M exponentials), written as that event's features and
// re-anchored there; if the positive exponent would pass 64 the row is
// re-anchored early.  Pass 1 gives each (i, c) its chunk's end state from
// zero, a per-pair scan over chunks the entering states and R_ij(T), hence
// C_ij = (W_j - R_ij(T)) / beta_ij; pass 2 writes the features at their
// type-sorted positions.  About 3M exponentials per event over all rows.
// S lives in shared memory ([j][thread], in P after the per-type counters).
template <int M, bool XS, typename EV, typename XP>
__device__ void build_features_matrix(int N, float T, const EV &ev, int Mrt, Sm<M> &sm, XP X,
                                      int xcap, XMap m) {
  constexpr int NQ = M / 4;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int NCm = NT / M;
  const int i = tid % M, c = tid / M;
  const bool act = c < NCm && i < Mrt;
  setup_chunks(NCm, N, T, ev, sm.bnd, sm.anc);  // ends with a barrier
  int *ctr = reinterpret_cast<int *>(sm.P);      // [type][chunk] counts, then positions
  float *S = sm.P + NT;                          // [j][thread]
  const float *bl = sm.bl2 + i * M;
  const int b0 = act ? sm.bnd[c] : 0, b1 = act ? sm.bnd[c + 1] : 0;
  const float a0 = act ? sm.anc[c] : 0.f, a1 = act ? sm.anc[c + 1] : 0.f;
  float bmax = 0.f;
  for (int j = 0; j < Mrt; ++j) bmax = fmaxf(bmax, bl[j]);
  if (act) {
    int cnt = 0;
    for (int n = b0; n < b1; ++n) cnt += ev.id(n) == i ? 1 : 0;
    ctr[i * NCm + c] = cnt;
  }
  if (tid == 0) {
    int acc = 0;
    for (int k = 0; k < M; ++k) {
      sm.tstart[k] = acc;
      acc += (k < Mrt) ? sm.cnt[k] : 0;
    }
    sm.tstart[M] = acc;
  }
  __syncthreads();
  if (tid < Mrt) {  // exclusive scan over chunks, per type, from the type's start
    int run = sm.tstart[tid];
    for (int cc = 0; cc < NCm; ++cc) {
      const int v = ctr[tid * NCm + cc];
      ctr[tid * NCm + cc] = run;
      run += v;
    }
  }
  // the lazy row walk; WRITE: materialise and write at the events of type i
  auto walk = [&](bool write) {
    float ta = a0, tprev = a0;
    int gs = b0;
    auto add = [&](int k) {
      const float tk = ev.time(k);
      float d = tk - ta;
      if (bmax * d > 64.f) {  // re-anchor at tk before the exponent grows too large
        for (int j = 0; j < M; ++j) S[j * NT + tid] *= exp2_acc(-bl[j] * d);
        ta = tk;
        d = 0.f;
      }
      const int u = ev.id(k);
      S[u * NT + tid] += ev.wt(k) * exp2_acc(bl[u] * d);
    };
    for (int n = b0; n < b1; ++n) {
      const float tn = ev.time(n);
      if (tn > tprev) {  // the previous tie group becomes history
        for (int k = gs; k < n; ++k) add(k);
        tprev = tn;
        gs = n;
      }
      if (write && ev.id(n) == i) {
        const float d = tn - ta;
        float x[M];
#pragma unroll
        for (int j = 0; j < M; ++j) {
          x[j] = S[j * NT + tid] * exp2_acc(-bl[j] * d);
          S[j * NT + tid] = x[j];
        }
        ta = tn;
        const int pos = ctr[i * NCm + c];
        ctr[i * NCm + c] = pos + 1;
#pragma unroll
        for (int q = 0; q < NQ; ++q)
          X[xidx<XS>(q, pos, xcap, NQ, m)] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
      }
    }
    for (int k = gs; k < b1; ++k) add(k);
    return ta;
  };
  // pass 1: each chunk's own contribution to the state at its end
  if (act) {
    for (int j = 0; j < M; ++j) S[j * NT + tid] = 0.f;
    const float ta = walk(false);
    for (int j = 0; j < M; ++j) sm.encR[(c * M + i) * M + j] = S[j * NT + tid] * exp2_acc(-bl[j] * (a1 - ta));
  }
  __syncthreads();
  // per-pair scan: entering states, R_ij(T), C_ij
  for (int p = tid; p < M * M; p += NT) {
    const int ii = p / M, jj = p % M;
    if (ii < Mrt && jj < Mrt) {
      float R = 0.f;
      for (int cc = 0; cc < NCm; ++cc) {
        const float v = sm.encR[(cc * M + ii) * M + jj];
        sm.encR[(cc * M + ii) * M + jj] = R;
        R = fmaf(exp2_acc(-sm.bl2[p] * (sm.anc[cc + 1] - sm.anc[cc])), R, v);
      }
      const float2 w = reinterpret_cast<const float2 *>(sm.W)[jj];
      const FF Cp = ff_div(ff_add(FF{w.x, w.y}, FF{-R, 0.f}), sm.beta[p]);
      sm.C[p] = Cp.hi + Cp.lo;
    } else {
      sm.C[p] = 0.f;
    }
  }
  __syncthreads();
  // pass 2: the features, from each chunk's entering state
  if (act) {
    for (int j = 0; j < M; ++j) S[j * NT + tid] = sm.encR[(c * M + i) * M + j];
    walk(true);
  }
  __syncthreads();
}

// Per-thread state of one evaluation over the sorted features: the current
// type i (its row alpha_i and mu_i in registers), the running sums of its
// gradient, and the segment flush when the thread's range crosses into the
// next type.  Segment sums go to P[(tid + i) * (M + 4) + 0..M].
template <int M>
struct XAcc {
  static constexpr int NQ = M / 4;
  static constexpr int AP = M + 4;
  static constexpr int PP = M + 4;
  int i, te;
  float mu, gm;
  float4 ar[NQ], g[NQ];

  __device__ __forceinline__ void begin(int i0, const Sm<M> &sm) {
    i = i0;
    te = sm.tstart[i + 1];
    mu = sm.mu[i];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      ar[q] = reinterpret_cast<const float4 *>(sm.alpha + i * AP)[q];
      g[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    gm = 0.f;
  }
  __device__ __forceinline__ void flush(const Sm<M> &sm) {
    float4 *slot = reinterpret_cast<float4 *>(sm.P + (threadIdx.x + i) * PP);
#pragma unroll
    for (int q = 0; q < NQ; ++q) slot[q] = g[q];
    sm.P[(threadIdx.x + i) * PP + M] = gm;
  }
  // the event at sorted position p with features x
  __device__ __forceinline__ float event(int p, const float4 (&x)[NQ], const Sm<M> &sm) {
    while (p >= te) {  // leave type i (types with no events are passed over)
      flush(sm);
#pragma unroll
      for (int q = 0; q < NQ; ++q) g[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      gm = 0.f;
      ++i;
      te = sm.tstart[i + 1];
      mu = sm.mu[i];
#pragma unroll
      for (int q = 0; q < NQ; ++q) ar[q] = reinterpret_cast<const float4 *>(sm.alpha + i * AP)[q];
    }
    float d0 = mu, d1 = 0.f;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      d0 = fmaf(ar[q].x, x[q].x, d0);
      d1 = fmaf(ar[q].y, x[q].y, d1);
      d0 = fmaf(ar[q].z, x[q].z, d0);
      d1 = fmaf(ar[q].w, x[q].w, d1);
    }
    const float lam = d0 + d1;
    const float r = rcp_ftz(lam);
    const float lg = lg2_ftz(lam);
    gm += r;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      g[q].x = fmaf(r, x[q].x, g[q].x);
      g[q].y = fmaf(r, x[q].y, g[q].y);
      g[q].z = fmaf(r, x[q].z, g[q].z);
      g[q].w = fmaf(r, x[q].w, g[q].w);
    }
    return lg;
  }
};

// One evaluation over the sorted features: this thread's range [p0, p1),
// starting in type i0, features read directly (shared memory, or global
// memory one step ahead in registers).  Two events per trip with two
// register buffers (no copies between them); with the block size a
// compile-time constant (NTC > 0) every global load is base + constant.
// The two events' log-intensities are added before the compensated sum.
template <int M, bool XS, int NTC, typename XP>
__device__ __forceinline__ void xpass(int p0, int p1, int i0, XP X, int xcap, XMap m,
                                      const Sm<M> &sm, float &Ls, float &Lc) {
  constexpr int NQ = M / 4;
  if (p0 >= p1) return;
  XAcc<M> acc;
  acc.begin(i0, sm);
  // slice q of position p: shared X[q * xcap + p]; global (step-major, this
  // thread's column) X[((p - p0) * NQ + q) * NT + tid]
  const int NT = NTC > 0 ? NTC : m.NT;
  const int qs = XS ? xcap : NT;
  const int ps = XS ? 1 : NQ * NT;
  const float4 *px = XS ? X + p0 : X + threadIdx.x;
  float4 xa[NQ], xb[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) xa[q] = px[q * qs];
  int p = p0;
  for (;;) {
    const bool hb = p + 1 < p1;
    if (hb) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) xb[q] = px[ps + q * qs];
    }
    const float la = acc.event(p, xa, sm);
    if (!hb) {
      kahan_add(Ls, Lc, la);
      break;
    }
    const bool ha = p + 2 < p1;
    if (ha) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) xa[q] = px[2 * ps + q * qs];
    }
    kahan_add(Ls, Lc, la + acc.event(p + 1, xb, sm));
    if (!ha) break;
    p += 2;
    px += 2 * ps;
  }
  acc.flush(sm);
}

// Streamed features through a ring of shared-memory buffers filled by bulk
// copies.  In the step-major global layout, step k of every thread is one
// contiguous block of NQ * NT float4, so S consecutive steps are one copy.
// The copies form an endless cyclic sequence over the window's stages (the
// features do not change between iterations), so the ring runs ahead across
// iteration boundaries; fill g holds stage (g - base) mod nst and lands in
// buffer g mod D, whose mbarrier completes for the (g / D)-th time.
struct XPipe {
  const float4 *src;  // the CTA's global feature slot
  int step_f4;        // float4 per step (NQ * NT)
  int L, S, D, nst;   // steps per pass, steps per stage, buffers, stages per pass
  uint32_t used, issued, base;  // fills consumed (all threads) / issued (thread 0)
  uint32_t polls;     // bound of a consumer's wait (0: the default)
};

template <int M>
__device__ __forceinline__ void xpipe_issue(XPipe &pp, const Sm<M> &sm) {
  const uint32_t g = pp.issued++;
  const int c = (int)((g - pp.base) % (uint32_t)pp.nst);
  const int slot = (int)(g % (uint32_t)pp.D);
  const int k0 = c * pp.S;
  const int ns = min(pp.S, pp.L - k0);
  const uint32_t bytes = (uint32_t)ns * (uint32_t)pp.step_f4 * 16u;
  uint64_t *bar = sm.mbar + slot;
  mbar_expect_tx(bar, bytes);
  bulk_copy_g2s(sm.ring + (size_t)slot * pp.S * pp.step_f4, pp.src + (size_t)k0 * pp.step_f4,
                bytes, bar);
}

// One evaluation through the ring.  Every thread walks all stages (threads
// without positions only keep step); a barrier closes each stage, after which
// thread 0 refills its buffer D fills ahead.  Returns false (uniformly) if a
// fill did not arrive within the wait bound.
template <int M>
__device__ __forceinline__ bool xpass_pipe(int p0, int p1, int i0, XPipe &pp, const Sm<M> &sm,
                                           float &Ls, float &Lc) {
  constexpr int NQ = M / 4;
  const int tid = threadIdx.x, NT = blockDim.x;
  const bool active = p0 < p1;
  XAcc<M> acc;
  if (active) acc.begin(i0, sm);
  float pend = 0.f;  // log2 of the first event of a pair, summed as in xpass
  for (int s = 0; s < pp.nst; ++s) {
    const uint32_t g = pp.used;
    const int slot = (int)(g % (uint32_t)pp.D);
    if (!mbar_wait_for(sm.mbar + slot, (g / (uint32_t)pp.D) & 1u, pp.polls)) sm.ctl[3] = 1;
    const float4 *buf = sm.ring + (size_t)slot * pp.S * pp.step_f4 + tid;
    const int k0 = s * pp.S, k1 = min(k0 + pp.S, pp.L);
    if (active) {
      for (int k = k0; k < k1; ++k) {
        const int p = p0 + k;
        if (p >= p1) break;
        float4 x[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) x[q] = buf[(k - k0) * pp.step_f4 + q * NT];
        const float lg = acc.event(p, x, sm);
        if ((k & 1) == 0) pend = lg;
        else kahan_add(Ls, Lc, pend + lg);
      }
    }
    __syncthreads();
    if (sm.ctl[3]) return false;  // fill g is still owed: the drain waits from it on
    ++pp.used;
    if (tid == 0) xpipe_issue<M>(pp, sm);
  }
  if (active) {
    if ((p1 - p0) & 1) kahan_add(Ls, Lc, pend);  // the unpaired last event
    acc.flush(sm);
  }
  return true;
}

// Waits out the D fills issued and not yet consumed, pp.used .. pp.used + D - 1
// (each with the full bound, whatever the consumers' bound): after the last
// stage of a window, or after a stage whose fill did not arrive in time (that
// fill included).  Returns (uniformly) whether every one of them landed; if
// not, a copy may still be writing into the ring, which is then not used again.
template <int M>
__device__ __forceinline__ bool xpipe_drain(XPipe &pp, const Sm<M> &sm) {
  bool ok = true;
  for (int d = 0; d < pp.D; ++d) {
    const uint32_t g = pp.used++;
    ok &= mbar_wait(sm.mbar + (g % (uint32_t)pp.D), (g / (uint32_t)pp.D) & 1u);
  }
  return __syncthreads_and(ok) != 0;
}

// Event part of the gradient of parameter p (mu_i or alpha_ij): the sum of
// the segment slots of type i.
// tf[i] holds the float offset of type i's first slot, (first thread + i) *
// (M + 4), and tl[i] the number of its slots (0: no events of type i).
template <int M>
__device__ __forceinline__ float xseg_sum(int i, int j, const Sm<M> &sm) {
  constexpr int PP = M + 4;
  const float *ps = sm.P + sm.tf[i] + j;
  const int cnt = sm.tl[i];
  float acc = 0.f;
#pragma unroll 4
  for (int s = 0; s < cnt; ++s) acc += ps[s * PP];  // in slot order; the loads of 4 slots overlap
  return acc;
}

enum : int { XM_GLOBAL = 0, XM_SHARED = 1, XM_RING = 2, XM_TMEM = 3 };

// One evaluation with the features of every thread in three tiers: steps
// [0, Kt) in tensor memory (row tb of this thread's lane, M columns per
// step), steps [Kt, Kt + Ks) in shared memory (XSt, step-major like the
// global scratch), the rest read from the global scratch as in xpass.  The
// tensor-memory loads are warp-collective, so every thread walks all Kt
// steps (Kt is the same for the whole CTA) and only the threads whose range
// covers a step use it.  The log-intensities are added to the compensated
// sum in pairs, as in xpass.
template <int M, int NTC>
__device__ __forceinline__ void xpass_t(int p0, int p1, int i0, const float4 *X, const float4 *XSt,
                                        XMap m, uint32_t tb, int Kt, int Ks, const Sm<M> &sm,
                                        float &Ls, float &Lc) {
  constexpr int NQ = M / 4;
  const bool active = p0 < p1;
  const int NT = NTC > 0 ? NTC : m.NT;
  XAcc<M> acc;
  if (active) acc.begin(i0, sm);
  float pend = 0.f;
  // tensor memory: one load and its wait per step (measured faster than
  // keeping the next step's load in flight, which needs 32 more registers)
  for (int k = 0; k < Kt; ++k) {
    float4 x[NQ];
    __syncwarp();
    tm_ld<NQ>(tb + (uint32_t)(k * M), x);
    if (p0 + k < p1) {
      const float lg = acc.event(p0 + k, x, sm);
      if (k & 1) kahan_add(Ls, Lc, pend + lg);
      else pend = lg;
    }
  }
  int cnt = active ? min(Kt, p1 - p0) : 0;  // events added so far (odd: pend is pending)
  const int ps = NQ * NT;
  for (int k = Kt; k < Kt + Ks && p0 + k < p1; ++k) {  // shared-memory tier
    float4 x[NQ];
    const float4 *px = XSt + (size_t)(k - Kt) * ps + threadIdx.x;
#pragma unroll
    for (int q = 0; q < NQ; ++q) x[q] = px[q * NT];
    const float lg = acc.event(p0 + k, x, sm);
    if (cnt & 1) kahan_add(Ls, Lc, pend + lg);
    else pend = lg;
    ++cnt;
  }
  if (cnt & 1) kahan_add(Ls, Lc, pend);
  int p = p0 + Kt + Ks;
  if (p < p1) {  // the steps past both tiers: global, one step ahead
    const float4 *px = X + threadIdx.x + (size_t)(Kt + Ks) * ps;
    float4 xa[NQ], xb[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) xa[q] = px[q * NT];
    for (;;) {
      const bool hb = p + 1 < p1;
      if (hb) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) xb[q] = px[ps + q * NT];
      }
      const float la = acc.event(p, xa, sm);
      if (!hb) {
        kahan_add(Ls, Lc, la);
        break;
      }
      const bool ha = p + 2 < p1;
      if (ha) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) xa[q] = px[2 * ps + q * NT];
      }
      kahan_add(Ls, Lc, la + acc.event(p + 1, xb, sm));
      if (!ha) break;
      p += 2;
      px += 2 * ps;
    }
  }
  if (active) acc.flush(sm);
}

// Residency: the streamed M = 32 fit is bound by how many warps per SM keep
// feature loads and their dependent FMA chains in flight, so the 128-thread
// build is held to 168 registers for three CTAs per SM (12 warps; shared
// memory allows three): 355 ms against 373 ms at two CTAs for the 65,536-
// window fit to 1e-5.  The 256-thread build keeps its registers (two CTAs
// would leave 128 and spill 428 bytes).
template <int M, int NTC, int XM>
struct XBounds {
  static constexpr bool three = NTC == 128 && M >= 32 && XM != XM_TMEM;
  static constexpr int threads = NTC > 256 ? NTC : (three ? 128 : 256);
  static constexpr int ctas = NTC > 256 ? 1 : (three ? 3 : (M >= 32 ? 1 : 2));
};

template <int M, int BM, int XM, int NTC>
__global__ void __launch_bounds__(XBounds<M, NTC, XM>::threads, XBounds<M, NTC, XM>::ctas) k_fit_x(FitArgs a) {
  constexpr bool XS = XM == XM_SHARED;
  constexpr bool XT = XM == XM_TMEM;
  extern __shared__ __align__(16) unsigned char smem[];
  Sm<M> sm;
  sm.bind(smem, a.carve);
  constexpr int AP = M + 4;
  const int Mrt = a.Mrt;
  const int nb = BM == 0 ? 1 : (BM == 1 ? Mrt : Mrt * Mrt);
  const int np = Mrt + Mrt * Mrt + nb;
  const int nupd = Mrt + Mrt * Mrt;
  const int tid = threadIdx.x, NT = NTC > 0 ? NTC : (int)blockDim.x;
  const int xcap = a.ev_cap;
  // global slot: (xcap + 768) rows, enough for L * NT with the odd rounding of
  // L for every block size up to 384 (one stride for all launches of a plan)
  float4 *Xg = XS ? nullptr
                  : a.xbuf + (size_t)(a.slot_base + blockIdx.x) * (M / 4) * (size_t)(xcap + 768);
  constexpr bool pipe = XM == XM_RING;
  XPipe pp{Xg, (M / 4) * NT, 1, a.pipe_steps, a.pipe_stages, 1, 0u, 0u, 0u, a.wait_polls};
  bool ring_lost = false;  // a drain gave up: fills may still be landing in the ring
  if (pipe) {
    if (tid == 0) {
      for (int d = 0; d < pp.D; ++d) mbar_init(sm.mbar + d, 1);
      mbar_init_fence();
    }
    __syncthreads();
  }
  // tensor-memory feature rows: a.tmem_cols columns for this CTA (the host
  // sizes them so that every CTA resident on an SM gets its share of 512);
  // lane = tid mod 128, and threads sharing a lane split its columns
  uint32_t tb = 0;
  int tsteps = 0;
  // shared-memory tier of the same mode: a.smem_steps steps per thread after
  // the carve, [step][slice][thread]
  float4 *xst = XT ? reinterpret_cast<float4 *>(smem + a.carve.total) : nullptr;
  if constexpr (XT) {
    if (tid < 32) {
      tm_alloc((uint32_t)__cvta_generic_to_shared(sm.ctl + 8), (uint32_t)a.tmem_cols);
      tm_relinquish();
    }
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const int share = NT > 128 ? a.tmem_cols / (NT / 128) / M * M : a.tmem_cols;
    tb = (uint32_t)sm.ctl[8] + ((uint32_t)(32 * ((tid >> 5) & 3)) << 16) + (uint32_t)((tid >> 7) * share);
    tsteps = share / M;
  }
  for (;;) {
    if (tid == 0) {
      const int qb = a.range ? a.range[0] : a.qbegin;
      const int qe = a.range ? a.range[1] : a.qend;
      int pos = -1;
      if (a.qdir == 0) {
        const int q = atomicAdd(a.queue, 1);
        pos = qb + q < qe ? qb + q : -1;
      } else if (atomicAdd(a.dq, 1) < qe - qb) {  // a window is left: take it from this end
        pos = a.qdir == 1 ? qb + atomicAdd(a.dq + 1, 1) : qe - 1 - atomicAdd(a.dq + 2, 1);
      }
      sm.ctl[1] = pos;
    }
    __syncthreads();
    const int pos = sm.ctl[1];
    __syncthreads();
    if (pos < 0) break;
    const int b = a.order ? a.order[pos] : pos;
    const int64_t o0 = a.offsets[b];
    const int N = (int)(a.offsets[b + 1] - o0);
    const float T = a.T[b];
    const float *tg = a.t + o0;
    const int16_t *ug = a.id + o0;
    const float *wg = a.w ? a.w + o0 : nullptr;
    int st = (pipe && ring_lost) ? (int)kE_TIMEOUT
             : (N > xcap)        ? (int)kE_ARG
                                 : stage_and_validate<M, false>(tg, ug, wg, N, T, Mrt, sm);
    if (st != kOK) {
      if (tid == 0) {
        a.status[b] = st;
        a.loglik[b] = __longlong_as_double(0x7ff8000000000000LL);
        a.iters[b] = 0;
      }
      __syncthreads();
      continue;
    }
    load_params<M, BM>(b, Mrt, a.mu, a.alpha, a.beta, sm);
    __syncthreads();
    if (a.init == 1) {
      for (int p = tid; p < Mrt * Mrt; p += NT) {
        const int i = p / Mrt, j = p % Mrt;
        sm.alpha[i * AP + j] = 0.5f * sm.beta[BM == 0 ? 0 : (BM == 1 ? j : i * M + j)] / (float)Mrt;
      }
      for (int i = tid; i < Mrt; i += NT) sm.mu[i] = 0.5f * (float)max(sm.cnt[i], 1) / T;
    }
    if (a.optimizer == 1) {
      for (int p = tid; p < np; p += NT) {
        sm.am[p] = 0.f;
        sm.av[p] = 0.f;
      }
    }
    const EvG ev{tg, ug, wg};
    setup_chunks(NT, N, T, ev, sm.bnd, sm.anc);
    if constexpr (BM != 2) prepare_states<M, 1, BM, false>(NT, ev, Mrt, sm);
    // thread ranges over the sorted features; an odd length keeps the
    // lanes' shared-memory float4 reads on distinct bank groups
    int L = (N + NT - 1) / NT;
    L = max(L | 1, 1);
    const XMap xm{L, NT};
    if constexpr (BM == 2) {
      if (XS) build_features_matrix<M, true>(N, T, ev, Mrt, sm, sm.xs, xcap, xm);
      else build_features_matrix<M, false>(N, T, ev, Mrt, sm, Xg, xcap, xm);
    } else {
      if (XS) build_features<M, BM, true>(N, ev, Mrt, sm, sm.xs, xcap, xm);
      else build_features<M, BM, false>(N, ev, Mrt, sm, Xg, xcap, xm);
    }
    if (pipe) fence_proxy_async_global();  // this thread's feature stores -> the copy engine
    const int Kt = XT ? min(L, tsteps) : 0;
    const int Ks = XT ? min(L - Kt, a.smem_steps) : 0;
    if constexpr (XT) {  // this thread's first Kt + Ks steps: global scratch -> its rows
      __syncwarp();
      for (int k = 0; k < Kt; ++k) {
        float4 x[M / 4];
#pragma unroll
        for (int q = 0; q < M / 4; ++q) x[q] = Xg[(size_t)(k * (M / 4) + q) * NT + tid];
        tm_st<M / 4>(tb + (uint32_t)(k * M), x);
      }
      tm_wait_st();
      for (int k = Kt; k < Kt + Ks; ++k)
#pragma unroll
        for (int q = 0; q < M / 4; ++q)
          xst[(size_t)((k - Kt) * (M / 4) + q) * NT + tid] = Xg[(size_t)(k * (M / 4) + q) * NT + tid];
    }
    const int p0 = min(tid * L, N), p1 = min(p0 + L, N);
    int i0 = 0;
    while (i0 < M - 1 && sm.tstart[i0 + 1] <= p0) ++i0;
    for (int i = tid; i < M; i += NT) {
      const int first = sm.tstart[i] / L;
      const bool has = sm.tstart[i + 1] > sm.tstart[i];
      sm.tf[i] = (first + i) * (M + 4);
      sm.tl[i] = has ? (sm.tstart[i + 1] - 1) / L - first + 1 : 0;
    }
    if (tid == 0) sm.ctl[3] = 0;
    __syncthreads();
    if (pipe) {  // start the ring: the first D fills of this window's cyclic stage sequence
      pp.L = L;
      pp.nst = (L + pp.S - 1) / pp.S;
      pp.base = pp.used;
      if (tid == 0) {
        pp.issued = pp.used;
        for (int d = 0; d < pp.D; ++d) xpipe_issue<M>(pp, sm);
      }
    }
    const float invN = 1.f / (float)max(N, 1);
    FF lnl_prev{0.f, 0.f}, lnl_out{0.f, 0.f};
    const bool use_tol = a.tol > 0.0;
    const float tolf = (float)a.tol;
    int streak = 0, k = 0;
    bool timed_out = false;
    int wst = a.tol > 0.0 ? kE_MAXITER : kOK;
    float b1t = 1.f, b2t = 1.f;
    // Part2 + Part3 of the current point: computed here for theta_0, then
    // accumulated by the update loop while it forms theta_{k+1}
    float Ps = 0.f, Pc = 0.f;
    for (int p = tid; p < M + M * M; p += NT) {  // padded entries hold zeros
      if (p < M) {
        kahan_add(Ps, Pc, -T * sm.mu[p]);
      } else {
        const int qq = p - M, i = qq / M, j = qq % M;
        kahan_add(Ps, Pc, -sm.alpha[i * AP + j] * sm.C[BM == 2 ? i * M + j : j]);
      }
    }
    for (k = 0; k < a.max_iters; ++k) {
      float Ls = 0.f, Lc = 0.f;
      if (XS) {
        xpass<M, true, 0>(p0, p1, i0, (const float4 *)sm.xs, xcap, xm, sm, Ls, Lc);
      } else if constexpr (pipe) {
        if (!xpass_pipe<M>(p0, p1, i0, pp, sm, Ls, Lc)) {  // a fill did not arrive in time
          if (tid == 0) {
            a.status[b] = kE_TIMEOUT;
            a.loglik[b] = __longlong_as_double(0x7ff8000000000000LL);
            a.iters[b] = k;
          }
          // the fills in flight land before the CTA goes on; if they do not,
          // its later windows report the timeout without touching the ring
          if (!xpipe_drain<M>(pp, sm)) ring_lost = true;
          timed_out = true;
          break;
        }
      } else if constexpr (XT) {
        xpass_t<M, NTC>(p0, p1, i0, (const float4 *)Xg, xst, xm, tb, Kt, Ks, sm, Ls, Lc);
      } else {
        xpass<M, false, NTC>(p0, p1, i0, (const float4 *)Xg, xcap, xm, sm, Ls, Lc);
      }
      // block sums of Part1 and Part2 + Part3 (ends with a barrier)
      float h1 = Ls, l1 = -Lc, h2 = Ps, l2 = -Pc;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float x1 = __shfl_xor_sync(0xffffffffu, h1, o), y1 = __shfl_xor_sync(0xffffffffu, l1, o);
        const float x2 = __shfl_xor_sync(0xffffffffu, h2, o), y2 = __shfl_xor_sync(0xffffffffu, l2, o);
        pair_add(h1, l1, x1);
        l1 += y1;
        pair_add(h2, l2, x2);
        l2 += y2;
      }
      if ((tid & 31) == 0) reinterpret_cast<float4 *>(sm.red)[tid >> 5] = make_float4(h1, l1, h2, l2);
      __syncthreads();
      int bad = 0;
      // the convergence decision is taken by lane 0 of the last warp (that
      // warp has the fewest parameters to update when they do not divide
      // evenly), after the warp has added the warps' partial sums as a tree
      const int dec = NT - 32;
      FF val{0.f, 0.f};
      if (tid >= dec) val = lnl_total_ff_warp(sm.red, NT >> 5);
      if (tid == dec) {
        bad = !isfinite(val.hi);
        int decision = 0;
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
      // gradient and tentative update of this thread's parameters (each
      // parameter always belongs to the same thread): gbuf keeps theta_k and
      // prev theta_{k-1}, so a stop returns theta_k and a non-finite
      // evaluation returns the last finite point theta_{k-1}
      b1t *= a.b1;
      b2t *= a.b2;
      // Adam's bias corrections as two reciprocals per iteration; per
      // parameter the step takes the approximate square root and reciprocal
      // (relative error near 2^-22 in the step, which only sets where the next
      // point lies; the likelihood and its gradient are exact as before)
      const float c1 = 1.f / (1.f - b1t), c2 = 1.f / (1.f - b2t);
      Ps = 0.f;
      Pc = 0.f;
      for (int p = tid; p < M + M * M; p += NT) {
        int i, j, pc;
        if (p < M) {
          i = p; j = M; pc = p;
        } else {
          i = (p - M) / M; j = (p - M) % M; pc = Mrt + i * Mrt + j;
        }
        if (i >= Mrt || (j < M && j >= Mrt)) continue;
        const float cj = (j == M) ? T : sm.C[BM == 2 ? i * M + j : j];
        const float g = xseg_sum<M>(i, j, sm) - cj;
        bad |= !isfinite(g);
        float &th = (j == M) ? sm.mu[i] : sm.alpha[i * AP + j];
        const float gs = g * invN;
        float step;
        if (a.optimizer == 1) {
          const float m1 = a.b1 * sm.am[pc] + (1.f - a.b1) * gs;
          const float m2 = a.b2 * sm.av[pc] + (1.f - a.b2) * gs * gs;
          sm.am[pc] = m1;
          sm.av[pc] = m2;
          step = a.lr * (m1 * c1) * rcp_ftz(sqrt_ftz(m2 * c2) + a.eps);
        } else {
          step = a.lr * gs;
        }
        const float fl = (j == M) ? a.mu_floor : a.alpha_floor;
        sm.prev[pc] = sm.gbuf[pc];
        sm.gbuf[pc] = th;
        const float tn = fmaxf(th + step, fl);
        th = tn;
        kahan_add(Ps, Pc, -tn * cj);  // Part2 (-T mu_i) or Part3 (-alpha_ij C_j) of theta_{k+1}
      }
      bad = __syncthreads_or(bad);
      const int stop = bad ? 1 : sm.ctl[2];
      if (stop) {
        const float *src = (bad && k > 0) ? sm.prev : sm.gbuf;
        for (int p = tid; p < nupd; p += NT) param_ref<M>(p, Mrt, sm) = src[p];
        if (bad) wst = kE_NONFINITE;
        else ++k;
        __syncthreads();
        break;
      }
    }
    if (timed_out) continue;  // window reported, ring drained
    if (pipe && !xpipe_drain<M>(pp, sm)) ring_lost = true;  // fills issued for an iteration that never ran
    for (int p = tid; p < Mrt * Mrt; p += NT)
      a.alpha[(int64_t)b * Mrt * Mrt + p] = sm.alpha[(p / Mrt) * AP + (p % Mrt)];
    for (int i = tid; i < Mrt; i += NT) a.mu[(int64_t)b * Mrt + i] = sm.mu[i];
    for (int j = tid; j < nb; j += NT)
      a.beta[(int64_t)b * nb + j] = sm.beta[BM == 2 ? (j / Mrt) * M + (j % Mrt) : j];
    if (tid == NT - 32) {  // the thread that took the decisions
      a.loglik[b] = ff_to_double(lnl_out);
      a.iters[b] = k;
      a.status[b] = wst;
    }
    __syncthreads();
  }
  if constexpr (XT) {  // every thread's tensor-memory accesses are complete
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    if (tid < 32) tm_dealloc((uint32_t)sm.ctl[8], (uint32_t)a.tmem_cols);
  }
}

}  // namespace mdhp
