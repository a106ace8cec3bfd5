// Device side of MDHP-GDS for sm_103a: one CTA owns one window at a time.
//
// Model (arXiv 2411.10258): MDHP intensity of Sec. II and the closed-form
// log-likelihood of Sec. IV-B.1 (Part1 + Part2 + Part3, App. B).  Instead of
// the paper's padded O(D^2 L^2) broadcast (Alg. 1-3) the window is walked in
// time order with the exact recursion
//   R_j(t) = sum_{k: u_k = j, t_k < t} w_k exp(-beta_j (t - t_k))      (decay state of source j)
//   S_j(t) = sum_{k: u_k = j, t_k < t} w_k (t - t_k) exp(-beta_j (t - t_k))   (its beta-derivative)
//   lambda_n = mu_{u_n} + sum_j alpha_{u_n j} R_j(t_n)
// which costs O(N M) per evaluation.  The compensator (Part2 + Part3) comes
// from the state at T_span: C_j = (W_j - R_j(T)) / beta_j, W_j = sum of source
// j's weights, and d C_j / d beta_j = (S_j(T) - C_j) / beta_j.
//
// Parallel decomposition of a window (events are sorted by time):
//   * the CTA's threads form NC = blockDim / SPL chunk groups; chunk c owns the
//     contiguous events [b_c, b_{c+1}), boundaries moved past tie groups so that
//     a timestamp never straddles two chunks;
//   * SPL threads of a chunk split the M sources (MS = M / SPL each), so the
//     per-thread state R[MS] (and S[MS]) lives in registers;
//   * pass 1 computes each chunk's local effect (state at the next chunk's
//     anchor, starting from zero), a per-source scan over chunks composes the
//     affine maps (R, S) -> (A R + R_loc, A (S + D R) + S_loc), A = exp(-beta D),
//     and gives every chunk its entering state; with fixed beta this runs once
//     per window, with learned beta once per evaluation;
//   * pass 2 walks each chunk from its entering state and accumulates ln lambda
//     (Kahan, FP32), d/dmu and d/dalpha (shared-memory atomics) and d/dbeta
//     (registers).
// Ties (Sec. II: the inner sum is strict): the increments of a tie group are
// added only when time advances past it.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mdhp {

constexpr float kLog2e = 1.4426950408889634f;
constexpr double kLn2 = 0.69314718055994530942;

enum : int {
  kOK = 0, kE_ARG = 1, kE_UNSORTED = 2, kE_ID_RANGE = 3, kE_TIME_RANGE = 4,
  kE_NONFINITE = 5, kE_MAXITER = 6
};

__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// First event of chunk c out of NC over [0, N): the even split moved forward
// past any tie group, so every chunk starts at a new timestamp.
template <typename TP>
__device__ __forceinline__ int chunk_begin(int c, int NC, int N, TP t) {
  if (c >= NC) return N;
  int b = (int)(((long long)c * (long long)N) / NC);
  while (b > 0 && b < N && t[b] == t[b - 1]) ++b;
  return b;
}

// ---------------------------------------------------------------------------
// Shared-memory carve of one CTA (sizes depend on M, NC, event capacity).
// ---------------------------------------------------------------------------
struct Carve {
  // byte offsets
  int alpha, ga, mu, gm, beta, bl2, gb, W, cnt, C, dC, endR, endS, anc, bnd, encR, encS, prev,
      gbuf, am, av, red, ctl, ev_t, ev_u, ev_w;
  int total;
};

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

// np_max = M + M*M + M parameters.
__host__ __device__ inline Carve make_carve(int M, int NC, int ev_cap, bool weights, bool learn,
                                            bool adam, bool fit) {
  Carve c;
  int o = 0;
  const int AP = M + 1;
  const int npm = M + M * M + M;
  auto take = [&](int bytes) { int r = o; o = align_up(o + bytes, 16); return r; };
  c.red = take(32 * 8);
  c.ctl = take(16 * 4);
  c.alpha = take(M * AP * 4);
  c.ga = take(M * AP * 4);
  c.mu = take(M * 4);
  c.gm = take(M * 4);
  c.beta = take(M * 4);
  c.bl2 = take(M * 4);
  c.gb = take(M * 4);
  c.W = take(M * 4);
  c.cnt = take(M * 4);
  c.C = take(M * 4);
  c.dC = take(M * 4);
  c.endR = take(M * 4);
  c.endS = take(M * 4);
  c.anc = take((NC + 1) * 4);
  c.bnd = take((NC + 1) * 4);
  c.encR = take(NC * M * 4);
  c.encS = learn ? take(NC * M * 4) : c.encR;
  c.prev = fit ? take(npm * 4) : 0;
  c.gbuf = fit ? take(npm * 4) : 0;
  c.am = (fit && adam) ? take(npm * 4) : 0;
  c.av = (fit && adam) ? take(npm * 4) : 0;
  c.ev_t = ev_cap > 0 ? take(ev_cap * 4) : 0;
  c.ev_w = (ev_cap > 0 && weights) ? take(ev_cap * 4) : 0;
  c.ev_u = ev_cap > 0 ? take(ev_cap * 2) : 0;
  c.total = o;
  return c;
}

// Everything a CTA needs about its current window.
struct WinCtx {
  const float *t;      // events (shared or global)
  const int16_t *u;
  const float *w;      // nullptr => weight 1
  int N;
  float T;
  int Mrt;             // runtime number of types (<= M)
};

template <int M>
struct Sm {
  float *alpha, *ga, *mu, *gm, *beta, *bl2, *gb, *W, *C, *dC, *endR, *endS, *anc, *encR, *encS,
      *prev, *gbuf, *am, *av;
  int *bnd, *cnt, *ctl;
  double *red;
  float *ev_t, *ev_w;
  int16_t *ev_u;
  __device__ void bind(unsigned char *base, const Carve &c) {
    alpha = (float *)(base + c.alpha); ga = (float *)(base + c.ga); mu = (float *)(base + c.mu);
    gm = (float *)(base + c.gm); beta = (float *)(base + c.beta); bl2 = (float *)(base + c.bl2);
    gb = (float *)(base + c.gb); W = (float *)(base + c.W); cnt = (int *)(base + c.cnt);
    C = (float *)(base + c.C); dC = (float *)(base + c.dC); endR = (float *)(base + c.endR);
    endS = (float *)(base + c.endS); anc = (float *)(base + c.anc); bnd = (int *)(base + c.bnd);
    encR = (float *)(base + c.encR); encS = (float *)(base + c.encS);
    prev = (float *)(base + c.prev); gbuf = (float *)(base + c.gbuf); am = (float *)(base + c.am); av = (float *)(base + c.av);
    red = (double *)(base + c.red); ctl = (int *)(base + c.ctl);
    ev_t = (float *)(base + c.ev_t); ev_w = (float *)(base + c.ev_w);
    ev_u = (int16_t *)(base + c.ev_u);
  }
};

// ---------------------------------------------------------------------------
// Block reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum_double(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];  // every thread gets the same order
  return s;
}

// ---------------------------------------------------------------------------
// Per-thread recursion pieces.  MS sources starting at `base`.
// ---------------------------------------------------------------------------
template <int MS, int BM, bool LEARN>
struct Walker {
  float R[MS];
  float S[LEARN ? MS : 1];
  float b2[BM == 0 ? 1 : MS];  // beta * log2(e)

  __device__ __forceinline__ void load_beta(const float *bl2, int base) {
    if (BM == 0) {
      b2[0] = bl2[0];
    } else {
#pragma unroll
      for (int jj = 0; jj < (BM == 0 ? 1 : MS); ++jj) b2[jj] = bl2[base + jj];
    }
  }
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int jj = 0; jj < MS; ++jj) {
      R[jj] = 0.f;
      if (LEARN) S[jj] = 0.f;
    }
  }
  __device__ __forceinline__ void decay(float dt) {
    if (BM == 0) {
      const float a = exp2f(-b2[0] * dt);
#pragma unroll
      for (int jj = 0; jj < MS; ++jj) {
        if (LEARN) S[jj] = a * fmaf(dt, R[jj], S[jj]);
        R[jj] *= a;
      }
    } else {
#pragma unroll
      for (int jj = 0; jj < MS; ++jj) {
        const float a = exp2f(-b2[(BM == 0) ? 0 : jj] * dt);
        if (LEARN) S[jj] = a * fmaf(dt, R[jj], S[jj]);
        R[jj] *= a;
      }
    }
  }
  // add the increments of events [k0, k1) (a finished tie group)
  template <typename TP, typename UP, typename WP>
  __device__ __forceinline__ void add_events(int k0, int k1, TP, UP u, WP w, int base) {
    for (int k = k0; k < k1; ++k) {
      const int uk = (int)u[k] - base;
      const float wk = w ? w[k] : 1.f;
#pragma unroll
      for (int jj = 0; jj < MS; ++jj) R[jj] += (uk == jj) ? wk : 0.f;
    }
  }
};

// Pass 1 for chunk [b0, b1) anchored at a0, ending at a1: local state -> encR/encS[c].
template <int M, int SPL, int BM, bool LEARN, typename TP, typename UP, typename WP>
__device__ __forceinline__ void pass1_chunk(int c, int s, int b0, int b1, float a0, float a1,
                                            TP t, UP u, WP w, const float *bl2, float *encR,
                                            float *encS) {
  constexpr int MS = M / SPL;
  const int base = s * MS;
  Walker<MS, BM, LEARN> wk;
  wk.load_beta(bl2, base);
  wk.zero();
  float tprev = a0;
  int gs = b0;
  for (int n = b0; n < b1; ++n) {
    const float tn = t[n];
    if (tn > tprev) {
      wk.add_events(gs, n, t, u, w, base);
      wk.decay(tn - tprev);
      tprev = tn;
      gs = n;
    }
  }
  wk.add_events(gs, b1, t, u, w, base);
  if (a1 > tprev) wk.decay(a1 - tprev);
#pragma unroll
  for (int jj = 0; jj < MS; ++jj) {
    encR[c * M + base + jj] = wk.R[jj];
    if (LEARN) encS[c * M + base + jj] = wk.S[jj];
  }
}

// Per-source scan over chunks: encR/encS[c] become entering states; end state
// (at T_span, all events included) goes to endR/endS.  Threads j < M.
template <int M, bool LEARN>
__device__ __forceinline__ void scan_chunks(int NC, const float *anc, const float *bl2, int bm,
                                            float *encR, float *encS, float *endR, float *endS) {
  const int j = threadIdx.x;
  if (j >= M) return;
  const float b = bl2[bm == 0 ? 0 : j];
  float R = 0.f, S = 0.f;
  for (int c = 0; c < NC; ++c) {
    const float lr = encR[c * M + j];
    const float ls = LEARN ? encS[c * M + j] : 0.f;
    encR[c * M + j] = R;
    if (LEARN) encS[c * M + j] = S;
    const float D = anc[c + 1] - anc[c];
    const float A = exp2f(-b * D);
    if (LEARN) S = fmaf(A, fmaf(D, R, S), ls);
    R = fmaf(A, R, lr);
  }
  endR[j] = R;
  if (LEARN) endS[j] = S;
}

// Pass 2 for chunk c: lnL (log2 units, Kahan), atomics into gm/ga, beta grads in gbl.
template <int M, int SPL, int BM, bool LEARN, typename TP, typename UP, typename WP>
__device__ __forceinline__ void pass2_chunk(int c, int s, int b0, int b1, float a0, TP t, UP u,
                                            WP w, const float *bl2, const float *encR,
                                            const float *encS, const float *alpha, const float *mu,
                                            float *ga, float *gm, float &Ls, float &Lc,
                                            float (&gbl)[LEARN ? M / SPL : 1], float *r_out) {
  constexpr int MS = M / SPL;
  constexpr int AP = M + 1;
  const int base = s * MS;
  const int lane = threadIdx.x & 31;
  const unsigned gmask = (SPL == 32) ? 0xffffffffu
                                     : (((1u << SPL) - 1u) << (lane & ~(SPL - 1)));
  Walker<MS, BM, LEARN> wk;
  wk.load_beta(bl2, base);
#pragma unroll
  for (int jj = 0; jj < MS; ++jj) {
    wk.R[jj] = encR[c * M + base + jj];
    if (LEARN) wk.S[jj] = encS[c * M + base + jj];
  }
  float tprev = a0;
  int gs = b0;
  for (int n = b0; n < b1; ++n) {
    const float tn = t[n];
    const int un = (int)u[n];
    if (tn > tprev) {
      wk.add_events(gs, n, t, u, w, base);
      wk.decay(tn - tprev);
      tprev = tn;
      gs = n;
    }
    const float *arow = alpha + un * AP + base;
    float av[MS];
    float dot = 0.f;
#pragma unroll
    for (int jj = 0; jj < MS; ++jj) {
      av[jj] = arow[jj];
      dot = fmaf(av[jj], wk.R[jj], dot);
    }
#pragma unroll
    for (int o = 1; o < SPL; o <<= 1) dot += __shfl_xor_sync(gmask, dot, o);
    const float lam = mu[un] + dot;
    const float r = __frcp_rn(lam);
    if (s == 0) {
      kahan_add(Ls, Lc, __log2f(lam));
      atomicAdd(&gm[un], r);
      if (r_out) r_out[n] = r;
    }
    float *grow = ga + un * AP + base;
#pragma unroll
    for (int jj = 0; jj < MS; ++jj) atomicAdd(&grow[jj], r * wk.R[jj]);
    if (LEARN) {
#pragma unroll
      for (int jj = 0; jj < MS; ++jj) gbl[jj] = fmaf(-r * av[jj], wk.S[jj], gbl[jj]);
    }
  }
}

// ---------------------------------------------------------------------------
// Window-level phases
// ---------------------------------------------------------------------------

// Stage (optional) and validate the window; counts and weight sums per type.
// Returns the window status (uniform across the CTA).
template <int M, bool STAGE>
__device__ int stage_and_validate(const float *tg, const int16_t *ug, const float *wg, int N,
                                  float T, int Mrt, Sm<M> &sm) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) sm.ctl[0] = 0x7fffffff;
  for (int j = tid; j < M; j += nt) {
    sm.cnt[j] = 0;
    sm.W[j] = 0.f;
  }
  __syncthreads();
  int code = 0x7fffffff;
  if (tid == 0 && (!(T >= 0.f) || !isfinite(T))) code = kE_TIME_RANGE;
  for (int n = tid; n < N; n += nt) {
    const float tv = tg[n];
    const int uv = (int)ug[n];
    const float wv = wg ? wg[n] : 1.f;
    if (!isfinite(tv) || !isfinite(wv)) code = min(code, (int)kE_NONFINITE);
    if (tv < 0.f || tv > T) code = min(code, (int)kE_TIME_RANGE);
    if (uv < 0 || uv >= Mrt) code = min(code, (int)kE_ID_RANGE);
    if (n > 0 && tv < tg[n - 1]) code = min(code, (int)kE_UNSORTED);
    if (STAGE) {
      sm.ev_t[n] = tv;
      sm.ev_u[n] = (int16_t)uv;
      if (wg) sm.ev_w[n] = wv;
    }
    if (uv >= 0 && uv < Mrt) {
      atomicAdd(&sm.cnt[uv], 1);
      atomicAdd(&sm.W[uv], wv);
    }
  }
  if (code != 0x7fffffff) atomicMin(&sm.ctl[0], code);
  __syncthreads();
  const int st = sm.ctl[0];
  return st == 0x7fffffff ? kOK : st;
}

// Chunk boundaries and anchors (a_c = first time of chunk c, T for an empty tail).
template <typename TP>
__device__ void setup_chunks(int NC, int N, float T, TP t, int *bnd, float *anc) {
  for (int c = threadIdx.x; c <= NC; c += blockDim.x) {
    const int b = chunk_begin(c, NC, N, t);
    bnd[c] = b;
    anc[c] = (c < NC && b < N) ? t[b] : T;
  }
  __syncthreads();
}

// Pass 1 + scan + compensator constants.  Leaves C, dC, endR, endS in smem.
template <int M, int SPL, int BM, bool LEARN, typename TP, typename UP, typename WP>
__device__ void prepare_states(int NC, TP t, UP u, WP w, float T, int Mrt, Sm<M> &sm) {
  const int tid = threadIdx.x;
  const int c = tid / SPL, s = tid % SPL;
  if (c < NC) {
    pass1_chunk<M, SPL, BM, LEARN>(c, s, sm.bnd[c], sm.bnd[c + 1], sm.anc[c], sm.anc[c + 1], t, u,
                                   w, sm.bl2, sm.encR, sm.encS);
  }
  __syncthreads();
  scan_chunks<M, LEARN>(NC, sm.anc, sm.bl2, BM, sm.encR, sm.encS, sm.endR, sm.endS);
  __syncthreads();
  for (int j = tid; j < M; j += blockDim.x) {
    if (j < Mrt) {
      const float b = sm.beta[BM == 0 ? 0 : j];
      const float Cj = (sm.W[j] - sm.endR[j]) / b;
      sm.C[j] = Cj;
      sm.dC[j] = LEARN ? (sm.endS[j] - Cj) / b : 0.f;
    } else {
      sm.C[j] = 0.f;
      sm.dC[j] = 0.f;
    }
  }
  __syncthreads();
}

// One lnL + gradient evaluation at the parameters in smem.  On return (after
// a barrier) ga/gm/gb hold the event sums, and the returned double is lnL
// (identical on every thread).  r_out: optional 1/lambda per event (global).
template <int M, int SPL, int BM, bool LEARN, typename TP, typename UP, typename WP>
__device__ double evaluate(int NC, TP t, UP u, WP w, float T, int Mrt, Sm<M> &sm, float *r_out) {
  constexpr int MS = M / SPL;
  constexpr int AP = M + 1;
  const int tid = threadIdx.x;
  const int c = tid / SPL, s = tid % SPL;
  float Ls = 0.f, Lc = 0.f;
  float gbl[LEARN ? MS : 1];
#pragma unroll
  for (int jj = 0; jj < (LEARN ? MS : 1); ++jj) gbl[jj] = 0.f;
  if (c < NC) {
    pass2_chunk<M, SPL, BM, LEARN>(c, s, sm.bnd[c], sm.bnd[c + 1], sm.anc[c], t, u, w, sm.bl2,
                                   sm.encR, sm.encS, sm.alpha, sm.mu, sm.ga, sm.gm, Ls, Lc, gbl,
                                   r_out);
    if (LEARN) {
      if (BM == 0) {
        float acc = 0.f;
#pragma unroll
        for (int jj = 0; jj < MS; ++jj) acc += gbl[jj];
        atomicAdd(&sm.gb[0], acc);
      } else {
#pragma unroll
        for (int jj = 0; jj < MS; ++jj) atomicAdd(&sm.gb[s * MS + jj], gbl[jj]);
      }
    }
  }
  // Part2 and Part3 terms for this thread's share of the parameters
  double part = ((double)Ls - (double)Lc) * kLn2;
  for (int p = tid; p < Mrt + Mrt * Mrt; p += blockDim.x) {
    if (p < Mrt) {
      part -= (double)T * (double)sm.mu[p];
    } else {
      const int q = p - Mrt, i = q / Mrt, j = q % Mrt;
      part -= (double)sm.alpha[i * AP + j] * (double)sm.C[j];
    }
  }
  return block_sum_double(part, sm.red);  // contains the barrier after the atomics
}

// Final gradient of parameter p (compact index: mu | alpha | beta).
template <int M, int BM, bool LEARN>
__device__ __forceinline__ float grad_of(int p, int Mrt, float T, const Sm<M> &sm) {
  constexpr int AP = M + 1;
  if (p < Mrt) return sm.gm[p] - T;
  const int q = p - Mrt;
  if (q < Mrt * Mrt) {
    const int i = q / Mrt, j = q % Mrt;
    return sm.ga[i * AP + j] - sm.C[j];
  }
  if (!LEARN) return 0.f;
  const int jb = q - Mrt * Mrt;
  if (BM == 0) {
    float acc = sm.gb[0];
    for (int j = 0; j < Mrt; ++j) {
      float col = 0.f;
      for (int i = 0; i < Mrt; ++i) col += sm.alpha[i * AP + j];
      acc -= col * sm.dC[j];
    }
    return acc;
  }
  float col = 0.f;
  for (int i = 0; i < Mrt; ++i) col += sm.alpha[i * AP + jb];
  return sm.gb[jb] - col * sm.dC[jb];
}

template <int M>
__device__ __forceinline__ float &param_ref(int p, int Mrt, Sm<M> &sm) {
  constexpr int AP = M + 1;
  if (p < Mrt) return sm.mu[p];
  const int q = p - Mrt;
  if (q < Mrt * Mrt) return sm.alpha[(q / Mrt) * AP + (q % Mrt)];
  return sm.beta[q - Mrt * Mrt];
}

template <int M>
__device__ __forceinline__ void zero_accumulators(Sm<M> &sm) {
  constexpr int AP = M + 1;
  for (int p = threadIdx.x; p < M * AP; p += blockDim.x) sm.ga[p] = 0.f;
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    sm.gm[j] = 0.f;
    sm.gb[j] = 0.f;
  }
}

}  // namespace mdhp
