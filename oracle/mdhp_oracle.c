/*
 * FP64 CPU oracle for MDHP-GDS (test infrastructure only).
 *
 * This file is the checker, not the product: only tests/, the smoke entry and
 * the CPU-baseline leg of the benchmark load it.  It shares no code, header,
 * table or helper with the CUDA path; the two meet only through the seeded
 * input generator (a separate module that holds none of the arithmetic here).
 *
 * What it computes, and where the paper defines it (arXiv 2411.10258):
 *   - intensity      lambda_i(t) = theta_i + sum_j sum_{k: T_j^k < t}
 *                    alpha_ij exp(-beta_ij (t - T_j^k))          (Sec. II, MDHP intensity eq.)
 *   - log-likelihood lnL = Part1 + Part2 + Part3 with
 *                    Part1 = sum over events of ln lambda_{u_n}(t_n)
 *                    Part2 = -T_span sum_i theta_i
 *                    Part3 = sum_ij (alpha_ij/beta_ij) sum_{k in j}
 *                            (exp(-beta_ij (T_span - T_j^k)) - 1)  (Sec. IV-B.1, closed-form lnL eq.;
 *                                                                    App. B derivation of Gamma)
 *   - its analytic gradient in (theta, alpha, beta) and in optional per-event
 *     weights w_k (w = 1 recovers the paper's likelihood exactly);
 *   - projected gradient ascent on lnL / N_w (Sec. IV-B.2: "three autograd
 *     tensors ... optimised with a PyTorch optimizer"; the optimiser, step and
 *     stopping rule are not given in the paper, the readings used are stated
 *     at oracle_fit below).
 *
 * Readings of points the paper leaves open (all documented in the design notes):
 *   - alpha index: row = target i, column = source j, as in the intensity formula.
 *   - ties: the inner sum is strict (T_j^k < t), so events sharing a timestamp
 *     do not excite one another; every lambda of a tie group is evaluated before
 *     any of that group's increments is added.
 *   - the algorithms' "clamp_max(., 80)" exists only for padded entries of the
 *     broadcast design; every exponent here is <= 0, so there is no clamp.
 *   - Part3 keeps the "-1" term printed in the closed-form equation and App. B
 *     (Alg. 3 omits it).
 *
 * Method: the exact O(N * M^2) forward recursion on R_ij(t) =
 * sum_{k in j, t_k < t} w_k exp(-beta_ij (t - t_k)) and
 * S_ij(t) = sum w_k (t - t_k) exp(-beta_ij (t - t_k)) (the beta-derivative state),
 * plain double sums, libm exp/log/expm1.  The reverse recursion for the event
 * weights carries P_ij(t) = sum_{n: t_n > t, u_n = i} r_n exp(-beta_ij (t_n - t)).
 * Pinned in tests against: an O(N^2) brute-force double sum, piecewise
 * quadrature of the compensator, the alpha = 0 closed form, the univariate
 * (Ozaki) form, central finite differences, invariances and parameter recovery.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_E_ARG 1
#define ORC_E_UNSORTED 2
#define ORC_E_ID_RANGE 3
#define ORC_E_TIME_RANGE 4
#define ORC_E_NONFINITE 5
#define ORC_E_MAXITER 6

/* beta for pair (target i, source j) under the three shapes:
 * 0 = one scalar, 1 = one per source j, 2 = full matrix. */
static double beta_at(int mode, const double *beta, int M, int i, int j) {
  if (mode == 0) return beta[0];
  if (mode == 1) return beta[j];
  return beta[(int64_t)i * M + j];
}

static int nbeta(int mode, int M) { return mode == 0 ? 1 : (mode == 1 ? M : M * M); }

/* Input checks; returns the smallest violated code (0 if none). */
int oracle_validate(int M, int64_t N, const double *t, const int32_t *id,
                    const double *w, double T) {
  int code = 0;
#define ORC_FLAG(c) do { if (code == 0 || (c) < code) code = (c); } while (0)
  if (!(T >= 0.0) || !isfinite(T)) ORC_FLAG(ORC_E_TIME_RANGE);
  for (int64_t n = 0; n < N; ++n) {
    if (!isfinite(t[n]) || (w && !isfinite(w[n]))) ORC_FLAG(ORC_E_NONFINITE);
    if (t[n] < 0.0 || t[n] > T) ORC_FLAG(ORC_E_TIME_RANGE);
    if (id[n] < 0 || id[n] >= M) ORC_FLAG(ORC_E_ID_RANGE);
    if (n > 0 && t[n] < t[n - 1]) ORC_FLAG(ORC_E_UNSORTED);
  }
#undef ORC_FLAG
  return code;
}

/*
 * lnL and gradient for one window.
 *   t[N] (sorted, seconds from window start, 0 <= t <= T), id[N] in [0, M),
 *   w[N] event weights or NULL (= 1), mu[M], alpha[M*M] (row = target),
 *   beta: [1] | [M] | [M*M] per mode.
 * Outputs (any may be NULL except out_lnL): g_mu[M], g_alpha[M*M],
 *   g_beta (same shape as beta), g_w[N], r_out[N] = 1 / lambda_{u_n}(t_n).
 * Returns a status code (inputs are validated first).
 */
int oracle_loglik_grad(int M, int mode, int64_t N, const double *t, const int32_t *id,
                       const double *w, double T, const double *mu, const double *alpha,
                       const double *beta, double *out_lnL, double *g_mu, double *g_alpha,
                       double *g_beta, double *g_w, double *r_out) {
  if (M <= 0 || mode < 0 || mode > 2 || N < 0) return ORC_E_ARG;
  int st = oracle_validate(M, N, t, id, w, T);
  if (st) return st;
  const int64_t MM = (int64_t)M * M;
  double *R = calloc(MM, sizeof(double)), *S = calloc(MM, sizeof(double));
  double *ga = calloc(MM, sizeof(double)), *gb = calloc(MM, sizeof(double));
  double *gm = calloc(M, sizeof(double));
  double *bij = malloc(MM * sizeof(double));
  double *r = malloc((N > 0 ? N : 1) * sizeof(double));
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) bij[(int64_t)i * M + j] = beta_at(mode, beta, M, i, j);

  /* Part1 by the forward recursion, one tie group at a time. */
  double part1 = 0.0, tprev = 0.0;
  int64_t n = 0;
  while (n < N) {
    const double tg = t[n];
    int64_t ge = n;
    while (ge < N && t[ge] == tg) ++ge;
    const double dt = tg - tprev;
    if (dt > 0.0) {
      for (int64_t p = 0; p < MM; ++p) {
        const double a = exp(-bij[p] * dt);
        S[p] = a * (S[p] + dt * R[p]);
        R[p] = a * R[p];
      }
    }
    for (int64_t k = n; k < ge; ++k) {
      const int i = id[k];
      const double *Ri = R + (int64_t)i * M, *Si = S + (int64_t)i * M;
      const double *ai = alpha + (int64_t)i * M;
      double lam = mu[i];
      for (int j = 0; j < M; ++j) lam += ai[j] * Ri[j];
      part1 += log(lam);
      const double rk = 1.0 / lam;
      r[k] = rk;
      gm[i] += rk;
      for (int j = 0; j < M; ++j) {
        ga[(int64_t)i * M + j] += rk * Ri[j];
        gb[(int64_t)i * M + j] -= rk * ai[j] * Si[j];
      }
    }
    for (int64_t k = n; k < ge; ++k) {
      const int j = id[k];
      const double wk = w ? w[k] : 1.0;
      for (int i = 0; i < M; ++i) R[(int64_t)i * M + j] += wk;
    }
    tprev = tg;
    n = ge;
  }

  /* Part2 and Part3 (the compensator), event by event. */
  double part2 = 0.0;
  for (int i = 0; i < M; ++i) part2 -= T * mu[i];
  double *C = calloc(MM, sizeof(double)), *dC = calloc(MM, sizeof(double));
  for (int64_t k = 0; k < N; ++k) {
    const int j = id[k];
    const double tau = T - t[k], wk = w ? w[k] : 1.0;
    for (int i = 0; i < M; ++i) {
      const int64_t p = (int64_t)i * M + j;
      const double b = bij[p];
      const double e = exp(-b * tau);
      const double om = -expm1(-b * tau); /* 1 - exp(-b tau) */
      C[p] += wk * om / b;
      dC[p] += wk * (tau * e / b - om / (b * b));
    }
  }
  double part3 = 0.0;
  for (int64_t p = 0; p < MM; ++p) part3 -= alpha[p] * C[p];
  *out_lnL = part1 + part2 + part3;

  if (g_mu)
    for (int i = 0; i < M; ++i) g_mu[i] = gm[i] - T;
  if (g_alpha)
    for (int64_t p = 0; p < MM; ++p) g_alpha[p] = ga[p] - C[p];
  if (g_beta) {
    for (int q = 0; q < nbeta(mode, M); ++q) g_beta[q] = 0.0;
    for (int i = 0; i < M; ++i)
      for (int j = 0; j < M; ++j) {
        const int64_t p = (int64_t)i * M + j;
        const double v = gb[p] - alpha[p] * dC[p];
        if (mode == 0) g_beta[0] += v;
        else if (mode == 1) g_beta[j] += v;
        else g_beta[p] = v;
      }
  }
  if (r_out)
    for (int64_t k = 0; k < N; ++k) r_out[k] = r[k];

  /* d lnL / d w_k: reverse recursion over tie groups (strict t_n > t_k). */
  if (g_w && N > 0) {
    double *P = calloc(MM, sizeof(double));
    double tnext = t[N - 1];
    int64_t e = N;
    while (e > 0) {
      const double tg = t[e - 1];
      int64_t gs = e - 1;
      while (gs > 0 && t[gs - 1] == tg) --gs;
      const double dt = tnext - tg;
      if (dt > 0.0)
        for (int64_t p = 0; p < MM; ++p) P[p] *= exp(-bij[p] * dt);
      for (int64_t k = gs; k < e; ++k) {
        const int j = id[k];
        double acc = 0.0;
        for (int i = 0; i < M; ++i) acc += alpha[(int64_t)i * M + j] * P[(int64_t)i * M + j];
        const double tau = T - t[k];
        double comp = 0.0;
        for (int i = 0; i < M; ++i) {
          const double b = bij[(int64_t)i * M + j];
          comp += alpha[(int64_t)i * M + j] * (-expm1(-b * tau)) / b;
        }
        g_w[k] = acc - comp;
      }
      for (int64_t k = gs; k < e; ++k) {
        const int i = id[k];
        for (int j = 0; j < M; ++j) P[(int64_t)i * M + j] += r[k];
      }
      tnext = tg;
      e = gs;
    }
    free(P);
  }
  free(R); free(S); free(ga); free(gb); free(gm); free(bij); free(r); free(C); free(dC);
  return isfinite(*out_lnL) ? ORC_OK : ORC_E_NONFINITE;
}

/*
 * Cold start used when no initial guess is given (the paper does not state
 * one): mu_i = 0.5 max(N_i, 1) / T, alpha_ij = 0.5 beta_ij / M, which puts the
 * spectral radius of alpha/beta at 0.5.  beta is left as given.
 */
void oracle_cold_init(int M, int mode, int64_t N, const int32_t *id, double T,
                      const double *beta, double *mu, double *alpha) {
  for (int i = 0; i < M; ++i) mu[i] = 0.0;
  for (int64_t n = 0; n < N; ++n)
    if (id[n] >= 0 && id[n] < M) mu[id[n]] += 1.0;
  for (int i = 0; i < M; ++i) mu[i] = 0.5 * (mu[i] > 1.0 ? mu[i] : 1.0) / T;
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) alpha[(int64_t)i * M + j] = 0.5 * beta_at(mode, beta, M, i, j) / M;
}

/* Fit options, mirrored field for field by the Python wrapper. */
typedef struct {
  int32_t optimizer;   /* 0 = projected gradient ascent, 1 = projected Adam */
  int32_t max_iters;   /* number of lnL/gradient evaluations */
  int32_t fit_beta;    /* 1: beta is a parameter too */
  int32_t patience;    /* consecutive small changes needed to stop (3) */
  double lr;
  double tol;          /* stop when |lnL_k - lnL_{k-1}| <= tol |lnL_k|, patience times in a row */
  double mu_floor, alpha_floor, beta_floor;
  double adam_b1, adam_b2, adam_eps;
} oracle_fit_opts;

/*
 * Projected ascent on f = lnL / max(N, 1) (the readings of the paper's
 * unspecified optimiser):
 *   for k = 0, 1, ...: evaluate (lnL_k, g_k) at theta_k; stop if converged,
 *   non-finite or k = max_iters - 1; else theta_{k+1} = Proj(theta_k + step(g_k / N)).
 * Proj clamps mu >= mu_floor, alpha >= alpha_floor, beta >= beta_floor.
 * On return mu/alpha/beta hold the last evaluated point, *lnL its value and
 * *iters the number of evaluations.  A non-finite evaluation restores the
 * previous point and its lnL.
 */
int oracle_fit(int M, int mode, int64_t N, const double *t, const int32_t *id, const double *w,
               double T, const oracle_fit_opts *o, double *mu, double *alpha, double *beta,
               double *lnL_out, int32_t *iters_out) {
  const int64_t MM = (int64_t)M * M;
  const int nb = nbeta(mode, M);
  const int np = M + (int)MM + nb;
  int st = oracle_validate(M, N, t, id, w, T);
  *iters_out = 0;
  if (st) { *lnL_out = NAN; return st; }
  double *th = malloc(np * sizeof(double)), *prev = malloc(np * sizeof(double));
  double *g = malloc(np * sizeof(double));
  double *m1 = calloc(np, sizeof(double)), *m2 = calloc(np, sizeof(double));
  memcpy(th, mu, M * sizeof(double));
  memcpy(th + M, alpha, MM * sizeof(double));
  memcpy(th + M + MM, beta, nb * sizeof(double));
  const double scale = 1.0 / (double)(N > 0 ? N : 1);
  double lnL = 0.0, lnL_prev = 0.0;
  int streak = 0, k = 0;
  st = (o->tol > 0.0) ? ORC_E_MAXITER : ORC_OK;
  double b1t = 1.0, b2t = 1.0;
  for (k = 0; k < o->max_iters; ++k) {
    double val;
    int s = oracle_loglik_grad(M, mode, N, t, id, w, T, th, th + M, th + M + MM, &val,
                               g, g + M, g + M + MM, NULL, NULL);
    int finite = (s == ORC_OK);
    for (int q = 0; q < np && finite; ++q) finite = isfinite(g[q]);
    if (!finite) {
      if (k > 0) memcpy(th, prev, np * sizeof(double));
      else lnL = val;
      st = ORC_E_NONFINITE;
      break;
    }
    if (k > 0 && o->tol > 0.0 && fabs(val - lnL_prev) <= o->tol * fabs(val)) ++streak;
    else streak = 0;
    lnL = val;
    lnL_prev = val;
    if (o->tol > 0.0 && streak >= o->patience) { st = ORC_OK; ++k; break; }
    if (k == o->max_iters - 1) { ++k; break; }
    memcpy(prev, th, np * sizeof(double));
    const int nupd = o->fit_beta ? np : M + (int)MM;
    b1t *= o->adam_b1;
    b2t *= o->adam_b2;
    for (int q = 0; q < nupd; ++q) {
      const double gs = g[q] * scale;
      double step;
      if (o->optimizer == 1) {
        m1[q] = o->adam_b1 * m1[q] + (1.0 - o->adam_b1) * gs;
        m2[q] = o->adam_b2 * m2[q] + (1.0 - o->adam_b2) * gs * gs;
        const double mh = m1[q] / (1.0 - b1t), vh = m2[q] / (1.0 - b2t);
        step = o->lr * mh / (sqrt(vh) + o->adam_eps);
      } else {
        step = o->lr * gs;
      }
      const double fl = q < M ? o->mu_floor : (q < M + MM ? o->alpha_floor : o->beta_floor);
      const double v = th[q] + step;
      th[q] = v > fl ? v : fl;
    }
  }
  memcpy(mu, th, M * sizeof(double));
  memcpy(alpha, th + M, MM * sizeof(double));
  memcpy(beta, th + M + MM, nb * sizeof(double));
  *lnL_out = lnL;
  *iters_out = k;
  free(th); free(prev); free(g); free(m1); free(m2);
  return st;
}

/*
 * Batched fit over B windows in CSR layout (offsets[B+1]); FP32 timestamps and
 * int16 ids are widened to double here, exactly as the GPU path receives them.
 * A plain OpenMP loop over windows: this is what the CPU baseline times.
 * Parameter arrays are [B*M], [B*M*M], [B*nb] (in/out).
 */
int oracle_fit_batch(int B, int M, int mode, const int64_t *offsets, const float *t32,
                     const int16_t *id16, const float *w32, const float *Tspan,
                     const oracle_fit_opts *o, double *mu, double *alpha, double *beta,
                     double *lnL, int32_t *iters, int32_t *status, int nthreads) {
  const int64_t MM = (int64_t)M * M;
  const int nb = nbeta(mode, M);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int b = 0; b < B; ++b) {
    const int64_t o0 = offsets[b], N = offsets[b + 1] - offsets[b];
    double *t = malloc((N > 0 ? N : 1) * sizeof(double));
    int32_t *id = malloc((N > 0 ? N : 1) * sizeof(int32_t));
    double *w = w32 ? malloc((N > 0 ? N : 1) * sizeof(double)) : NULL;
    for (int64_t n = 0; n < N; ++n) {
      t[n] = (double)t32[o0 + n];
      id[n] = (int32_t)id16[o0 + n];
      if (w) w[n] = (double)w32[o0 + n];
    }
    status[b] = oracle_fit(M, mode, N, t, id, w, (double)Tspan[b], o, mu + (int64_t)b * M,
                           alpha + (int64_t)b * MM, beta + (int64_t)b * nb, lnL + b, iters + b);
    free(t); free(id); free(w);
  }
  return 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
