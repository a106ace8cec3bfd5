/*
 * Seeded synthetic workload generator: exact simulation of an exponential-kernel
 * multi-dimensional Hawkes process by Ogata's thinning (Ogata, IEEE Trans. Inf.
 * Theory 27(1), 1981), for the intensity of Sec. II of arXiv 2411.10258:
 *   lambda_i(t) = mu_i + sum_j alpha_ij sum_{k in j, t_k < t} exp(-beta_ij (t - t_k)).
 *
 * This module only produces inputs.  It is shared by the CUDA path's tests and
 * benchmark and by the FP64 oracle's tests, and it contains none of the
 * likelihood / gradient / fitting arithmetic of either side.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) used as a
 * counter-based generator, u_k = mix(key + k * 0x9e3779b97f4a7c15), 53-bit
 * uniforms in [0, 1).  One key per window, so windows are independent of the
 * thread that simulates them.
 *
 * Thinning with the superposition split: the total intensity is
 *   Lambda = sum_i mu_i + sum_j c_j R_j,  c_j = sum_i alpha_ij  (beta per source j),
 * it only decays between events, so its value just after the current time
 * bounds it until the next event.  An accepted point is attributed to the
 * background (type i with prob. mu_i / sum mu) or to source j (prob. c_j R_j),
 * and then to target i with prob. alpha_ij / c_j: the type distribution is
 * exactly lambda_i / Lambda.  Full-matrix beta keeps M*M states instead.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

typedef struct { uint64_t key, ctr; } sim_rng;

static inline double rng_u01(sim_rng *r) {
  r->ctr += 1;
  const uint64_t z = sm64_mix(r->key + r->ctr * 0x9e3779b97f4a7c15ULL);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

/* Key for window w of stream `stream` under base seed `seed`. */
uint64_t sim_window_key(uint64_t seed, uint64_t stream, uint64_t w) {
  return sm64_mix(sm64_mix(sm64_mix(seed) ^ (stream + 0x632be59bd9b4e019ULL)) ^ (w + 1));
}

/*
 * Simulate one window.
 *   mode 0: beta[0] scalar; 1: beta[j] per source; 2: beta[i*M+j] matrix.
 *   n_target > 0: stop after n_target accepted events; T_span is then the time
 *                 of the next accepted event (not recorded), so the window is a
 *                 valid observation of exactly n_target events.
 *   T_max   > 0: stop at T_max instead (T_span = T_max); the count is random.
 *   cap: capacity of t_out/id_out.  Returns the number of events written, or
 *   -1 if cap was exceeded.
 */
int64_t sim_window(int M, int mode, const double *mu, const double *alpha, const double *beta,
                   int64_t n_target, double T_max, uint64_t key, int64_t cap,
                   double *t_out, int32_t *id_out, double *T_out) {
  sim_rng rng = {key, 0};
  const int64_t MM = (int64_t)M * M;
  const int nst = (mode == 2) ? (int)MM : M; /* decaying states */
  double *R = calloc(nst, sizeof(double));
  double *bst = malloc(nst * sizeof(double));
  double *c = calloc(M, sizeof(double));
  double mu_tot = 0.0;
  for (int i = 0; i < M; ++i) mu_tot += mu[i];
  if (mode == 2) {
    for (int64_t p = 0; p < MM; ++p) bst[p] = beta[p];
  } else {
    for (int j = 0; j < M; ++j) bst[j] = (mode == 0) ? beta[0] : beta[j];
    for (int j = 0; j < M; ++j)
      for (int i = 0; i < M; ++i) c[j] += alpha[(int64_t)i * M + j];
  }
  double t = 0.0, lam_bar;
  int64_t n = 0;
  int done = 0;
  double Tspan = T_max;
  /* intensity just after the current time */
#define SIM_TOTAL(out)                                                     \
  do {                                                                     \
    double s_ = mu_tot;                                                    \
    if (mode == 2) {                                                       \
      for (int64_t p_ = 0; p_ < MM; ++p_) s_ += alpha[p_] * R[p_];         \
    } else {                                                               \
      for (int j_ = 0; j_ < M; ++j_) s_ += c[j_] * R[j_];                  \
    }                                                                      \
    (out) = s_;                                                            \
  } while (0)
  SIM_TOTAL(lam_bar);
  while (!done) {
    if (!(lam_bar > 0.0)) { Tspan = (T_max > 0.0) ? T_max : t; break; }
    const double e = -log1p(-rng_u01(&rng));
    const double tc = t + e / lam_bar;
    if (T_max > 0.0 && tc > T_max) { Tspan = T_max; break; }
    const double dt = tc - t;
    for (int s = 0; s < nst; ++s) R[s] *= exp(-bst[s] * dt);
    t = tc;
    double lam;
    SIM_TOTAL(lam);
    const double u = rng_u01(&rng) * lam_bar;
    if (u <= lam) {
      if (n_target > 0 && n == n_target) { Tspan = t; break; }
      if (n >= cap) { n = -1; break; }
      /* attribute the point: background or one source's excitation */
      double v = rng_u01(&rng) * lam;
      int ty = -1;
      if (v < mu_tot) {
        for (int i = 0; i < M; ++i) { if (v < mu[i]) { ty = i; break; } v -= mu[i]; }
        if (ty < 0) ty = M - 1;
      } else if (mode == 2) {
        v -= mu_tot;
        for (int64_t p = 0; p < MM; ++p) {
          const double q = alpha[p] * R[p];
          if (v < q) { ty = (int)(p / M); break; }
          v -= q;
        }
        if (ty < 0) ty = M - 1;
      } else {
        v -= mu_tot;
        int src = -1;
        for (int j = 0; j < M; ++j) {
          const double q = c[j] * R[j];
          if (v < q) { src = j; break; }
          v -= q;
        }
        if (src < 0) src = M - 1;
        double v2 = rng_u01(&rng) * c[src];
        for (int i = 0; i < M; ++i) {
          const double a = alpha[(int64_t)i * M + src];
          if (v2 < a) { ty = i; break; }
          v2 -= a;
        }
        if (ty < 0) ty = M - 1;
      }
      t_out[n] = t;
      id_out[n] = ty;
      ++n;
      if (mode == 2) {
        for (int i = 0; i < M; ++i) R[(int64_t)i * M + ty] += 1.0;
      } else {
        R[ty] += 1.0;
      }
      SIM_TOTAL(lam_bar);
    } else {
      lam_bar = lam;
    }
  }
#undef SIM_TOTAL
  *T_out = Tspan;
  free(R); free(bst); free(c);
  return n;
}

/*
 * Batch of B windows with known exact counts n_target[b] into CSR arrays
 * (offsets[b] = sum of earlier counts), timestamps rounded to float32 and ids
 * narrowed to int16 -- the layout the library consumes.  Parameters per window:
 * mu[B*M], alpha[B*M*M], beta[B*nb].  OpenMP over windows.
 * Returns 0, or -1 if any window failed.
 */
int sim_batch(int B, int M, int mode, const double *mu, const double *alpha, const double *beta,
              const int64_t *n_target, const int64_t *offsets, uint64_t seed, uint64_t stream,
              float *t32, int16_t *id16, float *Tspan32, int nthreads) {
  const int nb = mode == 0 ? 1 : (mode == 1 ? M : M * M);
  const int64_t MM = (int64_t)M * M;
  int bad = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
#endif
  for (int b = 0; b < B; ++b) {
    const int64_t N = n_target[b];
    double *t = malloc((N > 0 ? N : 1) * sizeof(double));
    int32_t *id = malloc((N > 0 ? N : 1) * sizeof(int32_t));
    double T;
    const int64_t got = sim_window(M, mode, mu + (int64_t)b * M, alpha + (int64_t)b * MM,
                                   beta + (int64_t)b * nb, N, 0.0, sim_window_key(seed, stream, b),
                                   N, t, id, &T);
    if (got != N) {
      bad |= 1;
    } else {
      const int64_t o = offsets[b];
      for (int64_t n = 0; n < N; ++n) {
        t32[o + n] = (float)t[n];
        id16[o + n] = (int16_t)id[n];
      }
      float Tf = (float)T;
      /* float rounding keeps order; never let T_span fall below the last event */
      if (N > 0 && Tf < t32[o + N - 1]) Tf = t32[o + N - 1];
      Tspan32[b] = Tf;
    }
    free(t); free(id);
  }
  return bad ? -1 : 0;
}
