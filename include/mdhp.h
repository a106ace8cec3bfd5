/*
 * mdhp.h -- C ABI of the GB300 (sm_103a) MDHP-GDS library.
 *
 * MDHP-GDS (arXiv 2411.10258, Sec. IV-B) fits the parameters of an
 * exponential-kernel multi-dimensional Hawkes process to windows of
 * time-stamped messages by gradient ascent on the log-likelihood:
 *
 *   lambda_i(t) = mu_i + sum_j sum_{k: t_k < t, u_k = j} w_k alpha_ij exp(-beta_ij (t - t_k))
 *                                                   (Sec. II, MDHP intensity eq.; mu is the paper's theta)
 *   lnL = sum_n ln lambda_{u_n}(t_n)                                        (Part1)
 *         - T_span sum_i mu_i                                               (Part2)
 *         + sum_ij (alpha_ij / beta_ij) sum_{k: u_k = j} w_k (exp(-beta_ij (T_span - t_k)) - 1)   (Part3)
 *                                                   (Sec. IV-B.1 closed-form lnL eq.; App. B)
 *
 * w_k are optional per-event weights (NULL = 1, which is the paper's model).
 * Index convention: alpha is row-major [M][M], row = target i, column = source j,
 * as in the intensity formula.  beta has one of three shapes (mdhp_beta_mode).
 * Events that share a timestamp do not excite one another (the sum is strict).
 *
 * Conventions for every entry point:
 *   - All array pointers are DEVICE pointers unless stated otherwise, owned by
 *     the caller; the library never frees them.  The library allocates device
 *     memory only inside an mdhp_plan (mdhp_plan_create) and frees it in
 *     mdhp_plan_destroy.
 *   - Calls are asynchronous and stream-ordered on `stream` (a cudaStream_t,
 *     NULL = the legacy default stream).
 *   - Argument errors are returned synchronously and nothing is launched.
 *     Data errors are reported per window in win_status[] (int32 mdhp_status);
 *     the call itself then still returns MDHP_OK.  MDHP_E_CUDA means a launch
 *     failed; mdhp_last_error() gives the text.
 *   - Gradients are of lnL itself (ascent direction), not of -lnL.
 *   - Matrix-shaped beta (MDHP_BETA_MATRIX, the paper's general form) is
 *     supported by mdhp_fit_batch with a fixed beta (fit_beta = 0) for M <= 32
 *     on a plan with a stated max_events_per_window (the decoupled kernels);
 *     every other call with matrix beta returns MDHP_E_UNSUPPORTED.
 *   - M (number of event types / message IDs) is limited to 1..64.
 */
#ifndef MDHP_H_
#define MDHP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MDHP_OK = 0,
  MDHP_E_ARG = 1,          /* bad argument (sizes, NULL, unsupported M) */
  MDHP_E_UNSORTED = 2,     /* window timestamps not non-decreasing */
  MDHP_E_ID_RANGE = 3,     /* an id outside [0, M) */
  MDHP_E_TIME_RANGE = 4,   /* a timestamp outside [0, T_span], or T_span < 0 / not finite */
  MDHP_E_NONFINITE = 5,    /* NaN/Inf in inputs, or lnL / gradient not finite */
  MDHP_E_MAXITER = 6,      /* fit: tolerance requested but not met within max_iters */
  MDHP_E_TIMEOUT = 7,      /* a bounded device-side wait gave up (window results invalid) */
  MDHP_E_CUDA = 8,         /* a CUDA call failed */
  MDHP_E_NOMEM = 9,        /* plan allocation failed */
  MDHP_E_UNSUPPORTED = 10, /* valid request this build does not implement */
  MDHP_E_SIM_STALLED = 11  /* mdhp_simulate: the intensity vanished (or the candidate
                              limit was hit) before the window had its events */
} mdhp_status;

typedef enum {
  MDHP_BETA_SCALAR = 0,     /* beta[B]: one decay per window */
  MDHP_BETA_PER_SOURCE = 1, /* beta[B][M]: beta_ij = beta_j (decay of source j's excitation) */
  MDHP_BETA_MATRIX = 2      /* beta[B][M][M]: the paper's general (D, D) form (fixed-beta fits) */
} mdhp_beta_mode;

/*
 * A batch of B independent windows in CSR layout (replaces the paper's
 * padding to maxTimeLen, Sec. IV-B.3 Stage 1).
 *   offsets   int64[B+1], offsets[0] = 0, non-decreasing; window b holds events
 *             offsets[b] .. offsets[b+1]-1.
 *   t         float32[n_events], seconds from the window start, non-decreasing
 *             within a window, 0 <= t <= T_span[b].
 *   id        int16[n_events], event type (message ID) in [0, M).
 *   T_span    float32[B], observation length of each window (the integral of
 *             the compensator runs over [0, T_span]).
 *   weights   float32[n_events] or NULL.
 *   max_events  an upper bound on events per window, 0 = unknown.  When it is
 *             known and small enough, windows are staged in shared memory;
 *             a window longer than a stated max_events gets MDHP_E_ARG.
 */
typedef struct {
  int32_t B;
  int32_t M;
  int64_t n_events;
  const int64_t *offsets;
  const float *t;
  const int16_t *id;
  const float *T_span;
  const float *weights;
  int32_t beta_mode;
  int32_t max_events;
} mdhp_batch;

/*
 * lnL and its gradient for every window at the given parameters
 * (closed-form lnL, Sec. IV-B.1; gradient by the same O(N M) recursion).
 *   mu     float32[B][M]           (the paper's theta)
 *   alpha  float32[B][M][M]        row = target
 *   beta   float32[B] | [B][M]     per batch->beta_mode
 * Outputs (device):
 *   loglik    float64[B]             lnL per window (NaN if the window is invalid)
 *   g_mu      float32[B][M]          d lnL / d mu
 *   g_alpha   float32[B][M][M]       d lnL / d alpha
 *   g_beta    float32[B] | [B][M], or NULL (skips the beta-derivative states)
 *   g_weights float32[n_events], or NULL: d lnL / d w_k for every event
 *   r_work    float32[n_events] caller-provided scratch, required iff
 *             g_weights != NULL (holds 1/lambda at each event between the
 *             forward and the reverse pass)
 *   win_status int32[B] (mdhp_status per window)
 */
mdhp_status mdhp_loglik_grad(const mdhp_batch *batch, const float *mu, const float *alpha,
                             const float *beta, double *loglik, float *g_mu, float *g_alpha,
                             float *g_beta, float *g_weights, float *r_work, int32_t *win_status,
                             void *stream);

/*
 * Options of the fit.  The paper fixes none of the optimiser, step, start
 * point or stopping rule (Sec. IV-B.2: "a PyTorch optimizer"); these are the
 * library's readings:
 *   objective  f = lnL / max(N_w, 1) per window (scale-free step size)
 *   optimizer  0: projected gradient ascent  theta <- max(theta + lr * grad f, floor)
 *              1: projected Adam (adam_b1, adam_b2, adam_eps) on grad f
 *   iteration  k = 0, 1, ...: evaluate lnL_k and its gradient at theta_k; stop when
 *              |lnL_k - lnL_{k-1}| <= tol |lnL_k| held `patience` times in a row
 *              (tol > 0), or k = max_iters - 1, or the evaluation is not finite
 *              (then the previous point is restored); otherwise update.
 *              The returned parameters are the last evaluated point.
 *   floors     mu >= mu_floor, alpha >= alpha_floor, beta >= beta_floor
 *   fit_beta   1: beta is updated too (per-source or scalar)
 *   init       0: start from the parameters passed in (warm start / resume)
 *              1: cold start, mu_i = 0.5 max(N_i,1) / T_span, alpha_ij = 0.5 beta_ij / M
 *                 (spectral radius of alpha/beta = 0.5); beta as passed in
 *              2: learned initializer (the plan must hold a model, see
 *                 mdhp_plan_set_init_model; M <= 32); beta as passed in
 */
typedef struct {
  int32_t optimizer;
  int32_t max_iters;
  int32_t fit_beta;
  int32_t patience;
  float lr;
  float mu_floor;
  float alpha_floor;
  float beta_floor;
  float adam_b1;
  float adam_b2;
  float adam_eps;
  int32_t init;
  double tol;
} mdhp_fit_opts;

/* Fills the defaults: optimizer 0, max_iters 200, fit_beta 0, patience 3,
 * lr 1e-2, floors 1e-10 / 0 / 1e-6, Adam 0.9 / 0.999 / 1e-8, init 1, tol 0. */
void mdhp_fit_opts_default(mdhp_fit_opts *opts);

/*
 * A plan owns the device scratch of batched fitting (length-sorted work queue,
 * counters, sort workspace) and the tuned launch shape.  It is created for one
 * (M, beta_mode) and at most max_windows windows of at most
 * max_events_per_window events (0 = no stated bound: long windows are then
 * streamed from device memory).  autotune_cache: path of a JSON file written
 * by mdhp_plan_autotune and read here, or NULL.
 * Not thread-safe: one plan per concurrent stream.
 */
typedef struct mdhp_plan mdhp_plan;

mdhp_status mdhp_plan_create(mdhp_plan **plan, int32_t M, int32_t beta_mode, int32_t max_windows,
                             int64_t max_events_per_window, const char *autotune_cache);
void mdhp_plan_destroy(mdhp_plan *plan);

/*
 * Batched MDHP-GDS: fits every window of `batch` (B <= the plan's max_windows)
 * in one persistent launch per length class, windows taken longest first.
 *   mu, alpha, beta  in/out, shapes as in mdhp_loglik_grad
 *   loglik   float64[B] lnL at the returned parameters
 *   iters    int32[B]   number of lnL/gradient evaluations
 *   win_status int32[B] MDHP_OK, MDHP_E_MAXITER, MDHP_E_NONFINITE or an input error
 * Capturable in a CUDA graph (no host synchronisation, no allocation).
 */
mdhp_status mdhp_fit_batch(mdhp_plan *plan, const mdhp_batch *batch, const mdhp_fit_opts *opts,
                           float *mu, float *alpha, float *beta, double *loglik, int32_t *iters,
                           int32_t *win_status, void *stream);

/* Device time (ms) of the fit kernels of the last mdhp_fit_batch call on this
 * plan (the learned initializer's prediction and the length sort excluded),
 * measured with CUDA events recorded on the call's stream around them
 * (the call synchronises on those events).  Requires timing to have been
 * enabled with mdhp_plan_set_timing(plan, 1) before the call.  Returns <0 if
 * no timing is available. */
mdhp_status mdhp_plan_set_timing(mdhp_plan *plan, int32_t enable);
float mdhp_plan_last_fit_ms(mdhp_plan *plan);

/* Number of kernels the last mdhp_fit_batch on this plan launched (length
 * keys, the radix sort counted as one kernel, the range split, the fit
 * kernels, and with init = 2 the learned initializer's features, GEMM and
 * head kernels), or -1 for a NULL plan. */
int32_t mdhp_plan_last_launches(const mdhp_plan *plan);

/* Launch shape (for tests, reports and tuning): threads per window and
 * threads per chunk of the event recursion, and the shared-memory cutoff:
 * windows of at most this many events are staged in shared memory (the
 * recursion) or keep their decoupled features in shared memory (fixed beta);
 * longer windows stream from device memory.  A cutoff of 0 streams all.
 * When the plan has decoupled-feature scratch and the path is MDHP_PATH_AUTO,
 * get_shape reports the decoupled kernels' threads per window and cutoff. */
mdhp_status mdhp_plan_get_shape(const mdhp_plan *plan, int32_t *threads_per_window,
                                int32_t *threads_per_chunk, int32_t *smem_cutoff_events);
mdhp_status mdhp_plan_set_shape(mdhp_plan *plan, int32_t threads_per_window,
                                int32_t threads_per_chunk, int32_t smem_cutoff_events);

/*
 * Autotuner (an addition of this library): times mdhp_fit_batch on `batch`
 * with `opts` for each candidate launch shape and keeps the fastest in the
 * plan.  Candidates: 64, 128 and 256 threads per window; for the decoupled
 * fixed-beta kernels the shared-memory class (none, half, the largest that
 * fits), the feature ring (none; 1x4, 2x3, 2x4, 4x3 steps x stages) and the
 * two-launch split (off; 256 x 1, 256 x 2, 128 x 1, 128 x 2 long threads x CTAs per
 * SM; not tried when the plan's split was disabled with mdhp_plan_set_split before the
 * call), and at template width 32 the tensor-memory feature store
 * (mdhp_plan_set_feature_store 1, 2 and 3; no ring, no split; the
 * choice is read back with mdhp_plan_get_feature_store); for the event
 * recursion every built threads-per-chunk split and the
 * staging cutoff (none, the default, the largest that fits).  One warm-up
 * run comes first.  With opts->tol == 0 each candidate runs tune_iters
 * iterations (<= 0: 20) on every window.  With opts->tol > 0 each candidate
 * runs the caller's fit to that tolerance (its optimizer, start and patience),
 * at most min(opts->max_iters, tune_iters) evaluations per window (tune_iters
 * <= 0: 500): the makespan of such a fit is set by its slowest-converging
 * windows, which fixed-count runs do not see.
 *   mu, alpha, beta  device, as for mdhp_fit_batch; used as the starting point
 *                    when opts->init == 0 and restored on return
 *   loglik, iters, win_status  device scratch, overwritten
 *   chosen   int32[9] host or NULL: path (0 decoupled, 1 recursion), threads
 *            per window, threads per chunk (0 for decoupled), cutoff, the
 *            feature ring's steps per stage and stages (mdhp_plan_set_pipeline),
 *            and the split (enabled, long_threads, long_ctas_per_sm;
 *            mdhp_plan_set_split)
 *   best_ms  float host or NULL: device time of the chosen shape
 * When the plan was created with an autotune_cache path, the choice is
 * written there under a key of the device name and compute capability, M,
 * beta_mode, max_windows and max_events_per_window and the kernel family;
 * mdhp_plan_create with the same arguments and file applies it.
 * Synchronises `stream`; allocates a temporary copy of mu/alpha/beta; not
 * capturable in a CUDA graph (tune first, then capture).
 */
mdhp_status mdhp_plan_autotune(mdhp_plan *plan, const mdhp_batch *batch, const mdhp_fit_opts *opts,
                               float *mu, float *alpha, float *beta, double *loglik, int32_t *iters,
                               int32_t *win_status, int32_t tune_iters, int32_t *chosen,
                               float *best_ms, void *stream);

/*
 * Learned warm start (an addition of this library; the paper starts its
 * descent from an unstated point).  A 4-layer MLP (BF16 weights and
 * activations, FP32 accumulation, ReLU, width `hidden`) maps per-window
 * features to a starting point (mu, alpha) for the fit; it is trained on the
 * GPU by mdhp_init_train_step on windows whose targets the fit itself produced.
 *
 * Features of a window (feature_dim = M + 32 M^2 + 3, zero-padded to a multiple
 * of 64, BF16 row-major [B][feature_dim]): the share N_i / N of each type; for
 * every ordered pair (i, j) a 32-bin histogram of log2(gap * N / T), gap = time
 * from each type-i event back to the last strictly earlier type-j event, bin
 * floor(log2) + 16 clamped to [0, 31], normalised to sum 1; log N, log T, beta.
 * mu_cold [B][M] receives the fit's cold start 0.5 max(N_i, 1) / T.
 * Head: mu_i = mu_cold_i exp(clamp(y_i, -6, 6)), alpha_ij = beta_ij / M * softplus(y_ij).
 * Training loss per window (mean over the batch):
 *   sum_i (y_i - clamp(log(mu*_i / mu_cold_i), -6, 6))^2 + sum_ij (softplus(y_ij) - alpha*_ij M / beta_ij)^2
 * (the clamp matches the head's range: a mu* at its floor is not chased to -inf).
 * M is limited to 1..32.
 */
typedef struct mdhp_init_model mdhp_init_model;

/* Allocates weights (FP32 master + BF16 copy, uniform(+-1/sqrt(fan_in)) from
 * `seed`, zero biases), AdamW moments and activations for batches of up to
 * max_batch windows. */
mdhp_status mdhp_init_model_create(mdhp_init_model **model, int32_t M, int32_t hidden,
                                   int32_t max_batch, uint64_t seed);
void mdhp_init_model_destroy(mdhp_init_model *model);

/* Sizes: feature_dim (padded), out_dim = M + M^2, num_params (the flat FP32
 * parameter vector: layer l's W_l [out][in] row-major then b_l [out], each
 * block starting at a multiple of 256 floats). */
mdhp_status mdhp_init_model_info(const mdhp_init_model *model, int32_t *feature_dim,
                                 int32_t *out_dim, int64_t *num_params);

/* Copy the FP32 parameters (what = 0) or the gradient of the last
 * mdhp_init_train_step (what = 1) into dst [num_params] (device). */
mdhp_status mdhp_init_model_get(const mdhp_init_model *model, int32_t what, float *dst,
                                void *stream);

/* Replace the parameters from src [num_params] (device) and refresh the BF16
 * copy (checkpoint load). */
mdhp_status mdhp_init_model_set_params(mdhp_init_model *model, const float *src, void *stream);

/* Features of every window of `batch` (beta per batch->beta_mode). */
mdhp_status mdhp_init_features(const mdhp_batch *batch, const float *beta, void *features_bf16,
                               float *mu_cold, void *stream);

/* Network output y [B][out_dim] (FP32) for precomputed features. */
mdhp_status mdhp_init_forward(mdhp_init_model *model, const void *features_bf16, int32_t B,
                              float *out, void *stream);

/* Features -> network -> head: writes mu [B][M] and alpha [B][M][M]. */
mdhp_status mdhp_init_predict(mdhp_init_model *model, const mdhp_batch *batch, const float *beta,
                              float *mu, float *alpha, void *stream);

/* One AdamW step (b1 0.9, b2 0.999, eps 1e-8, decay on matrices only) on a
 * batch of B <= max_batch precomputed feature rows with targets mu* [B][M],
 * alpha* [B][M][M]; beta is [B] (beta_stride 1) or [B][M] (beta_stride M).
 * loss_out (device float, nullable) receives the batch loss before the step. */
mdhp_status mdhp_init_train_step(mdhp_init_model *model, const void *features_bf16,
                                 const float *mu_cold, const float *beta, int32_t beta_stride,
                                 const float *mu_target, const float *alpha_target, int32_t B,
                                 float lr, float weight_decay, float *loss_out, void *stream);

/* The training step in two halves, for data-parallel training over several
 * processes: mdhp_init_backward computes the loss and its gradient (into the
 * model's gradient buffer, readable with mdhp_init_model_get(what = 1)) for
 * this process's B windows; the caller averages the buffers over processes
 * (an all-reduce of num_params floats) and writes the mean back with
 * mdhp_init_set_grads; mdhp_init_apply then takes the AdamW step.
 * mdhp_init_train_step = backward + apply. */
mdhp_status mdhp_init_backward(mdhp_init_model *model, const void *features_bf16,
                               const float *mu_cold, const float *beta, int32_t beta_stride,
                               const float *mu_target, const float *alpha_target, int32_t B,
                               float *loss_out, void *stream);
mdhp_status mdhp_init_set_grads(mdhp_init_model *model, const float *src, void *stream);
mdhp_status mdhp_init_apply(mdhp_init_model *model, float lr, float weight_decay, void *stream);

/* Engine of the model's matrix products: 0 (default) the tensor-core GEMM
 * of mdhp_gemm_bf16 (tcgen05) wherever its operand layouts apply, else the
 * warp-level MMA kernel; 1 the warp-level MMA kernel (mma.sync) for every
 * product.  Errors: engine outside 0..1 (MDHP_E_ARG). */
mdhp_status mdhp_init_model_set_gemm(mdhp_init_model *model, int32_t engine);

/*
 * BF16 matrix product with FP32 accumulation, the initializer's layer GEMM
 * (an addition of this library; the paper has no initializer):
 *   C[m][n] = sum_k A(m,k) B(k,n) (+ bias[n], then ReLU if relu)      accumulate = 0
 *   C[m][n] += sum_k A(m,k) B(k,n)                                    accumulate = 1
 * A(m,k) = A[m*lda + k] (a_mn = 0, K contiguous) or A[k*lda + m] (a_mn = 1);
 * B(k,n) = B[n*ldb + k] (b_mn = 0, K contiguous) or B[k*ldb + n] (b_mn = 1);
 * all device pointers, BF16 operands, row-major outputs with pitch ldc: C
 * (FP32, nullable when accumulate = 0 and C_bf16 is given) and C_bf16 (BF16
 * copy of the result, nullable; ignored when accumulate = 1).
 * engine 0: fifth-generation tensor cores (tcgen05.mma, accumulators in tensor
 * memory; 128 x up-to-256 tiles, K split over CTAs when the tiles alone do not
 * fill the GPU, in which case C is required and holds the partial sums); with
 * both operands K-contiguous the tiles are loaded by the tensor-memory
 * accelerator (cp.async.bulk.tensor, 128-byte swizzle), otherwise by 16-byte
 * copies from every thread.  It needs 16-byte aligned A and B, lda and ldb
 * multiples of 8, K a multiple of 8 and, for an M/N-contiguous operand, M
 * (resp. N) a multiple of 8; other shapes return MDHP_E_UNSUPPORTED.
 * engine 1: warp-level MMA (mma.sync) on 64 x 64 tiles, any layout.  engine
 * 2: as 0 with the 16-byte copies for every layout (for comparison).
 * Asynchronous on `stream`.  Errors: NULL operands, sizes < 1, engine
 * outside 0..2 (MDHP_E_ARG).
 */
mdhp_status mdhp_gemm_bf16(const void *A, int64_t lda, int32_t a_mn, const void *B, int64_t ldb,
                           int32_t b_mn, int32_t M, int32_t N, int32_t K, const float *bias,
                           int32_t relu, float *C, void *C_bf16, int64_t ldc, int32_t accumulate,
                           int32_t engine, void *stream);

/* Synchronises the device and reports (then clears) the number of
 * tensor-core GEMM CTAs whose bounded waits gave up since the last call
 * (their tiles were not written). */
mdhp_status mdhp_gemm_check(int32_t *timeouts);

/* Attach a trained model to a plan: mdhp_fit_batch with opts->init == 2 then
 * predicts the starting point with it (the plan does not own the model). */
mdhp_status mdhp_plan_set_init_model(mdhp_plan *plan, mdhp_init_model *model);

/* Kernel family used by mdhp_fit_batch for fixed beta:
 *   MDHP_PATH_AUTO (0)      decoupled features when the plan has scratch for
 *                           them (M <= 32 and a stated max_events_per_window),
 *                           else the event recursion;
 *   MDHP_PATH_RECURSION (1) always re-run the event recursion each iteration.
 * Both compute the same quantities; the choice only affects speed. */
#define MDHP_PATH_AUTO 0
#define MDHP_PATH_RECURSION 1
mdhp_status mdhp_plan_set_path(mdhp_plan *plan, int32_t path);

/* Streaming of the decoupled kernels' features (fixed beta, windows longer
 * than the shared-memory class): the features of each window are re-read
 * every iteration from the plan's device scratch.  With stages > 0 they pass
 * through a ring of `stages` shared-memory buffers of `steps_per_stage` steps
 * each (a step is one feature row per thread), filled by bulk asynchronous
 * copies that run up to `stages` buffers ahead, across iterations; stages = 0
 * reads them through L1 with a one-step register prefetch.  stages 0..8,
 * steps_per_stage 1..16.  Default 0 stages (register prefetch measured
 * faster on the 4,096-window M=16 and M=32 workloads); a ring that does not
 * fit the block's shared memory falls back to stages = 0 for that launch.
 * Results do not depend on the choice. */
mdhp_status mdhp_plan_set_pipeline(mdhp_plan *plan, int32_t steps_per_stage, int32_t stages);
mdhp_status mdhp_plan_get_pipeline(const mdhp_plan *plan, int32_t *steps_per_stage,
                                   int32_t *stages);

/* Feature store of the decoupled kernels' streamed windows (Sec. IV-B.3
 * Stage 1, "Decoupling": the beta-only features are computed once per fit
 * and read at every iteration).  Applies to the single-launch shapes without
 * a feature ring (mdhp_plan_set_pipeline stages = 0) at template width 32
 * (M 17..32) with 256 threads per window (store 3: its own 384); other
 * shapes ignore it.
 *   store = 0 (default): every feature step is re-read from the plan's
 *             scratch at every iteration.
 *   store = 1: the first steps of every thread (one 32-float row per step)
 *             stay in the SM's tensor memory, 512 columns per SM shared
 *             evenly by the CTAs resident on it (8 steps per thread for the
 *             one 256-thread CTA per SM); the kernel
 *             allocates the columns when its CTA starts and frees them before
 *             it exits (a CTA waits for its columns while another kernel on
 *             the same SM holds them).
 *   store = 2: as 1, and the next steps stay in the shared memory the
 *             kernel's other data leave at its occupancy.
 *   store = 3: as 2, with 384 threads per window (12 warps, 168 registers:
 *             more loads in flight and fewer parameters per thread in the
 *             update; 5 steps per thread in tensor memory).
 * Only the remaining steps are re-read from the scratch.  Results do not
 * depend on the choice beyond rounding: stores 1 and 2 change only the order
 * of the per-thread log-intensity sums; store 3 partitions the features over
 * more threads.  MDHP_E_ARG for store outside {0, 1, 2, 3}. */
mdhp_status mdhp_plan_set_feature_store(mdhp_plan *plan, int32_t store);
/* The setting above, or -1 for a NULL plan. */
int32_t mdhp_plan_get_feature_store(const mdhp_plan *plan);

/* Streamed events of the event recursion (windows without a stated bound, or
 * longer than the staging cutoff; beta learned, or MDHP_PATH_RECURSION):
 * enable = 1 delivers each chunk's events to the recursion through a ring of
 * two shared-memory stages of 128 events per chunk, filled by bulk
 * asynchronous copies (cp.async.bulk, CTA-local) running a stage ahead, with
 * bounded waits; enable = 0 (default) reads them from global memory through
 * the read-only cache.  The ring is used
 * when the batch's t and id arrays are 16-byte aligned and there are no
 * per-event weights; otherwise, or when it does not fit the block's shared
 * memory, events are read from global memory.  Results do not depend on it
 * beyond the run-to-run rounding of learned-beta fits. */
mdhp_status mdhp_plan_set_event_ring(mdhp_plan *plan, int32_t enable);

/* Bound of a consumer's wait on a bulk-copy ring (the feature ring of
 * mdhp_plan_set_pipeline and the event ring of mdhp_plan_set_event_ring):
 * polls = 0 (default) waits up to 2^22 suspending polls, far beyond any
 * copy's latency; polls > 0 gives up after that many non-blocking tests.
 * A feature-ring wait that gives up reports the window as MDHP_E_TIMEOUT
 * (loglik NaN, parameters not written back); an event-ring wait that gives
 * up switches that CTA's remaining chunks to global-memory reads (same
 * results).  Either way the copies already in flight are waited out with the
 * full bound before the shared memory is used again, and a CTA whose drain
 * also gives up reports its later windows as MDHP_E_TIMEOUT without touching
 * the ring.  Small bounds exist to exercise these paths; errors: polls < 0
 * (MDHP_E_ARG). */
mdhp_status mdhp_plan_set_wait_limit(mdhp_plan *plan, int32_t polls);

/* Split of the decoupled kernels' streamed windows over two concurrent
 * launches that share one length-sorted queue from its two ends: the longest
 * windows are taken from the front by CTAs of long_threads threads
 * (long_ctas_per_sm per SM), the shortest from the back by CTAs of the plan's
 * threads per window, as many per SM as the rest of the SM holds; the two
 * meet in the middle, so neither needs a split point.  Fewer, wider CTAs on
 * the long windows keep fewer windows' features in flight (they then stay in
 * L2).  Used when the threads per window differ from long_threads and no
 * shared-memory feature class is set.  Default: enabled, 256 threads, 1 per
 * SM.  long_threads 64, 128 or 256; long_ctas_per_sm 1..8.  Results do not
 * depend on the split beyond rounding: each window is fitted by one CTA
 * either way, with the summation order of its block size, and which of the
 * two launches takes a window near the meeting point depends on timing.  In
 * a CUDA graph the two launches are sibling nodes with no order between
 * them; measured on GB300 (65,536 windows, M = 32), a graph replay of a
 * split fit ran markedly slower than the same call issued on streams, so
 * capture a plan with the split disabled. */
mdhp_status mdhp_plan_set_split(mdhp_plan *plan, int32_t enable, int32_t long_threads,
                                int32_t long_ctas_per_sm);
mdhp_status mdhp_plan_get_split(const mdhp_plan *plan, int32_t *enable, int32_t *long_threads,
                                int32_t *long_ctas_per_sm);

/*
 * Batched fit without a plan and without allocating device memory.  (An
 * addition of this library; the paper has no counterpart.)
 *
 * For callers that cannot call cudaMalloc: processes whose device memory is
 * owned by another framework's pooling allocator, deployments that forbid
 * allocation after start-up (a detector fitting every incoming window in a
 * vehicle, say), or threads that must not risk the implicit synchronisation
 * of an allocation.  It runs the same iteration as mdhp_fit_batch (the event
 * recursion kernels, windows taken longest first by length bucket) and
 * returns the same results within rounding, but keeps its work queue and
 * window order in a fixed device array compiled into the library.
 *   - B is limited to MDHP_NOALLOC_MAX_WINDOWS; larger batches get MDHP_E_ARG
 *     (split them).  opts->init must be 0 or 1 (no learned initializer).
 *   - Arguments and outputs as for mdhp_fit_batch; batch->max_events, when
 *     known and small enough, stages windows in shared memory.
 *   - The array (about 256 KB) is held by every GPU that loads the library
 *     until the process exits.  The first call on each device looks up its
 *     address (cudaGetSymbolAddress with that device current); make that first
 *     call before any stream capture.
 *   - All calls share the array: calls that overlap on the GPU (different
 *     streams or host threads on one device) race and must be serialised by
 *     the caller.  Each call clears what it needs before use.
 */
#define MDHP_NOALLOC_MAX_WINDOWS 65536
mdhp_status mdhp_fit_batch_noalloc(const mdhp_batch *batch, const mdhp_fit_opts *opts, float *mu,
                                   float *alpha, float *beta, double *loglik, int32_t *iters,
                                   int32_t *win_status, void *stream);

/*
 * Bulk simulation of windows of the exponential-kernel MDHP (the intensity of
 * Sec. II, with beta scalar or per source) by Ogata's thinning (Ogata 1981)
 * on the GPU, one thread per window in FP64.  Produces training windows for
 * the learned initializer and test data; an addition of this library (the
 * paper's windows are recorded traffic).
 *   M, beta_mode   1..64; MDHP_BETA_SCALAR or MDHP_BETA_PER_SOURCE (matrix:
 *                  MDHP_E_UNSUPPORTED).
 *   mu       double[B][M]     baseline rates (>= 0, finite)
 *   alpha    double[B][M][M]  row = target, column = source (>= 0, finite)
 *   beta     double[B][nb]    decays (> 0, finite), nb = 1 or M
 *   offsets  int64[B+1]       CSR output layout; window b gets exactly
 *                             N_b = offsets[b+1] - offsets[b] events
 *   order    int32[B] or NULL a permutation of 0..B-1: thread r simulates
 *                             window order[r] (longest first keeps a warp's
 *                             lanes busy for similar times); NULL = identity
 *   seed, stream_id, first_window
 *                             window b draws from the SplitMix64 counter
 *                             stream keyed by (seed, stream_id, first_window + b)
 *                             (Steele, Lea, Flood 2014), so its events do not
 *                             depend on the launch or on the other windows
 *   t        float[offsets[B]]  out: event times (seconds from window start,
 *                             non-decreasing; FP64 simulation rounded to float)
 *   id       int16[offsets[B]]  out: event types
 *   T_span   float[B]         out: the time of the (N_b + 1)-th accepted point,
 *                             which closes the window (never below its last event)
 *   win_status int32[B]       out: MDHP_OK, MDHP_E_ARG (bad parameters or
 *                             offsets; nothing written but T_span = 0) or
 *                             MDHP_E_SIM_STALLED (events written so far kept)
 * The same (seed, stream_id, window index) gives the events of the CPU
 * generator with the same definition, up to the rounding of exp/log1p and of
 * the sums.  Asynchronous on `stream`; no allocation.
 */
mdhp_status mdhp_simulate(int32_t M, int32_t beta_mode, int32_t B, const double *mu,
                          const double *alpha, const double *beta, const int64_t *offsets,
                          const int32_t *order, uint64_t seed, uint64_t stream_id,
                          uint64_t first_window, float *t, int16_t *id, float *T_span,
                          int32_t *win_status, void *stream);

/*
 * MDHP-LSTM cell (the paper's MDHP-LSTM equation, Sec. "MDHP-LSTM"): an LSTM
 * whose cell update is multiplied by a per-sequence Hawkes gate built from a
 * window's fitted MDHP parameters,
 *   hks = tanh(A vec(alpha) - Bm (beta T_span) + C mu)          [H]
 *   i, f, o = sigmoid(W_{i,f,o} x_t + U_{i,f,o} h_{t-1} + b_{i,f,o})
 *   g = tanh(W_c x_t + U_c h_{t-1} + b_c)
 *   c_t = hks * (f * c_{t-1} + i * g),  h_t = o * tanh(c_t),  y_t = Wy h_t
 * with h_{-1} = c_{-1} = 0 (step t consumes x_t and emits y_t: the paper
 * writes x^{t-1} and Wy h^{t-1}).  FP32, device pointers, row-major:
 *   x [B][L][D]; mu [B][M]; alpha [B][M][M]; beta [B][nb] (nb = 1 or M);
 *   T_span [B]; W [4H][D], U [4H][H], b [4H] (gate rows i, f, g, o);
 *   A [H][M*M], Bm [H][nb], C [H][M]; Wy [O][H].
 * Forward outputs (all written): y [B][L][O]; and for the backward pass
 * h_seq, c_seq [B][L][H], gates [B][L][4H] (activations), hks [B][H].
 * Backward: gradients of sum(y * dy) with respect to x, every weight and the
 * MDHP inputs (mu, alpha, beta); dW, dU, db, dA, dBm, dC, dWy are
 * overwritten; dz_work [B][L][4H] and dpre_work [B][H] are scratch.
 * Limits: H 1..256, D <= 3H, O <= 4H, M 1..64, L >= 1; MDHP_E_ARG otherwise.
 * Both calls are asynchronous on `stream` and allocate nothing.  Execution:
 * one CTA carries S in {1, 4, 8, 16} sequences through all L steps, S chosen
 * from the batch size and the kernels' occupancy (environment variable
 * MDHP_LSTM_SEQ_PER_CTA = 1, 4, 8 or 16 forces a value that can run).  For
 * S > 1 the gate activations use the fast exponential and division
 * (about 1e-6 relative for the sigmoid, 1e-7 absolute for tanh).
 */
typedef struct {
  int32_t B, L, D, H, M, nb, O;
} mdhp_lstm_dims;

mdhp_status mdhp_lstm_forward(const mdhp_lstm_dims *dims, const float *x, const float *mu,
                              const float *alpha, const float *beta, const float *T_span,
                              const float *W, const float *U, const float *b, const float *A,
                              const float *Bm, const float *C, const float *Wy, float *y,
                              float *h_seq, float *c_seq, float *gates, float *hks, void *stream);
mdhp_status mdhp_lstm_backward(const mdhp_lstm_dims *dims, const float *x, const float *mu,
                               const float *alpha, const float *beta, const float *T_span,
                               const float *W, const float *U, const float *A, const float *Bm,
                               const float *C, const float *Wy, const float *h_seq,
                               const float *c_seq, const float *gates, const float *hks,
                               const float *dy, float *dz_work, float *dpre_work, float *dx,
                               float *dW, float *dU, float *db, float *dA, float *dBm, float *dC,
                               float *dWy, float *dmu, float *dalpha, float *dbeta, void *stream);

/*
 * Throughput probe of one arithmetic pipe of the current GPU, for rooflines
 * (an addition of this library; the paper has no counterpart).  Launches a
 * kernel that fills every SM to its thread limit with independent dependency
 * chains of one operation, times it with CUDA events on `stream` (best of
 * three runs after a warm-up run), synchronises the stream and returns
 * operations per second in *ops_per_s (and the best time in *ms, nullable):
 *   what 0  FP32 fused multiply-add, counted as 2 floating-point operations
 *   what 1  ex2.approx (MUFU)     what 2  lg2.approx (MUFU)     what 3  rcp.approx (MUFU)
 * Allocates nothing; runs for a few tens of milliseconds.  The clock the GPU
 * ran at is not controlled: sample it beside the call to compare rates.
 */
mdhp_status mdhp_probe_peak(int32_t what, double *ops_per_s, float *ms, void *stream);

/* Text of the last error in this thread (static storage). */
const char *mdhp_last_error(void);

/* Library version, major * 10000 + minor * 100 + patch. */
int32_t mdhp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MDHP_H_ */
