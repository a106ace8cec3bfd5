// C ABI of the MDHP-GDS library (declared in include/mdhp.h).
#include <cub/device/device_radix_sort.cuh>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include <unistd.h>

#include "mdhp.h"
#include "mdhp_dispatch.h"

namespace mdhp {

static thread_local std::string g_last_error;

static mdhp_status fail(mdhp_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

// Lets other translation units of the library report through mdhp_last_error().
void record_error(const char *msg) { g_last_error = msg; }

static mdhp_status cuda_check(const char *what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(MDHP_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return MDHP_OK;
}

// Template capacity for a runtime M.
static int cap_of(int M) {
  if (M <= 4) return 4;
  if (M <= 8) return 8;
  if (M <= 16) return 16;
  if (M <= 32) return 32;
  return 64;
}

LlgFn get_llg(int M, int SPL, int BM, bool learn, bool stage) {
  switch (M) {
    case 4: return get_llg_m4(SPL, BM, learn, stage);
    case 8: return get_llg_m8(SPL, BM, learn, stage);
    case 16: return get_llg_m16(SPL, BM, learn, stage);
    case 32: return get_llg_m32(SPL, BM, learn, stage);
    case 64: return get_llg_m64(SPL, BM, learn, stage);
  }
  return nullptr;
}
FitFn get_fit(int M, int SPL, int BM, bool learn, bool stage) {
  switch (M) {
    case 4: return get_fit_m4(SPL, BM, learn, stage);
    case 8: return get_fit_m8(SPL, BM, learn, stage);
    case 16: return get_fit_m16(SPL, BM, learn, stage);
    case 32: return get_fit_m32(SPL, BM, learn, stage);
    case 64: return get_fit_m64(SPL, BM, learn, stage);
  }
  return nullptr;
}
FitFn get_fitx(int M, int BM, int xm, int nt) {
  switch (M) {
    case 4: return get_fitx_m4(BM, xm, nt);
    case 8: return get_fitx_m8(BM, xm, nt);
    case 16: return get_fitx_m16(BM, xm, nt);
    case 32: return get_fitx_m32(BM, xm, nt);
    case 64: return get_fitx_m64(BM, xm, nt);
  }
  return nullptr;
}
WgFn get_wg(int M, int BM) {
  switch (M) {
    case 4: return get_wg_m4(BM);
    case 8: return get_wg_m8(BM);
    case 16: return get_wg_m16(BM);
    case 32: return get_wg_m32(BM);
    case 64: return get_wg_m64(BM);
  }
  return nullptr;
}

Shape default_shape(int Mt) {
  switch (Mt) {
    case 4: return {128, 1, 16384};
    case 8: return {128, 2, 12288};
    case 16: return {128, 4, 8192};
    case 32: return {128, 8, 6144};
    default: return {256, 8, 8192};  // M = 64: 8 threads per chunk measured faster than 16 (learned beta, 50k-event windows)
  }
}

static bool use_priv(int Mt) { return Mt <= 32; }

static int max_dyn_smem() {
  static int v = -1;
  if (v < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  return v;
}

static int num_sms() {
  static int v = -1;
  if (v < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  }
  return v;
}

// the most threads per block a kernel was compiled for (its launch bound)
static int kernel_max_threads(const void *fn) {
  cudaFuncAttributes fa{};
  if (!fn || cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return fa.maxThreadsPerBlock;
}

// both recursion fit kernels (staged and streamed events) of this split take nt threads
static bool fit_takes(int Mt, int spl, int BM, bool learn, int nt) {
  const FitFn a = get_fit(Mt, spl, BM, learn, true), b = get_fit(Mt, spl, BM, learn, false);
  return a && b && kernel_max_threads((const void *)a) >= nt && kernel_max_threads((const void *)b) >= nt;
}

static mdhp_status prepare_kernel(const void *fn, int smem) {
  if (smem > 48 * 1024) {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
      return fail(MDHP_E_CUDA, "cudaFuncSetAttribute(%d bytes): %s", smem,
                  cudaGetErrorString(cudaGetLastError()));
  }
  return MDHP_OK;
}

static mdhp_status check_batch(const mdhp_batch *b, bool matrix_ok = false) {
  if (!b) return fail(MDHP_E_ARG, "batch is NULL");
  if (b->B < 0) return fail(MDHP_E_ARG, "B < 0");
  if (b->M < 1 || b->M > 64) return fail(MDHP_E_ARG, "M = %d outside 1..64", b->M);
  if (b->beta_mode == MDHP_BETA_MATRIX && !matrix_ok)
    return fail(MDHP_E_UNSUPPORTED, "matrix-shaped beta: only mdhp_fit_batch with a fixed beta");
  if (b->beta_mode != MDHP_BETA_SCALAR && b->beta_mode != MDHP_BETA_PER_SOURCE &&
      b->beta_mode != MDHP_BETA_MATRIX)
    return fail(MDHP_E_ARG, "beta_mode %d", b->beta_mode);
  if (b->n_events < 0) return fail(MDHP_E_ARG, "n_events < 0");
  if (b->n_events > 0 && (!b->t || !b->id)) return fail(MDHP_E_ARG, "t/id NULL");
  if (b->B > 0 && (!b->offsets || !b->T_span)) return fail(MDHP_E_ARG, "offsets/T_span NULL");
  if (b->max_events < 0) return fail(MDHP_E_ARG, "max_events < 0");
  return MDHP_OK;
}

}  // namespace mdhp

using namespace mdhp;

namespace mdhp {
// kernels one mdhp_init_predict call of B windows launches (mdhp_init.cu)
int init_predict_launches(const mdhp_init_model *model, int B);
}  // namespace mdhp

struct mdhp_plan {
  int M, Mt, beta_mode, max_windows;
  int64_t max_events;
  Shape shape;
  int *keys = nullptr, *keys_sorted = nullptr, *idx = nullptr, *order = nullptr;
  int *ctl = nullptr;  // [0] queue long, [1] queue short, [2..3] range long, [4..5] range short,
                       // [6..8] two-ended queue (claimed, front, back)
  void *sort_tmp = nullptr;
  size_t sort_tmp_bytes = 0;
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
  int timing = 0, timed = 0;
  // decoupled fixed-beta fit: per-CTA feature scratch for windows of up to xcap events
  float4 *xbuf = nullptr;
  int xcap = 0, xgrid = 0, xnt = 128;  // xnt: threads per window of the decoupled kernels
  int xres = 0, xrgrid = 0;  // windows of <= xres events keep their features in shared memory
  int xres_max = 0;          // largest shared-memory class the device allows
  int use_x = 1;  // 0 forces the recursion kernels (for tests and comparisons)
  // streamed features of the decoupled kernels: ring of pipe_stages shared-memory
  // buffers of pipe_steps steps filled by bulk copies (0 stages: register prefetch)
  int pipe_steps = 0, pipe_stages = 0;  // measured: register prefetch is faster on the bench workloads
  // two concurrent launches over one length-sorted queue: the longest windows
  // from the front with xnt_long threads (xcta_long CTAs per SM), the
  // shortest from the back with xnt threads, as many CTAs per SM as the rest
  // of the register file holds; fewer windows in flight keeps their features
  // in L2.  0 = one launch of xnt threads.
  int xdual = 1, xnt_long = 256, xcta_long = 1;
  // recursion fit: streamed events reach pass 2 through the bulk-copy ring
  // (off by default: the recursion spends ~2,000 instructions per event on
  // 6 bytes of event data, and the ring's shared-memory reads measured slower
  // than cached global loads)
  int ev_ring = 0;
  // decoupled fit, single launch of streamed features: the first feature
  // steps of every thread live in tensor memory (512 columns per SM shared
  // by the resident CTAs) instead of being re-read from the scratch at
  // every iteration
  int xtmem = 0;
  uint32_t wait_polls = 0;           // consumer waits on the bulk-copy rings (0: default bound)
  mdhp_init_model *model = nullptr;  // learned initializer (not owned)
  std::string cache;                 // autotune cache file ("" = none)
  int launches = 0;                  // kernel launches of the last mdhp_fit_batch
  // recursion fit: theta_{k-1} per resident CTA in device memory (frees
  // shared memory for a second CTA per SM at M = 64)
  float *pbuf = nullptr;
  int pslots = 0, pstride = 0;
};

// --- autotuner: cache of tuned launch shapes ---------------------------------
//
// The cache is a small JSON file, one entry per line:
//   {"format": "mdhp-autotune-1", "entries": [
//   {"key": "<device>|sm<cc>|M<M>|mode<m>|W<max_windows>|E<max_events>|<path>",
//    "threads_per_window": 64, "threads_per_chunk": 0, "smem_cutoff_events": 0,
//    "pipe_steps": 0, "pipe_stages": 0, "split": 1, "split_threads": 256, "split_ctas": 1,
//    "ms": 10.3},
//   ...]}
// keyed by the device and the plan's creation arguments; <path> is "decoupled"
// (fixed-beta features kernels: threads per window and the shared-memory
// class) or "recursion" (threads per window, threads per chunk, staging cutoff).
namespace mdhp {
namespace {

std::string tune_key(const mdhp_plan *p, int path) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, dev);
  std::string name = prop.name;
  for (char &c : name)
    if (c == '"' || c == '\\' || c == '|' || (unsigned char)c < 32) c = '_';
  char buf[512];
  snprintf(buf, sizeof(buf), "%s|sm%d%d|M%d|mode%d|W%d|E%lld|%s", name.c_str(), prop.major,
           prop.minor, p->M, p->beta_mode, p->max_windows, (long long)p->max_events,
           path == 0 ? "decoupled" : "recursion");
  return buf;
}

bool read_text(const std::string &path, std::string &out) {
  FILE *f = fopen(path.c_str(), "rb");
  if (!f) return false;
  char buf[4096];
  size_t n;
  out.clear();
  while ((n = fread(buf, 1, sizeof(buf), f)) > 0) out.append(buf, n);
  fclose(f);
  return true;
}

// (key, entry text) for every entry of a cache file
std::vector<std::pair<std::string, std::string>> cache_entries(const std::string &text) {
  std::vector<std::pair<std::string, std::string>> v;
  const std::string open = "{\"key\": \"";
  size_t pos = 0;
  while ((pos = text.find(open, pos)) != std::string::npos) {
    const size_t ks = pos + open.size();
    const size_t ke = text.find('"', ks);
    if (ke == std::string::npos) break;
    const size_t le = text.find('}', ke);
    if (le == std::string::npos) break;
    v.emplace_back(text.substr(ks, ke - ks), text.substr(pos, le - pos + 1));
    pos = le + 1;
  }
  return v;
}

int field_int(const std::string &entry, const char *name, int dflt) {
  const std::string pat = std::string("\"") + name + "\": ";
  const size_t p = entry.find(pat);
  if (p == std::string::npos) return dflt;
  return (int)strtol(entry.c_str() + p + pat.size(), nullptr, 10);
}

// largest events-per-window class of the decoupled kernels that fits the
// shared memory of one CTA of nt threads (0 if none)
int xres_fit(const mdhp_plan *p, int nt, bool adam) {
  const int fixed = make_carve_x(p->Mt, nt, 0, adam, 0, 0, p->beta_mode == 2).total;
  int fit = ((max_dyn_smem() - 1024 - fixed) / (p->Mt * 4)) / 32 * 32;
  if (fit > p->xcap) fit = p->xcap / 32 * 32;
  return fit >= 64 ? fit : 0;
}

// largest staging capacity of the recursion kernels for (nt, spl) (0 if none)
int stage_fit(const mdhp_plan *p, int nt, int spl, bool weights, bool learn, bool adam) {
  int lo = 0, hi = 1 << 20;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (make_carve(p->Mt, nt, spl, mid, weights, learn, adam, true, use_priv(p->Mt), false).total <=
        max_dyn_smem())
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo / 32 * 32;
}

bool apply_decoupled(mdhp_plan *p, int nt, int xres) {
  if (nt < 64 || nt > 256 || (nt & (nt - 1)) || nt < p->Mt) return false;
  if (xres < 0 || (xres > 0 && (xres < 64 || xres > xres_fit(p, nt, false)))) return false;
  p->xnt = nt;
  p->xres = xres;
  return true;
}

bool apply_recursion(mdhp_plan *p, int nt, int spl, int cutoff) {
  if (nt < 32 || nt > 256 || nt % 32 || nt < p->Mt || spl < 1 || nt % spl || cutoff < 0) return false;
  if (!get_fit(p->Mt, spl, p->beta_mode, false, true)) return false;
  p->shape = Shape{nt, spl, cutoff};
  return true;
}

void tune_load(mdhp_plan *p) {
  std::string text;
  if (!read_text(p->cache, text)) return;
  const auto v = cache_entries(text);
  for (int path = 0; path < 2; ++path) {
    const std::string key = tune_key(p, path);
    for (const auto &e : v) {
      if (e.first != key) continue;
      const int nt = field_int(e.second, "threads_per_window", 0);
      const int spl = field_int(e.second, "threads_per_chunk", 0);
      const int cut = field_int(e.second, "smem_cutoff_events", -1);
      if (path == 0 && p->xbuf && apply_decoupled(p, nt, cut)) {
        const int pd = field_int(e.second, "pipe_stages", p->pipe_stages);
        const int ps = field_int(e.second, "pipe_steps", p->pipe_steps);
        if (pd == 0 || (pd > 0 && pd <= 8 && ps >= 1 && ps <= 16)) {
          p->pipe_stages = pd;
          p->pipe_steps = pd > 0 ? ps : 0;
        }
        const int du = field_int(e.second, "split", p->xdual);
        const int ntl = field_int(e.second, "split_threads", p->xnt_long);
        const int cl = field_int(e.second, "split_ctas", p->xcta_long);
        if ((ntl == 64 || ntl == 128 || ntl == 256) && cl >= 1 && cl <= 8) {
          p->xdual = du ? 1 : 0;
          p->xnt_long = ntl;
          p->xcta_long = cl;
        }
        const int fs = field_int(e.second, "feature_store", p->xtmem);
        if (fs >= 0 && fs <= 3) p->xtmem = fs;
      }
      if (path == 1) apply_recursion(p, nt, spl, cut);
    }
  }
  cudaGetLastError();
}

struct TuneChoice {
  int nt, spl, cut, ps, pd, dual, ntl, cl;
  int tm = 0;  // decoupled: feature steps in tensor memory (mdhp_plan_set_feature_store)
};

bool tune_store(const mdhp_plan *p, int path, const TuneChoice &c, float ms) {
  if (p->cache.empty()) return true;
  std::string text;
  read_text(p->cache, text);
  auto v = cache_entries(text);
  const std::string key = tune_key(p, path);
  char line[768];
  snprintf(line, sizeof(line),
           "{\"key\": \"%s\", \"threads_per_window\": %d, \"threads_per_chunk\": %d, "
           "\"smem_cutoff_events\": %d, \"pipe_steps\": %d, \"pipe_stages\": %d, "
           "\"split\": %d, \"split_threads\": %d, \"split_ctas\": %d, \"feature_store\": %d, "
           "\"ms\": %.4f}",
           key.c_str(), c.nt, c.spl, c.cut, c.ps, c.pd, c.dual, c.ntl, c.cl, c.tm, ms);
  bool found = false;
  for (auto &e : v)
    if (e.first == key) {
      e.second = line;
      found = true;
    }
  if (!found) v.emplace_back(key, line);
  const std::string tmp = p->cache + ".tmp" + std::to_string((long)getpid());
  FILE *f = fopen(tmp.c_str(), "wb");
  if (!f) return false;
  fprintf(f, "{\"format\": \"mdhp-autotune-1\", \"entries\": [\n");
  for (size_t i = 0; i < v.size(); ++i) fprintf(f, "%s%s\n", v[i].second.c_str(), i + 1 < v.size() ? "," : "");
  fprintf(f, "]}\n");
  const bool ok = fclose(f) == 0;
  return ok && rename(tmp.c_str(), p->cache.c_str()) == 0;
}

// The two-launch decoupled fit (plan field xdual): both launches share the
// sorted range ctl[2..3] through the two-ended queue ctl[6..8].  *done is
// false (and nothing is launched) when the shapes do not fit together.
mdhp_status launch_dual(mdhp_plan *p, const FitArgs &ax, bool adam, cudaStream_t st, bool *done) {
  *done = false;
  const int ntL = p->xnt_long, ntS = p->xnt;
  FitFn fL = get_fitx(p->Mt, p->beta_mode, XM_GLOBAL, ntL);
  FitFn fS = get_fitx(p->Mt, p->beta_mode, XM_GLOBAL, ntS);
  if (!fL || !fS || ntL < p->Mt) return MDHP_OK;
  FitArgs aL = ax, aS = ax;
  aL.range = aS.range = p->ctl + 2;
  aL.dq = aS.dq = p->ctl + 6;
  aL.ev_cap = aS.ev_cap = p->xcap;
  aL.pipe_stages = aS.pipe_stages = 0;
  aL.qdir = 1;
  aS.qdir = 2;
  aL.carve = make_carve_x(p->Mt, ntL, 0, adam, 0, 0, p->beta_mode == 2);
  aS.carve = make_carve_x(p->Mt, ntS, 0, adam, 0, 0, p->beta_mode == 2);
  mdhp_status s;
  if ((s = prepare_kernel((const void *)fL, aL.carve.total)) != MDHP_OK) return s;
  if ((s = prepare_kernel((const void *)fS, aS.carve.total)) != MDHP_OK) return s;
  // CTAs per SM: the long class as configured (at most its occupancy); the
  // short class what the long one leaves of the registers, shared memory and
  // thread slots
  int dev = 0, regs_sm = 0, smem_sm = 0, thr_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  cudaFuncAttributes faL{}, faS{};
  if (cudaFuncGetAttributes(&faL, fL) != cudaSuccess || cudaFuncGetAttributes(&faS, fS) != cudaSuccess) {
    cudaGetLastError();
    return MDHP_OK;
  }
  int occL = 0, occS = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occL, fL, ntL, aL.carve.total);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occS, fS, ntS, aS.carve.total);
  const int cL = std::min(p->xcta_long, occL);
  if (cL < 1) return MDHP_OK;
  const int rL = (faL.numRegs + 7) / 8 * 8, rS = (faS.numRegs + 7) / 8 * 8;
  int cS = (regs_sm - cL * ntL * rL) / (ntS * rS);
  cS = std::min(cS, (smem_sm - cL * (aL.carve.total + 1024)) / (aS.carve.total + 1024));
  cS = std::min(cS, (thr_sm - cL * ntL) / ntS);
  cS = std::min(cS, occS);
  if (cS < 1) return MDHP_OK;
  const int gL = num_sms() * cL;
  int gS = num_sms() * cS;
  if (gL + gS > p->xgrid) gS = p->xgrid - gL;
  if (gS < 1) return MDHP_OK;
  aL.slot_base = 0;
  aS.slot_base = gL;
  cudaEventRecord(p->ev_fork, st);
  cudaStreamWaitEvent(p->side, p->ev_fork, 0);
  fL<<<gL, ntL, aL.carve.total, p->side>>>(aL);
  if ((s = cuda_check("k_fit_x (long windows, front of the queue)")) != MDHP_OK) return s;
  cudaEventRecord(p->ev_join, p->side);
  fS<<<gS, ntS, aS.carve.total, st>>>(aS);
  p->launches += 2;
  if ((s = cuda_check("k_fit_x (short windows, back of the queue)")) != MDHP_OK) return s;
  cudaStreamWaitEvent(st, p->ev_join, 0);
  *done = true;
  return MDHP_OK;
}

}  // namespace
}  // namespace mdhp

extern "C" {

const char *mdhp_last_error(void) { return g_last_error.c_str(); }

int32_t mdhp_version(void) { return 100; }

void mdhp_fit_opts_default(mdhp_fit_opts *o) {
  if (!o) return;
  o->optimizer = 0;
  o->max_iters = 200;
  o->fit_beta = 0;
  o->patience = 3;
  o->lr = 1e-2f;
  o->mu_floor = 1e-10f;
  o->alpha_floor = 0.f;
  o->beta_floor = 1e-6f;
  o->adam_b1 = 0.9f;
  o->adam_b2 = 0.999f;
  o->adam_eps = 1e-8f;
  o->init = 1;
  o->tol = 0.0;
}

mdhp_status mdhp_loglik_grad(const mdhp_batch *batch, const float *mu, const float *alpha,
                             const float *beta, double *loglik, float *g_mu, float *g_alpha,
                             float *g_beta, float *g_weights, float *r_work, int32_t *win_status,
                             void *stream) {
  mdhp_status s = check_batch(batch);
  if (s != MDHP_OK) return s;
  const int B = batch->B, M = batch->M, BM = batch->beta_mode;
  if (B == 0) return MDHP_OK;
  if (!mu || !alpha || !beta || !loglik || !g_mu || !g_alpha || !win_status)
    return fail(MDHP_E_ARG, "NULL parameter/output pointer");
  if (g_weights && !r_work) return fail(MDHP_E_ARG, "g_weights requires r_work");
  const int Mt = cap_of(M);
  const Shape sh = default_shape(Mt);
  const bool learn = g_beta != nullptr;
  const bool stage = batch->max_events > 0 && batch->max_events <= sh.cutoff;
  LlgFn fn = get_llg(Mt, sh.spl, BM, learn, stage);
  if (!fn) return fail(MDHP_E_UNSUPPORTED, "no kernel for M=%d", M);
  const int NC = sh.nt / sh.spl;
  LlgArgs a{};
  a.offsets = batch->offsets; a.t = batch->t; a.id = batch->id; a.T = batch->T_span;
  a.w = batch->weights; a.mu = mu; a.alpha = alpha; a.beta = beta; a.loglik = loglik;
  a.g_mu = g_mu; a.g_alpha = g_alpha; a.g_beta = g_beta;
  a.r_out = g_weights ? r_work : nullptr;
  a.status = win_status; a.B = B; a.Mrt = M; a.NC = NC;
  a.ev_cap = stage ? batch->max_events : 0;
  a.carve = make_carve(Mt, sh.nt, sh.spl, a.ev_cap, batch->weights != nullptr, learn, false, false,
                       use_priv(Mt));
  if (a.carve.total > max_dyn_smem())
    return fail(MDHP_E_ARG, "shared memory %d > %d", a.carve.total, max_dyn_smem());
  if ((s = prepare_kernel((const void *)fn, a.carve.total)) != MDHP_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  fn<<<B, sh.nt, a.carve.total, st>>>(a);
  if ((s = cuda_check("k_loglik_grad")) != MDHP_OK) return s;
  if (g_weights) {
    WgFn wf = get_wg(Mt, BM);
    WgArgs w{};
    w.offsets = batch->offsets; w.t = batch->t; w.id = batch->id; w.T = batch->T_span;
    w.alpha = alpha; w.beta = beta; w.r = r_work; w.g_w = g_weights; w.status = win_status;
    w.Mrt = M;
    const int nt = 128 > Mt ? 128 : Mt;
    w.NC = nt;
    const int smem = (Mt * (Mt + 1) + 3 * Mt + 2 * (nt + 1) + nt * Mt) * 4;
    if (smem > max_dyn_smem()) return fail(MDHP_E_ARG, "weight-grad shared memory %d", smem);
    if ((s = prepare_kernel((const void *)wf, smem)) != MDHP_OK) return s;
    wf<<<B, nt, smem, st>>>(w);
    if ((s = cuda_check("k_weight_grad")) != MDHP_OK) return s;
  }
  return MDHP_OK;
}

// --- plans -----------------------------------------------------------------

__global__ void k_lengths(const int64_t *offsets, int B, int *keys, int *idx) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) {
    const int64_t n = offsets[b + 1] - offsets[b];
    keys[b] = n > 0x7ffffff0LL ? 0x7ffffff0 : (n < 0 ? 0 : (int)n);
    idx[b] = b;
  }
}

// Sorted keys (descending) -> number of windows longer than the cutoff;
// writes the two work ranges and clears the queue counters.  Without a
// streamed launch every window goes to the staged kernel, which reports
// MDHP_E_ARG for a window longer than its staging capacity.
__global__ void k_split(const int *keys_sorted, int B, int cutoff, int has_long, int *ctl) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int lo = 0, hi = has_long ? B : 0;  // first position with key <= cutoff
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (keys_sorted[mid] > cutoff) lo = mid + 1;
      else hi = mid;
    }
    ctl[0] = 0;
    ctl[1] = 0;
    ctl[2] = 0;
    ctl[3] = lo;
    ctl[4] = lo;
    ctl[5] = B;
    ctl[6] = 0;  // two-ended queue: claimed, taken from the front, taken from the back
    ctl[7] = 0;
    ctl[8] = 0;
  }
}

mdhp_status mdhp_plan_create(mdhp_plan **out, int32_t M, int32_t beta_mode, int32_t max_windows,
                             int64_t max_events_per_window, const char *autotune_cache) {
  if (!out) return fail(MDHP_E_ARG, "plan out-pointer NULL");
  *out = nullptr;
  if (M < 1 || M > 64) return fail(MDHP_E_ARG, "M = %d outside 1..64", M);
  if (beta_mode != 0 && beta_mode != 1 && beta_mode != 2)
    return fail(MDHP_E_ARG, "beta_mode %d", beta_mode);
  if (beta_mode == MDHP_BETA_MATRIX && (M > 32 || max_events_per_window <= 0))
    return fail(MDHP_E_UNSUPPORTED,
                "matrix-shaped beta needs M <= 32 and a stated max_events_per_window (decoupled kernels)");
  if (max_windows < 1) return fail(MDHP_E_ARG, "max_windows < 1");
  if (max_events_per_window < 0) return fail(MDHP_E_ARG, "max_events_per_window < 0");
  mdhp_plan *p = new mdhp_plan();
  p->M = M;
  p->Mt = cap_of(M);
  p->beta_mode = beta_mode;
  p->max_windows = max_windows;
  p->max_events = max_events_per_window;
  p->shape = default_shape(p->Mt);
  p->xnt = 64;  // measured best on the 4,096 x M=16 and M=32 workloads (64/128/256 swept)
  bool ok = true;
  ok &= cudaMalloc(&p->keys, sizeof(int) * max_windows) == cudaSuccess;
  ok &= cudaMalloc(&p->keys_sorted, sizeof(int) * max_windows) == cudaSuccess;
  ok &= cudaMalloc(&p->idx, sizeof(int) * max_windows) == cudaSuccess;
  ok &= cudaMalloc(&p->order, sizeof(int) * max_windows) == cudaSuccess;
  ok &= cudaMalloc(&p->ctl, sizeof(int) * 16) == cudaSuccess;
  // per-CTA device slot of the recursion fit: theta_{k-1}, the gradient
  // buffer and the two Adam moments, pstride / 4 floats each
  p->pstride = 4 * ((p->Mt + p->Mt * p->Mt + p->Mt + 63) / 64 * 64);
  p->pslots = num_sms() * 16;
  ok &= cudaMalloc(&p->pbuf, sizeof(float) * (size_t)p->pslots * p->pstride) == cudaSuccess;
  if (ok) {
    cub::DeviceRadixSort::SortPairsDescending(nullptr, p->sort_tmp_bytes, p->keys, p->keys_sorted,
                                              p->idx, p->order, max_windows);
    ok &= cudaMalloc(&p->sort_tmp, p->sort_tmp_bytes > 0 ? p->sort_tmp_bytes : 16) == cudaSuccess;
  }
  if (ok && p->Mt <= 32 && max_events_per_window > 0 && max_events_per_window < (1 << 26)) {
    // scratch slots for the largest resident grid over the supported block sizes
    int slots = 0;
    for (int nt = 64; nt <= 256; nt *= 2) {
      FitFn fx = get_fitx(p->Mt, beta_mode, XM_GLOBAL, nt);
      const Carve cx = make_carve_x(p->Mt, nt, 0, true, 0, 0, beta_mode == 2);
      int occ = 0;
      if (fx && prepare_kernel((const void *)fx, cx.total) == MDHP_OK &&
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fx, nt, cx.total) == cudaSuccess &&
          num_sms() * occ > slots)
        slots = num_sms() * occ;
    }
    if (slots > 0) {
      p->xgrid = slots;
      p->xcap = (int)max_events_per_window;
      // per slot (xcap + 2 * 384) rows: the step-major layout pads each
      // window to L * threads with L odd (see mdhp_fitx.cuh)
      const size_t bytes = (size_t)p->xgrid * (size_t)(p->Mt / 4) * (size_t)(p->xcap + 768) *
                           sizeof(float4);
      if (cudaMalloc(&p->xbuf, bytes) != cudaSuccess) {
        cudaGetLastError();
        p->xbuf = nullptr;  // the recursion kernels still work without it
        p->xcap = 0;
      }
    }
    // shared-memory class: two CTAs per SM for M <= 16, one for M = 32
    FitFn fr = get_fitx(p->Mt, beta_mode, XM_SHARED, p->xnt);
    const int fixed = make_carve_x(p->Mt, p->xnt, 0, true, 0, 0, beta_mode == 2).total;
    const int target = (p->Mt <= 16 ? max_dyn_smem() / 2 : max_dyn_smem()) - 1024;
    int cap = (target - fixed) / (p->Mt * 4);
    cap = cap / 32 * 32;
    if (p->xbuf && fr && cap >= 64) {
      if (cap > p->xcap) cap = p->xcap;
      const Carve cr = make_carve_x(p->Mt, p->xnt, cap, true, 0, 0, beta_mode == 2);
      int occr = 0;
      if (prepare_kernel((const void *)fr, cr.total) == MDHP_OK &&
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occr, fr, p->xnt, cr.total) == cudaSuccess &&
          occr > 0) {
        p->xres_max = cap;
        p->xrgrid = num_sms() * occr;
        // measured default: streaming every window's features through L1/L2
        // beats keeping the short windows' features in shared memory (which
        // takes the L1 capacity the streaming class relies on)
        p->xres = 0;
      }
    }
    cudaGetLastError();
  }
  ok &= cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking) == cudaSuccess;
  ok &= cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  ok &= cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) == cudaSuccess;
  ok &= cudaEventCreate(&p->ev_t0) == cudaSuccess;
  ok &= cudaEventCreate(&p->ev_t1) == cudaSuccess;
  if (!ok) {
    mdhp_plan_destroy(p);
    cudaGetLastError();
    return fail(MDHP_E_NOMEM, "plan allocation failed");
  }
  if (autotune_cache && autotune_cache[0]) {
    p->cache = autotune_cache;
    tune_load(p);
  }
  *out = p;
  return MDHP_OK;
}

void mdhp_plan_destroy(mdhp_plan *p) {
  if (!p) return;
  cudaFree(p->keys);
  cudaFree(p->keys_sorted);
  cudaFree(p->idx);
  cudaFree(p->order);
  cudaFree(p->ctl);
  cudaFree(p->pbuf);
  cudaFree(p->sort_tmp);
  cudaFree(p->xbuf);
  if (p->side) cudaStreamDestroy(p->side);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  if (p->ev_t0) cudaEventDestroy(p->ev_t0);
  if (p->ev_t1) cudaEventDestroy(p->ev_t1);
  delete p;
}

mdhp_status mdhp_plan_set_timing(mdhp_plan *p, int32_t enable) {
  if (!p) return fail(MDHP_E_ARG, "plan NULL");
  p->timing = enable ? 1 : 0;
  p->timed = 0;
  return MDHP_OK;
}

float mdhp_plan_last_fit_ms(mdhp_plan *p) {
  if (!p || !p->timed) return -1.f;
  if (cudaEventSynchronize(p->ev_t1) != cudaSuccess) return -1.f;
  float ms = -1.f;
  if (cudaEventElapsedTime(&ms, p->ev_t0, p->ev_t1) != cudaSuccess) return -1.f;
  return ms;
}

mdhp_status mdhp_plan_set_init_model(mdhp_plan *p, mdhp_init_model *model) {
  if (!p) return fail(MDHP_E_ARG, "plan NULL");
  p->model = model;
  return MDHP_OK;
}

mdhp_status mdhp_plan_set_path(mdhp_plan *p, int32_t path) {
  if (!p) return fail(MDHP_E_ARG, "plan NULL");
  if (path != MDHP_PATH_AUTO && path != MDHP_PATH_RECURSION) return fail(MDHP_E_ARG, "path %d", path);
  p->use_x = path == MDHP_PATH_AUTO ? 1 : 0;
  return MDHP_OK;
}

mdhp_status mdhp_plan_set_event_ring(mdhp_plan *p, int32_t enable) {
  if (!p) return fail(MDHP_E_ARG, "plan NULL");
  p->ev_ring = enable ? 1 : 0;
  return MDHP_OK;
}

mdhp_status mdhp_plan_set_wait_limit(mdhp_plan *p, int32_t polls) {
  if (!p) return fail(MDHP_E_ARG, "plan NULL");
  if (polls < 0) return fail(MDHP_E_ARG, "polls %d < 0", polls);
  p->wait_polls = (uint32_t)polls;
  return MDHP_OK;
}

mdhp_status mdhp_plan_set_pipeline(mdhp_plan *p, int32_t steps_per_stage, int32_t stages) {
  if (!p) return fail(MDHP_E_ARG, "plan NULL");
  if (stages < 0 || stages > 8) return fail(MDHP_E_ARG, "stages %d (0..8)", stages);
  if (stages > 0 && (steps_per_stage < 1 || steps_per_stage > 16))
    return fail(MDHP_E_ARG, "steps per stage %d (1..16)", steps_per_stage);
  p->pipe_stages = stages;
  p->pipe_steps = stages > 0 ? steps_per_stage : 0;
  return MDHP_OK;
}

mdhp_status mdhp_plan_set_feature_store(mdhp_plan *p, int32_t tmem) {
  if (!p) return fail(MDHP_E_ARG, "plan NULL");
  if (tmem < 0 || tmem > 3) return fail(MDHP_E_ARG, "feature store %d (0..3)", tmem);
  p->xtmem = tmem;
  return MDHP_OK;
}

int32_t mdhp_plan_get_feature_store(const mdhp_plan *p) { return p ? p->xtmem : -1; }

int32_t mdhp_plan_last_launches(const mdhp_plan *p) { return p ? p->launches : -1; }

mdhp_status mdhp_plan_set_split(mdhp_plan *p, int32_t enable, int32_t long_threads,
                                int32_t long_ctas_per_sm) {
  if (!p) return fail(MDHP_E_ARG, "plan NULL");
  if (enable) {
    if (long_threads != 64 && long_threads != 128 && long_threads != 256)
      return fail(MDHP_E_ARG, "long_threads %d (64, 128 or 256)", long_threads);
    if (long_ctas_per_sm < 1 || long_ctas_per_sm > 8)
      return fail(MDHP_E_ARG, "long_ctas_per_sm %d (1..8)", long_ctas_per_sm);
    p->xnt_long = long_threads;
    p->xcta_long = long_ctas_per_sm;
  }
  p->xdual = enable ? 1 : 0;
  return MDHP_OK;
}

mdhp_status mdhp_plan_get_split(const mdhp_plan *p, int32_t *enable, int32_t *long_threads,
                                int32_t *long_ctas_per_sm) {
  if (!p) return fail(MDHP_E_ARG, "plan NULL");
  if (enable) *enable = p->xdual;
  if (long_threads) *long_threads = p->xnt_long;
  if (long_ctas_per_sm) *long_ctas_per_sm = p->xcta_long;
  return MDHP_OK;
}

mdhp_status mdhp_plan_get_pipeline(const mdhp_plan *p, int32_t *steps_per_stage, int32_t *stages) {
  if (!p) return fail(MDHP_E_ARG, "plan NULL");
  if (steps_per_stage) *steps_per_stage = p->pipe_steps;
  if (stages) *stages = p->pipe_stages;
  return MDHP_OK;
}

mdhp_status mdhp_plan_get_shape(const mdhp_plan *p, int32_t *nt, int32_t *spl, int32_t *cutoff) {
  if (!p) return fail(MDHP_E_ARG, "plan NULL");
  const bool x = p->use_x && p->xbuf;
  if (nt) *nt = x ? p->xnt : p->shape.nt;
  if (spl) *spl = p->shape.spl;
  if (cutoff) *cutoff = x ? p->xres : p->shape.cutoff;
  return MDHP_OK;
}

mdhp_status mdhp_plan_set_shape(mdhp_plan *p, int32_t nt, int32_t spl, int32_t cutoff) {
  if (!p) return fail(MDHP_E_ARG, "plan NULL");
  if (nt < 32 || nt > 256 || nt % 32 != 0) return fail(MDHP_E_ARG, "threads per window %d (32..256, multiple of 32)", nt);
  if (nt < p->Mt) return fail(MDHP_E_ARG, "threads per window must be >= %d", p->Mt);
  // (matrix beta runs only the decoupled kernels, which have no chunk split)
  if (p->beta_mode != MDHP_BETA_MATRIX && !get_fit(p->Mt, spl, p->beta_mode, false, true))
    return fail(MDHP_E_UNSUPPORTED, "threads per chunk %d not built for M<=%d", spl, p->Mt);
  if (p->beta_mode != MDHP_BETA_MATRIX &&
      !(fit_takes(p->Mt, spl, p->beta_mode, false, nt) && fit_takes(p->Mt, spl, p->beta_mode, true, nt)))
    return fail(MDHP_E_UNSUPPORTED, "%d threads per window exceed the kernel for %d threads per chunk", nt,
                spl);
  if (cutoff < 0) return fail(MDHP_E_ARG, "cutoff < 0");
  p->shape = Shape{nt, spl, cutoff};
  if (nt >= 64 && nt <= 256 && (nt & (nt - 1)) == 0 && nt >= p->Mt) p->xnt = nt;
  p->xres = cutoff < p->xres_max ? (cutoff / 32) * 32 : p->xres_max;
  if (p->xres < 64) p->xres = 0;
  return MDHP_OK;
}

mdhp_status mdhp_fit_batch(mdhp_plan *p, const mdhp_batch *batch, const mdhp_fit_opts *o,
                           float *mu, float *alpha, float *beta, double *loglik, int32_t *iters,
                           int32_t *win_status, void *stream) {
  if (!p) return fail(MDHP_E_ARG, "plan NULL");
  mdhp_status s = check_batch(batch, true);
  if (s != MDHP_OK) return s;
  if (!o) return fail(MDHP_E_ARG, "opts NULL");
  if (batch->M != p->M || batch->beta_mode != p->beta_mode)
    return fail(MDHP_E_ARG, "batch (M=%d, beta_mode=%d) does not match plan (M=%d, %d)", batch->M,
                batch->beta_mode, p->M, p->beta_mode);
  if (batch->B > p->max_windows) return fail(MDHP_E_ARG, "B=%d > plan max_windows=%d", batch->B, p->max_windows);
  if (p->beta_mode == MDHP_BETA_MATRIX) {  // decoupled kernels only
    const int64_t bnd = batch->max_events > 0 ? batch->max_events : p->max_events;
    if (o->fit_beta) return fail(MDHP_E_UNSUPPORTED, "matrix-shaped beta cannot be learned on the GPU");
    if (o->init == 2) return fail(MDHP_E_UNSUPPORTED, "no learned initializer for matrix-shaped beta");
    if (!p->use_x || !p->xbuf || bnd <= 0 || bnd > p->xcap)
      return fail(MDHP_E_UNSUPPORTED, "matrix-shaped beta needs the decoupled kernels (path auto, "
                                      "windows within the plan's max_events_per_window)");
  }
  if (o->max_iters < 1) return fail(MDHP_E_ARG, "max_iters < 1");
  if (o->optimizer != 0 && o->optimizer != 1) return fail(MDHP_E_ARG, "optimizer %d", o->optimizer);
  if (o->init < 0 || o->init > 2) return fail(MDHP_E_ARG, "init %d", o->init);
  if (o->init == 2 && !p->model)
    return fail(MDHP_E_ARG, "init = 2 needs a model (mdhp_plan_set_init_model)");
  if (o->patience < 1) return fail(MDHP_E_ARG, "patience < 1");
  if (!mu || !alpha || !beta || !loglik || !iters || !win_status)
    return fail(MDHP_E_ARG, "NULL parameter/output pointer");
  const int B = batch->B;
  if (B == 0) return MDHP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  mdhp_fit_opts oo = *o;
  int init_launches = 0;
  if (o->init == 2) {  // learned starting point, then the fit from it
    const mdhp_status si = mdhp_init_predict(p->model, batch, beta, mu, alpha, stream);
    if (si != MDHP_OK) return si;
    init_launches = init_predict_launches(p->model, B);
    oo.init = 0;
  }
  o = &oo;
  const Shape sh = p->shape;
  const int NC = sh.nt / sh.spl;
  const bool learn = o->fit_beta != 0;
  // staging capacity: the stated bound if it fits under the cutoff, else the cutoff
  int64_t bound = batch->max_events > 0 ? batch->max_events : p->max_events;
  int ev_cap = (bound > 0 && bound < sh.cutoff) ? (int)bound : sh.cutoff;
  const bool need_long = !(bound > 0 && bound <= sh.cutoff);

  // k_lengths, the radix sort (one kernel at these sizes), k_split, and the
  // initializer's kernels when it ran
  p->launches = 3 + init_launches;
  k_lengths<<<(B + 255) / 256, 256, 0, st>>>(batch->offsets, B, p->keys, p->idx);
  if ((s = cuda_check("k_lengths")) != MDHP_OK) return s;
  size_t tmp = p->sort_tmp_bytes;
  if (cub::DeviceRadixSort::SortPairsDescending(p->sort_tmp, tmp, p->keys, p->keys_sorted, p->idx,
                                                p->order, B, 0, 32, st) != cudaSuccess)
    return cuda_check("radix sort");
  const bool xpath = p->use_x && !learn && p->xbuf && bound > 0 && bound <= p->xcap;
  // decoupled path: windows longer than the shared-memory class form the first range
  int xcut = -1;
  if (p->xres > 0) {
    const int fixed = make_carve_x(p->Mt, p->xnt, 0, o->optimizer == 1, 0, 0, p->beta_mode == 2).total;
    const int fit = ((max_dyn_smem() - 1024 - fixed) / (p->Mt * 4)) / 32 * 32;
    xcut = p->xres < fit ? p->xres : fit;
    if (xcut < 64) xcut = -1;
  }
  k_split<<<1, 32, 0, st>>>(p->keys_sorted, B, xpath ? xcut : ev_cap, (xpath || need_long) ? 1 : 0,
                            p->ctl);
  if ((s = cuda_check("k_split")) != MDHP_OK) return s;

  FitArgs a{};
  a.offsets = batch->offsets; a.t = batch->t; a.id = batch->id; a.T = batch->T_span;
  a.w = batch->weights; a.mu = mu; a.alpha = alpha; a.beta = beta; a.loglik = loglik;
  a.iters = iters; a.status = win_status; a.order = p->order;
  a.Mrt = batch->M; a.NC = NC;
  a.optimizer = o->optimizer; a.max_iters = o->max_iters; a.fit_beta = o->fit_beta;
  a.patience = o->patience; a.init = o->init; a.lr = o->lr; a.mu_floor = o->mu_floor;
  a.alpha_floor = o->alpha_floor; a.beta_floor = o->beta_floor; a.b1 = o->adam_b1;
  a.b2 = o->adam_b2; a.eps = o->adam_eps; a.tol = o->tol;
  a.wait_polls = p->wait_polls;

  int xres = p->xres;
  if (xpath && xres > 0) {  // the largest class that fits this block size
    const int fixed = make_carve_x(p->Mt, p->xnt, 0, o->optimizer == 1, 0, 0, p->beta_mode == 2).total;
    const int fit = ((max_dyn_smem() - 1024 - fixed) / (p->Mt * 4)) / 32 * 32;
    if (xres > fit) xres = fit;
    if (xres < 64) xres = 0;
  }
  if (xpath) {
    // long windows: features in the per-CTA global scratch (side stream);
    // short windows: features in shared memory (this stream); both queues
    // are taken longest first
    FitArgs ax = a;
    ax.xbuf = p->xbuf;
    const bool any_long = !(xres > 0 && bound <= xres);
    if (p->timing) cudaEventRecord(p->ev_t0, st);
    bool dual_done = false;
    if (any_long && xres == 0 && p->xdual && p->xnt_long != p->xnt) {
      if ((s = launch_dual(p, ax, o->optimizer == 1, st, &dual_done)) != MDHP_OK) return s;
    }
    if (any_long && !dual_done) {
      FitArgs al = ax;
      al.queue = p->ctl + 0;
      al.range = p->ctl + 2;
      al.ev_cap = p->xcap;
      al.pipe_steps = p->pipe_steps;
      al.pipe_stages = p->pipe_stages;
      if (p->beta_mode == 2) al.pipe_stages = 0;  // the ring is not built for matrix beta
      al.carve = make_carve_x(p->Mt, p->xnt, 0, o->optimizer == 1, p->pipe_steps, al.pipe_stages,
                              p->beta_mode == 2);
      if (al.pipe_stages > 0 && al.carve.total > max_dyn_smem()) {  // ring too large for this block
        al.pipe_stages = 0;
        al.carve = make_carve_x(p->Mt, p->xnt, 0, o->optimizer == 1, 0, 0, p->beta_mode == 2);
      }
      FitFn fx = get_fitx(p->Mt, p->beta_mode, al.pipe_stages > 0 ? XM_RING : XM_GLOBAL, p->xnt);
      // feature store 3: the tensor-memory kernel with 384 threads (12 warps)
      const int ntx = (p->xtmem == 3 && al.pipe_stages == 0) ? 384 : p->xnt;
      FitFn ft = (p->xtmem && al.pipe_stages == 0) ? get_fitx(p->Mt, p->beta_mode, XM_TMEM, ntx)
                                                   : nullptr;
      if (ft) {
        fx = ft;
        al.carve = make_carve_x(p->Mt, ntx, 0, o->optimizer == 1, 0, 0, p->beta_mode == 2);
      }
      const int nlaunch = ft ? ntx : p->xnt;
      int dyn = al.carve.total;
      int occ = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fx, nlaunch, dyn);
      if (ft) {
        // each resident CTA's share of the 512 tensor-memory columns (a
        // power of two) and, with feature store 2 or 3, of the shared memory
        // the carve leaves at this occupancy: steps of NT float4 slices
        int cols = 512;
        while (cols > 32 && cols * std::max(occ, 1) > 512) cols >>= 1;
        al.tmem_cols = cols;
        const int sets = std::max(nlaunch / 128, 1);
        if (cols * std::max(occ, 1) > 512 || cols / sets < p->Mt)
          return fail(MDHP_E_UNSUPPORTED, "tensor-memory features: %d CTAs per SM leave no row", occ);
        al.smem_steps = 0;
        if (p->xtmem >= 2) {
          int dev = 0, smem_sm = 0;
          cudaGetDevice(&dev);
          cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
          const int step_bytes = p->Mt * 4 * nlaunch;
          const int room = std::min(smem_sm / std::max(occ, 1) - 1024, max_dyn_smem()) - dyn;
          al.smem_steps = std::max(0, std::min(room / step_bytes, 64));
          dyn += al.smem_steps * step_bytes;
        }
      }
      if ((s = prepare_kernel((const void *)fx, dyn)) != MDHP_OK) return s;
      cudaStream_t ls = st;
      if (xres > 0) {
        cudaEventRecord(p->ev_fork, st);
        cudaStreamWaitEvent(p->side, p->ev_fork, 0);
        ls = p->side;
      }
      int gl = num_sms() * (occ > 0 ? occ : 1);
      if (gl > p->xgrid) gl = p->xgrid;
      fx<<<gl, nlaunch, dyn, ls>>>(al);
      ++p->launches;
      if ((s = cuda_check("k_fit_x (global features)")) != MDHP_OK) return s;
      if (xres > 0) cudaEventRecord(p->ev_join, p->side);
    }
    if (xres > 0) {
      FitFn fr = get_fitx(p->Mt, p->beta_mode, XM_SHARED, p->xnt);
      FitArgs ar = ax;
      ar.queue = p->ctl + 1;
      ar.range = p->ctl + 4;
      ar.ev_cap = xres;
      ar.carve = make_carve_x(p->Mt, p->xnt, xres, o->optimizer == 1, 0, 0, p->beta_mode == 2);
      if ((s = prepare_kernel((const void *)fr, ar.carve.total)) != MDHP_OK) return s;
      int occr = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occr, fr, p->xnt, ar.carve.total);
      int grid = num_sms() * (occr > 0 ? occr : 1);
      if (grid > B) grid = B;
      fr<<<grid, p->xnt, ar.carve.total, st>>>(ar);
      ++p->launches;
      if ((s = cuda_check("k_fit_x (shared features)")) != MDHP_OK) return s;
      if (any_long) cudaStreamWaitEvent(st, p->ev_join, 0);
    }
    if (p->timing) {
      cudaEventRecord(p->ev_t1, st);
      p->timed = 1;
    }
    return MDHP_OK;
  }
  if (p->timing) cudaEventRecord(p->ev_t0, st);
  if (need_long) {
    FitFn fl = get_fit(p->Mt, sh.spl, p->beta_mode, learn, false);
    if (!fl || kernel_max_threads((const void *)fl) < sh.nt)
      return fail(MDHP_E_UNSUPPORTED, "no streamed fit kernel for this shape");
    FitArgs al = a;
    al.queue = p->ctl + 0;
    al.range = p->ctl + 2;
    al.ev_cap = 0;
    al.pbuf = p->pbuf;
    al.pstride = p->pstride;
    al.ring = (p->ev_ring && !batch->weights && ((uintptr_t)batch->t & 15) == 0 &&
               ((uintptr_t)batch->id & 15) == 0)
                  ? 1
                  : 0;
    al.n_total = batch->n_events;
    al.carve = make_carve(p->Mt, sh.nt, sh.spl, 0, batch->weights != nullptr, learn,
                          o->optimizer == 1, true, use_priv(p->Mt), false, al.ring != 0);
    if (al.ring && al.carve.total > max_dyn_smem()) {  // no room for the ring: read global memory
      al.ring = 0;
      al.carve = make_carve(p->Mt, sh.nt, sh.spl, 0, batch->weights != nullptr, learn,
                            o->optimizer == 1, true, use_priv(p->Mt), false);
    }
    if ((s = prepare_kernel((const void *)fl, al.carve.total)) != MDHP_OK) return s;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fl, sh.nt, al.carve.total);
    int grid = num_sms() * (occ > 0 ? occ : 1);
    if (grid > p->pslots) grid = p->pslots;
    fl<<<grid, sh.nt, al.carve.total, st>>>(al);
    ++p->launches;
    if ((s = cuda_check("k_fit (streamed)")) != MDHP_OK) return s;
  }
  {
    FitFn fs = get_fit(p->Mt, sh.spl, p->beta_mode, learn, true);
    if (!fs || kernel_max_threads((const void *)fs) < sh.nt)
      return fail(MDHP_E_UNSUPPORTED, "no staged fit kernel for this shape");
    FitArgs as = a;
    as.queue = p->ctl + 1;
    as.range = p->ctl + 4;
    as.ev_cap = ev_cap;
    as.pbuf = p->pbuf;
    as.pstride = p->pstride;
    as.carve = make_carve(p->Mt, sh.nt, sh.spl, ev_cap, batch->weights != nullptr, learn,
                          o->optimizer == 1, true, use_priv(p->Mt), false);
    if (as.carve.total > max_dyn_smem())
      return fail(MDHP_E_ARG, "shared memory %d > %d (lower the cutoff)", as.carve.total, max_dyn_smem());
    if ((s = prepare_kernel((const void *)fs, as.carve.total)) != MDHP_OK) return s;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fs, sh.nt, as.carve.total);
    int grid = num_sms() * (occ > 0 ? occ : 1);
    if (grid > B) grid = B;
    if (grid > p->pslots) grid = p->pslots;
    fs<<<grid, sh.nt, as.carve.total, st>>>(as);
    ++p->launches;
    if ((s = cuda_check("k_fit (staged)")) != MDHP_OK) return s;
  }
  if (p->timing) {
    cudaEventRecord(p->ev_t1, st);
    p->timed = 1;
  }
  return MDHP_OK;
}

mdhp_status mdhp_plan_autotune(mdhp_plan *p, const mdhp_batch *batch, const mdhp_fit_opts *o,
                               float *mu, float *alpha, float *beta, double *loglik, int32_t *iters,
                               int32_t *win_status, int32_t tune_iters, int32_t *chosen,
                               float *best_ms, void *stream) {
  if (!p) return fail(MDHP_E_ARG, "plan NULL");
  mdhp_status s = check_batch(batch, true);
  if (s != MDHP_OK) return s;
  if (!o) return fail(MDHP_E_ARG, "opts NULL");
  if (!mu || !alpha || !beta || !loglik || !iters || !win_status)
    return fail(MDHP_E_ARG, "NULL parameter/output pointer");
  if (batch->M != p->M || batch->beta_mode != p->beta_mode)
    return fail(MDHP_E_ARG, "batch does not match plan");
  const int B = batch->B;
  if (B == 0) return MDHP_OK;
  mdhp_fit_opts oo = *o;
  if (o->tol > 0.0) {
    // a fit to a tolerance ends when its slowest windows converge, so the
    // candidates run the caller's fit itself (same tolerance and start),
    // capped at tune_iters evaluations per window
    const int cap = tune_iters > 0 ? tune_iters : 500;
    oo.max_iters = o->max_iters < cap ? o->max_iters : cap;
  } else {
    oo.max_iters = tune_iters > 0 ? tune_iters : 20;  // every window runs the same count
  }
  const bool learn = oo.fit_beta != 0, adam = oo.optimizer == 1;
  const int64_t bound = batch->max_events > 0 ? batch->max_events : p->max_events;
  const int path = (p->use_x && !learn && p->xbuf && bound > 0 && bound <= p->xcap) ? 0 : 1;
  cudaStream_t st = (cudaStream_t)stream;
  // the fit overwrites mu / alpha / beta: keep the caller's values and put
  // them back before every timed run and at the end
  const size_t nmu = (size_t)B * p->M, nal = nmu * p->M,
               nbe = (size_t)B * (p->beta_mode == 0 ? 1 : p->M);
  float *snap = nullptr;
  if (cudaMalloc(&snap, (nmu + nal + nbe) * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return fail(MDHP_E_NOMEM, "autotune: snapshot allocation failed");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto copy_params = [&](bool save) {
    float *d[3] = {mu, alpha, beta};
    const size_t n[3] = {nmu, nal, nbe};
    size_t off = 0;
    for (int k = 0; k < 3; ++k) {
      if (save) cudaMemcpyAsync(snap + off, d[k], n[k] * sizeof(float), cudaMemcpyDeviceToDevice, st);
      else cudaMemcpyAsync(d[k], snap + off, n[k] * sizeof(float), cudaMemcpyDeviceToDevice, st);
      off += n[k];
    }
  };
  copy_params(true);
  using Cand = TuneChoice;
  std::vector<Cand> cands;
  static const int kPipes[][2] = {{0, 0}, {1, 4}, {2, 3}, {2, 4}, {4, 3}};
  for (int nt = 64; nt <= 256; nt *= 2) {
    if (nt < p->Mt) continue;
    if (path == 0) {
      const int fit = xres_fit(p, nt, adam);
      for (const auto &pd : kPipes) {
        if (pd[1] > 0 && (p->beta_mode == 2 ||
                          make_carve_x(p->Mt, nt, 0, adam, pd[0], pd[1]).total > max_dyn_smem()))
          continue;
        cands.push_back({nt, 0, 0, pd[0], pd[1], 0, 256, 1});
        if (fit >= 64) cands.push_back({nt, 0, fit, pd[0], pd[1], 0, 256, 1});
      }
      if (fit >= 128) cands.push_back({nt, 0, fit / 2 / 32 * 32, 0, 0, 0, 256, 1});
      if (p->beta_mode != 2 && get_fitx(p->Mt, p->beta_mode, XM_TMEM, nt)) {
        for (int tm = 1; tm <= 3; ++tm) {  // store 3 runs its own 384-thread kernel
          if (tm == 3 && !get_fitx(p->Mt, p->beta_mode, XM_TMEM, 384)) continue;
          cands.push_back({nt, 0, 0, 0, 0, 0, 256, 1, tm});
          if (fit >= 64) cands.push_back({nt, 0, fit, 0, 0, 0, 256, 1, tm});
        }
      }
      static const int kSplits[][2] = {{256, 1}, {256, 2}, {128, 1}, {128, 2}};
      for (const auto &sp : kSplits)  // a split the caller disabled is not a candidate
        if (p->xdual && sp[0] != nt && nt < 256) cands.push_back({nt, 0, 0, 0, 0, 1, sp[0], sp[1]});
    } else {
      for (int spl = 1; spl <= 32; spl *= 2) {
        if (nt % spl || !fit_takes(p->Mt, spl, p->beta_mode, learn, nt)) continue;
        const int fit = stage_fit(p, nt, spl, batch->weights != nullptr, learn, adam);
        const int dflt = default_shape(p->Mt).cutoff;
        cands.push_back({nt, spl, 0, 0, 0, 0, 256, 1});
        if (dflt <= fit) cands.push_back({nt, spl, dflt, 0, 0, 0, 256, 1});
        if (fit >= 64 && fit != dflt) cands.push_back({nt, spl, fit, 0, 0, 0, 256, 1});
      }
    }
  }
  if (cands.empty()) {
    cudaFree(snap);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return fail(MDHP_E_UNSUPPORTED, "autotune: no candidate shape for M=%d", p->M);
  }
  const Shape shape0 = p->shape;
  const int xnt0 = p->xnt, xres0 = p->xres, timing0 = p->timing;
  const int ps0 = p->pipe_steps, pd0 = p->pipe_stages;
  const int du0 = p->xdual, ntl0 = p->xnt_long, cl0 = p->xcta_long, tm0 = p->xtmem;
  p->timing = 0;
  float best = -1.f;
  Cand win{0, 0, 0, 0, 0, 0, 256, 1};
  mdhp_status last = MDHP_OK;
  for (size_t c = 0; c <= cands.size(); ++c) {
    const Cand cd = cands[c == 0 ? 0 : c - 1];  // run 0 warms the first candidate up
    const bool okc = path == 0 ? apply_decoupled(p, cd.nt, cd.cut)
                               : apply_recursion(p, cd.nt, cd.spl, cd.cut);
    if (!okc) continue;
    if (path == 0) {
      p->pipe_steps = cd.ps;
      p->pipe_stages = cd.pd;
      p->xdual = cd.dual;
      p->xnt_long = cd.ntl;
      p->xcta_long = cd.cl;
      p->xtmem = cd.tm;
    }
    copy_params(false);
    cudaEventRecord(e0, st);
    const mdhp_status r = mdhp_fit_batch(p, batch, &oo, mu, alpha, beta, loglik, iters, win_status, stream);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      last = fail(MDHP_E_CUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
    if (r != MDHP_OK) {  // this shape cannot run this batch: skip it
      last = r;
      cudaGetLastError();
      continue;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (c > 0 && (best < 0.f || ms < best)) {
      best = ms;
      win = cd;
    }
  }
  p->timing = timing0;
  p->shape = shape0;
  p->xnt = xnt0;
  p->xres = xres0;
  p->pipe_steps = ps0;
  p->pipe_stages = pd0;
  p->xdual = du0;
  p->xnt_long = ntl0;
  p->xcta_long = cl0;
  p->xtmem = tm0;
  copy_params(false);
  cudaStreamSynchronize(st);
  cudaFree(snap);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best < 0.f)
    return last != MDHP_OK ? last : fail(MDHP_E_UNSUPPORTED, "autotune: no candidate shape ran");
  if (path == 0) {
    apply_decoupled(p, win.nt, win.cut);
    p->pipe_steps = win.ps;
    p->pipe_stages = win.pd;
    p->xdual = win.dual;
    p->xnt_long = win.ntl;
    p->xcta_long = win.cl;
    p->xtmem = win.tm;
  } else {
    apply_recursion(p, win.nt, win.spl, win.cut);
  }
  if (chosen) {
    chosen[0] = path;
    chosen[1] = win.nt;
    chosen[2] = win.spl;
    chosen[3] = win.cut;
    chosen[4] = path == 0 ? win.ps : 0;
    chosen[5] = path == 0 ? win.pd : 0;
    chosen[6] = path == 0 ? win.dual : 0;
    chosen[7] = path == 0 ? win.ntl : 0;
    chosen[8] = path == 0 ? win.cl : 0;
  }
  if (best_ms) *best_ms = best;
  if (!tune_store(p, path, win, best))
    return fail(MDHP_E_ARG, "autotune: cannot write the cache file %s", p->cache.c_str());
  return MDHP_OK;
}

}  // extern "C"
