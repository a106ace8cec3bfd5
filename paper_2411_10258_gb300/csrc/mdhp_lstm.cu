// MDHP-LSTM cell (the paper's MDHP-LSTM equation, Sec. "MDHP-LSTM"): an LSTM
// whose cell update is gated by a per-sequence Hawkes state
//   hks = tanh(A vec(alpha) - Bm (beta T_span) + C mu)
//   i, f, o = sigmoid(W_{i,f,o} x_t + U_{i,f,o} h_{t-1} + b_{i,f,o})
//   g = tanh(W_c x_t + U_c h_{t-1} + b_c)
//   c_t = hks * (f * c_{t-1} + i * g),  h_t = o * tanh(c_t),  y_t = Wy h_t
// Forward and backward (backpropagation through time) in FP32.
//
// One CTA per sequence walks all L steps (the recursion is serial in t):
// thread r computes gate row r (4H rows: i, f, g, o), threads j < H update
// the cell.  The gate weights are staged transposed in shared memory when
// they fit ([input][row]: a warp's loads of one input are consecutive), else
// read from global memory.  The backward CTA walks t backwards, producing the
// pre-activation gate gradients dz (kept for the weight gradients), dx, and
// the gradient of the Hawkes gate.  The weight gradients are row sums of
// outer products, sum_r a_r^T b_r over the B*L steps, by a split reduction.
#include <cstdint>
#include <cstdio>

#include "mdhp.h"
#include "mdhp_dispatch.h"

namespace mdhp {
namespace {

__device__ __forceinline__ float sigm(float z) { return 1.f / (1.f + expf(-z)); }

struct LstmFwd {
  int B, L, D, H, M, nb, O, staged;
  const float *x, *mu, *alpha, *beta, *T, *W, *U, *b, *A, *Bm, *C, *Wy;
  float *y, *hs, *cs, *gates, *hks;
};

__global__ void __launch_bounds__(1024) k_lstm_fwd(LstmFwd a) {
  extern __shared__ __align__(16) float sm[];
  const int H = a.H, D = a.D, G = 4 * H, bq = blockIdx.x, r = threadIdx.x;
  float *xs = sm, *h = xs + D, *c = h + H, *z = c + H, *kh = z + G;
  float *WT = kh + H;         // [D][G]   (staged)
  float *UT = WT + D * G;     // [H][G]
  if (a.staged) {
    for (int p = r; p < G * D; p += blockDim.x) WT[(p % D) * G + p / D] = a.W[p];
    for (int p = r; p < G * H; p += blockDim.x) UT[(p % H) * G + p / H] = a.U[p];
  }
  const int MM = a.M * a.M;
  if (r < H) {  // the Hawkes gate of this sequence
    float s = 0.f;
    for (int k = 0; k < MM; ++k) s = fmaf(a.A[(int64_t)r * MM + k], a.alpha[(int64_t)bq * MM + k], s);
    for (int k = 0; k < a.nb; ++k)
      s = fmaf(-a.Bm[(int64_t)r * a.nb + k], a.beta[(int64_t)bq * a.nb + k] * a.T[bq], s);
    for (int k = 0; k < a.M; ++k) s = fmaf(a.C[(int64_t)r * a.M + k], a.mu[(int64_t)bq * a.M + k], s);
    kh[r] = tanhf(s);
    a.hks[(int64_t)bq * H + r] = kh[r];
    h[r] = 0.f;
    c[r] = 0.f;
  }
  const float br = r < G ? a.b[r] : 0.f;
  const bool tanh_row = r >= 2 * H && r < 3 * H;
  for (int t = 0; t < a.L; ++t) {
    const int64_t row = (int64_t)bq * a.L + t;
    if (r < D) xs[r] = a.x[row * D + r];
    __syncthreads();  // x_t in; h_{t-1} final
    if (r < G) {
      float s = br;
      if (a.staged) {
        for (int d = 0; d < D; ++d) s = fmaf(WT[d * G + r], xs[d], s);
        for (int k = 0; k < H; ++k) s = fmaf(UT[k * G + r], h[k], s);
      } else {
        for (int d = 0; d < D; ++d) s = fmaf(a.W[(int64_t)r * D + d], xs[d], s);
        for (int k = 0; k < H; ++k) s = fmaf(a.U[(int64_t)r * H + k], h[k], s);
      }
      const float v = tanh_row ? tanhf(s) : sigm(s);
      z[r] = v;
      a.gates[row * G + r] = v;
    }
    __syncthreads();  // gates in; everyone is done reading h_{t-1}
    if (r < H) {
      const float cn = kh[r] * fmaf(z[H + r], c[r], z[r] * z[2 * H + r]);
      const float hn = z[3 * H + r] * tanhf(cn);
      c[r] = cn;
      h[r] = hn;
      a.cs[row * H + r] = cn;
      a.hs[row * H + r] = hn;
    }
    __syncthreads();  // h_t in
    if (r < a.O) {
      float s = 0.f;
      for (int k = 0; k < H; ++k) s = fmaf(a.Wy[(int64_t)r * H + k], h[k], s);
      a.y[row * a.O + r] = s;
    }
  }
}

struct LstmBwd {
  int B, L, D, H, O, staged;
  const float *W, *U, *Wy, *hs, *cs, *gates, *hks, *dy;
  float *dz, *dpre, *dx;
};

__global__ void __launch_bounds__(1024) k_lstm_bwd(LstmBwd a) {
  extern __shared__ __align__(16) float sm[];
  const int H = a.H, D = a.D, G = 4 * H, bq = blockIdx.x, r = threadIdx.x;
  float *dh = sm, *dzs = dh + H;
  float *Ws = dzs + G;  // W [G][D] and U [G][H] as given (row r of gate r)
  float *Us = Ws + G * D;
  if (a.staged) {
    for (int p = r; p < G * D; p += blockDim.x) Ws[p] = a.W[p];
    for (int p = r; p < G * H; p += blockDim.x) Us[p] = a.U[p];
  }
  if (r < H) dh[r] = 0.f;
  float dc_next = 0.f, dhks = 0.f;
  const float kh = r < H ? a.hks[(int64_t)bq * H + r] : 0.f;
  __syncthreads();
  for (int t = a.L - 1; t >= 0; --t) {
    const int64_t row = (int64_t)bq * a.L + t;
    if (r < H) {
      float dht = dh[r];
      for (int k = 0; k < a.O; ++k) dht = fmaf(a.Wy[(int64_t)k * H + r], a.dy[row * a.O + k], dht);
      const float ig = a.gates[row * G + r], fg = a.gates[row * G + H + r];
      const float gg = a.gates[row * G + 2 * H + r], og = a.gates[row * G + 3 * H + r];
      const float cv = a.cs[row * H + r];
      const float cp = t > 0 ? a.cs[(row - 1) * H + r] : 0.f;
      const float tc = tanhf(cv);
      const float dc = fmaf(dht * og, 1.f - tc * tc, dc_next);
      const float inner = fmaf(fg, cp, ig * gg);
      dhks = fmaf(dc, inner, dhks);
      const float din = dc * kh;
      const float zi = din * gg * ig * (1.f - ig);
      const float zf = din * cp * fg * (1.f - fg);
      const float zg = din * ig * (1.f - gg * gg);
      const float zo = dht * tc * og * (1.f - og);
      dzs[r] = zi;
      dzs[H + r] = zf;
      dzs[2 * H + r] = zg;
      dzs[3 * H + r] = zo;
      a.dz[row * G + r] = zi;
      a.dz[row * G + H + r] = zf;
      a.dz[row * G + 2 * H + r] = zg;
      a.dz[row * G + 3 * H + r] = zo;
      dc_next = din * fg;
    }
    __syncthreads();  // dz_t in; dh (of step t) read by everyone
    if (r < H) {  // dh_{t-1} = U^T dz
      float s = 0.f;
      if (a.staged)
        for (int q = 0; q < G; ++q) s = fmaf(Us[q * H + r], dzs[q], s);
      else
        for (int q = 0; q < G; ++q) s = fmaf(a.U[(int64_t)q * H + r], dzs[q], s);
      dh[r] = s;
    } else if (r < H + D) {  // dx_t = W^T dz
      const int d = r - H;
      float s = 0.f;
      if (a.staged)
        for (int q = 0; q < G; ++q) s = fmaf(Ws[q * D + d], dzs[q], s);
      else
        for (int q = 0; q < G; ++q) s = fmaf(a.W[(int64_t)q * D + d], dzs[q], s);
      a.dx[row * D + d] = s;
    }
    __syncthreads();
  }
  if (r < H) a.dpre[(int64_t)bq * H + r] = dhks * (1.f - kh * kh);
}

// out[p][q] (+)= scale * sum_{r < R} A(r, p) B(r, q), A(r, p) = A[r * lda + p],
// B(r, q) = B[r * ldb + q] (or B[(r - 1) * ldb + q] with row r % L == 0 zero
// when shift_L > 0: h_{t-1}); B == nullptr means B(r, q) = 1 (row sums).
// 16 x 16 output tiles, the rows split over gridDim.z slices, atomic adds.
__global__ void __launch_bounds__(256) k_atb(const float *A, int64_t lda, const float *Bp, int64_t ldb,
                                             int P, int Q, int64_t R, int shift_L, float scale,
                                             float *out) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int p = blockIdx.y * 16 + ty, q = blockIdx.x * 16 + tx;
  __shared__ float As[32][17], Bs[32][17];
  const int64_t per = (R + gridDim.z - 1) / gridDim.z;
  const int64_t r0 = blockIdx.z * per, r1 = r0 + per < R ? r0 + per : R;
  float acc = 0.f;
  for (int64_t rb = r0; rb < r1; rb += 32) {
    for (int e = threadIdx.x; e < 32 * 16; e += 256) {
      const int rr = e >> 4, cc = e & 15;
      const int64_t r = rb + rr;
      const int pp = blockIdx.y * 16 + cc, qq = blockIdx.x * 16 + cc;
      As[rr][cc] = (r < r1 && pp < P) ? A[r * lda + pp] : 0.f;
      float bv = 0.f;
      if (r < r1 && qq < Q) {
        if (!Bp) bv = 1.f;
        else if (shift_L > 0) bv = (r % shift_L == 0) ? 0.f : Bp[(r - 1) * ldb + qq];
        else bv = Bp[r * ldb + qq];
      }
      Bs[rr][cc] = bv;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) acc = fmaf(As[k][ty], Bs[k][tx], acc);
    __syncthreads();
  }
  if (p < P && q < Q) atomicAdd(&out[(int64_t)p * Q + q], scale * acc);
}

// out[b][q] = scale * sum_p Din[b][p] Wm[p][q] * (rowscale ? rowscale[b] : 1)
__global__ void k_rowmat(const float *Din, const float *Wm, int Bn, int P, int Q, float scale,
                         const float *rowscale, float *out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)Bn * Q) return;
  const int b = (int)(e / Q), q = (int)(e % Q);
  float s = 0.f;
  for (int p = 0; p < P; ++p) s = fmaf(Din[(int64_t)b * P + p], Wm[(int64_t)p * Q + q], s);
  out[e] = scale * s * (rowscale ? rowscale[b] : 1.f);
}

// out[b][k] = in[b][k] * scale[b]
__global__ void k_scale_rows(const float *in, const float *scale, int Bn, int K, float *out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < (int64_t)Bn * K) out[e] = in[e] * scale[e / K];
}

int max_smem() {
  static int v = -1;
  if (v < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  return v;
}

mdhp_status check_dims(const mdhp_lstm_dims *d) {
  if (!d) return MDHP_E_ARG;
  if (d->B < 0 || d->L < 1 || d->D < 1 || d->H < 1 || d->H > 256 || d->M < 1 || d->M > 64 ||
      (d->nb != 1 && d->nb != d->M) || d->O < 0 || d->O > 4 * d->H || d->D > 3 * d->H)
    return MDHP_E_ARG;
  return MDHP_OK;
}

mdhp_status launched(const char *what) {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return MDHP_OK;
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  record_error(buf);
  return MDHP_E_CUDA;
}

}  // namespace
}  // namespace mdhp

using namespace mdhp;

extern "C" mdhp_status mdhp_lstm_forward(const mdhp_lstm_dims *d, const float *x, const float *mu,
                                         const float *alpha, const float *beta, const float *T_span,
                                         const float *W, const float *U, const float *b,
                                         const float *A, const float *Bm, const float *C,
                                         const float *Wy, float *y, float *h_seq, float *c_seq,
                                         float *gates, float *hks, void *stream) {
  if (check_dims(d) != MDHP_OK) {
    record_error("mdhp_lstm_forward: dims (H 1..256, D <= 3H, O <= 4H, M 1..64, nb 1 or M, L >= 1)");
    return MDHP_E_ARG;
  }
  if (d->B == 0) return MDHP_OK;
  if (!x || !mu || !alpha || !beta || !T_span || !W || !U || !b || !A || !Bm || !C || !Wy || !y ||
      !h_seq || !c_seq || !gates || !hks) {
    record_error("mdhp_lstm_forward: NULL argument");
    return MDHP_E_ARG;
  }
  const int G = 4 * d->H;
  const int base = (d->D + 2 * d->H + G + d->H) * 4;
  const int full = base + (d->D + d->H) * G * 4;
  const int staged = full <= max_smem() ? 1 : 0;
  const int smem = staged ? full : base;
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_lstm_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  LstmFwd a{d->B, d->L, d->D, d->H, d->M, d->nb, d->O, staged, x, mu, alpha, beta, T_span, W, U, b, A,
            Bm, C, Wy, y, h_seq, c_seq, gates, hks};
  const int threads = (G + 31) / 32 * 32;
  k_lstm_fwd<<<d->B, threads, smem, (cudaStream_t)stream>>>(a);
  return launched("k_lstm_fwd");
}

extern "C" mdhp_status mdhp_lstm_backward(
    const mdhp_lstm_dims *d, const float *x, const float *mu, const float *alpha, const float *beta,
    const float *T_span, const float *W, const float *U, const float *A, const float *Bm,
    const float *C, const float *Wy, const float *h_seq, const float *c_seq, const float *gates,
    const float *hks, const float *dy, float *dz_work, float *dpre_work, float *dx, float *dW,
    float *dU, float *db, float *dA, float *dBm, float *dC, float *dWy, float *dmu, float *dalpha,
    float *dbeta, void *stream) {
  if (check_dims(d) != MDHP_OK) {
    record_error("mdhp_lstm_backward: dims");
    return MDHP_E_ARG;
  }
  if (!x || !mu || !alpha || !beta || !T_span || !W || !U || !A || !Bm || !C || !Wy || !h_seq ||
      !c_seq || !gates || !hks || !dy || !dz_work || !dpre_work || !dx || !dW || !dU || !db || !dA ||
      !dBm || !dC || !dWy || !dmu || !dalpha || !dbeta) {
    record_error("mdhp_lstm_backward: NULL argument");
    return MDHP_E_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int H = d->H, D = d->D, G = 4 * H, M = d->M, MM = M * M, nb = d->nb, O = d->O;
  cudaMemsetAsync(dW, 0, (size_t)G * D * 4, st);
  cudaMemsetAsync(dU, 0, (size_t)G * H * 4, st);
  cudaMemsetAsync(db, 0, (size_t)G * 4, st);
  cudaMemsetAsync(dA, 0, (size_t)H * MM * 4, st);
  cudaMemsetAsync(dBm, 0, (size_t)H * nb * 4, st);
  cudaMemsetAsync(dC, 0, (size_t)H * M * 4, st);
  cudaMemsetAsync(dWy, 0, (size_t)(O > 0 ? O : 1) * H * 4, st);
  if (d->B == 0) return launched("mdhp_lstm_backward");
  const int base = (H + G) * 4;
  const int full = base + (D + H) * G * 4;
  const int staged = full <= max_smem() ? 1 : 0;
  const int smem = staged ? full : base;
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_lstm_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  LstmBwd a{d->B, d->L, D, H, O, staged, W, U, Wy, h_seq, c_seq, gates, hks, dy, dz_work, dpre_work, dx};
  const int threads = (G + 31) / 32 * 32;
  k_lstm_bwd<<<d->B, threads, smem, st>>>(a);
  mdhp_status s = launched("k_lstm_bwd");
  if (s != MDHP_OK) return s;
  const int64_t R = (int64_t)d->B * d->L;
  auto atb = [&](const float *Ap, int64_t lda, const float *Bp, int64_t ldb, int P, int Q, int64_t rows,
                 int shift, float scale, float *out) {
    const int64_t split = rows >= 4096 ? 32 : (rows >= 512 ? 8 : 1);
    dim3 grid((Q + 15) / 16, (P + 15) / 16, (unsigned)split);
    k_atb<<<grid, 256, 0, st>>>(Ap, lda, Bp, ldb, P, Q, rows, shift, scale, out);
  };
  atb(dz_work, G, x, D, G, D, R, 0, 1.f, dW);          // dW = sum_r dz_r^T x_r
  atb(dz_work, G, h_seq, H, G, H, R, d->L, 1.f, dU);   // dU = sum_r dz_r^T h_{r-1}
  atb(dz_work, G, nullptr, 0, G, 1, R, 0, 1.f, db);    // db = sum_r dz_r
  if (O > 0) atb(dy, O, h_seq, H, O, H, R, 0, 1.f, dWy);  // dWy = sum_r dy_r^T h_r
  // Hawkes gate: dA, dBm, dC over sequences; d(alpha, beta, mu) per sequence
  atb(dpre_work, H, alpha, MM, H, MM, d->B, 0, 1.f, dA);
  atb(dpre_work, H, mu, M, H, M, d->B, 0, 1.f, dC);
  const int eb = 256;
  k_rowmat<<<(int)(((int64_t)d->B * MM + eb - 1) / eb), eb, 0, st>>>(dpre_work, A, d->B, H, MM, 1.f,
                                                                      nullptr, dalpha);
  k_rowmat<<<(int)(((int64_t)d->B * M + eb - 1) / eb), eb, 0, st>>>(dpre_work, C, d->B, H, M, 1.f,
                                                                     nullptr, dmu);
  // d(beta T)/d beta = T: dbeta[b] = -(dpre[b] Bm) T[b]
  k_rowmat<<<(int)(((int64_t)d->B * nb + eb - 1) / eb), eb, 0, st>>>(dpre_work, Bm, d->B, H, nb, -1.f,
                                                                      T_span, dbeta);
  // dBm = -sum_b dpre_b^T (beta_b T_b): beta_b T_b formed into the work buffer
  // (free now: the reductions reading dz were enqueued before on this stream)
  k_scale_rows<<<(int)(((int64_t)d->B * nb + eb - 1) / eb), eb, 0, st>>>(beta, T_span, d->B, nb, dz_work);
  atb(dpre_work, H, dz_work, nb, H, nb, d->B, 0, -1.f, dBm);
  return launched("lstm hawkes gradients");
}
