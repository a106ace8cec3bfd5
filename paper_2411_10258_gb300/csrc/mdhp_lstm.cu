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
#include <cstdlib>
#include <cstdio>

#include "mdhp.h"
#include "mdhp_dispatch.h"

namespace mdhp {
namespace {

__device__ __forceinline__ float sigm(float z) { return 1.f / (1.f + expf(-z)); }

// Gate activations of the multi-sequence kernels from the fast exponential
// and division intrinsics: sigmoid(z) = 1 / (1 + e^-z), tanh(z) =
// 2 sigmoid(2z) - 1.  Error about 1e-6 relative for the sigmoid and 1e-7
// absolute for tanh (the intrinsic's error grows with |z|, and at |z| > 80
// e^-z overflows to inf, where the quotient is 0).
__device__ __forceinline__ float sigm_fast(float z) { return __fdividef(1.f, 1.f + __expf(-z)); }
__device__ __forceinline__ float tanh_fast(float z) { return fmaf(2.f, sigm_fast(2.f * z), -1.f); }

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

// S sequences per CTA.  Forward: thread r keeps S accumulators of gate row
// r, so each staged weight is read once per step for S sequences and the two
// barriers of a step serve S sequences.  The matvec operands x_t and h_{t-1}
// are [unit][SP] (SP = S + 4: one 16-byte load gives four sequences, and the
// padding spreads the element-wise writes over the banks); the cell state and
// Hawkes gate are [sequence][unit], so the element-wise phase runs with the
// unit index fastest and its global loads and stores coalesce.  The input of
// step t + 1 is fetched during the element-wise phase of step t.  y = Wy h is
// left to k_lstm_out: it does not feed the recursion.
template <int S, bool ST>
__global__ void __launch_bounds__(S >= 16 ? 512 : 1024) k_lstm_fwd_s(LstmFwd a) {
  constexpr bool STG = ST;
  constexpr int SP = S + 4;
  extern __shared__ __align__(16) float sm[];
  const int H = a.H, D = a.D, G = 4 * H, ZP = G + 1, r = threadIdx.x, nt = blockDim.x;
  const int s0 = blockIdx.x * S;
  float *xs = sm;               // [2][D][SP]  x_t in buffer t & 1
  float *h = xs + 2 * D * SP;   // [H][SP]     h_{t-1}
  float *c = h + H * SP;        // [S][H]      c_{t-1}
  float *kh = c + S * H;        // [S][H]      Hawkes gate
  float *z = kh + S * H;        // [S][ZP]     gate activations of step t
  float *WT = z + S * ZP;       // [D][G]      (staged)
  float *UT = WT + D * G;       // [H][G]
  if (STG) {
    for (int p = r; p < G * D; p += nt) WT[(p % D) * G + p / D] = a.W[p];
    for (int p = r; p < G * H; p += nt) UT[(p % H) * G + p / H] = a.U[p];
  }
  const int MM = a.M * a.M;
  for (int p = r; p < S * H; p += nt) {
    const int s = p / H, j = p % H, q = s0 + s;
    float v = 0.f;
    if (q < a.B) {
      float acc = 0.f;
      for (int k = 0; k < MM; ++k) acc = fmaf(a.A[(int64_t)j * MM + k], a.alpha[(int64_t)q * MM + k], acc);
      for (int k = 0; k < a.nb; ++k)
        acc = fmaf(-a.Bm[(int64_t)j * a.nb + k], a.beta[(int64_t)q * a.nb + k] * a.T[q], acc);
      for (int k = 0; k < a.M; ++k) acc = fmaf(a.C[(int64_t)j * a.M + k], a.mu[(int64_t)q * a.M + k], acc);
      v = tanhf(acc);
      a.hks[(int64_t)q * H + j] = v;
    }
    kh[p] = v;
    c[p] = 0.f;
    h[j * SP + s] = 0.f;
  }
  for (int p = r; p < S * D; p += nt) {
    const int s = p / D, d = p % D, q = s0 + s;
    xs[d * SP + s] = q < a.B ? a.x[(int64_t)q * a.L * D + d] : 0.f;
  }
  __syncthreads();
  const float br = r < G ? a.b[r] : 0.f;
  const bool tanh_row = r >= 2 * H && r < 3 * H;
  // The block has at least 4H threads: a thread owns at most S/4 of the S*H
  // cells, and S/4 register slots cover the S*D inputs when D <= H (wider
  // inputs fetch the rest after the matvec).
  constexpr int XI = S / 4, CI = S / 4;
  for (int t = 0; t < a.L; ++t) {
    const float *xc = xs + (t & 1) * D * SP;
    float xr[XI];  // x_{t+1}, fetched now and stored after the matvec
#pragma unroll
    for (int i = 0; i < XI; ++i) {
      const int p = r + i * nt, s = p / D, q = s0 + s;
      xr[i] = (t + 1 < a.L && p < S * D && q < a.B) ? a.x[((int64_t)q * a.L + t + 1) * D + p % D] : 0.f;
    }
    if (r < G) {
      float acc[S];
#pragma unroll
      for (int e = 0; e < S; ++e) acc[e] = br;
      for (int d = 0; d < D; ++d) {
        const float w = STG ? WT[d * G + r] : a.W[(int64_t)r * D + d];
#pragma unroll
        for (int e = 0; e < S; e += 4) {
          const float4 v = *reinterpret_cast<const float4 *>(xc + d * SP + e);
          acc[e] = fmaf(w, v.x, acc[e]);
          acc[e + 1] = fmaf(w, v.y, acc[e + 1]);
          acc[e + 2] = fmaf(w, v.z, acc[e + 2]);
          acc[e + 3] = fmaf(w, v.w, acc[e + 3]);
        }
      }
#pragma unroll 4
      for (int k = 0; k < H; ++k) {
        const float w = STG ? UT[k * G + r] : a.U[(int64_t)r * H + k];
#pragma unroll
        for (int e = 0; e < S; e += 4) {
          const float4 v = *reinterpret_cast<const float4 *>(h + k * SP + e);
          acc[e] = fmaf(w, v.x, acc[e]);
          acc[e + 1] = fmaf(w, v.y, acc[e + 1]);
          acc[e + 2] = fmaf(w, v.z, acc[e + 2]);
          acc[e + 3] = fmaf(w, v.w, acc[e + 3]);
        }
      }
#pragma unroll
      for (int e = 0; e < S; ++e) {
        const float v = tanh_row ? tanh_fast(acc[e]) : sigm_fast(acc[e]);
        z[e * ZP + r] = v;
        if (s0 + e < a.B) a.gates[((int64_t)(s0 + e) * a.L + t) * G + r] = v;
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < CI; ++i) {
      const int p = r + i * nt;
      if (p >= S * H) break;
      const int s = p / H, j = p % H, q = s0 + s;
      const float *zs = z + s * ZP;
      const float cn = kh[p] * fmaf(zs[H + j], c[p], zs[j] * zs[2 * H + j]);
      const float hn = zs[3 * H + j] * tanh_fast(cn);
      c[p] = cn;
      h[j * SP + s] = hn;
      if (q < a.B) {
        const int64_t o = ((int64_t)q * a.L + t) * H + j;
        a.cs[o] = cn;
        a.hs[o] = hn;
      }
    }
    float *xn = xs + ((t + 1) & 1) * D * SP;
#pragma unroll
    for (int i = 0; i < XI; ++i) {
      const int p = r + i * nt;
      if (p < S * D) xn[(p % D) * SP + p / D] = xr[i];
    }
    for (int p = r + XI * nt; p < S * D; p += nt) {
      const int q = s0 + p / D;
      xn[(p % D) * SP + p / D] = (t + 1 < a.L && q < a.B) ? a.x[((int64_t)q * a.L + t + 1) * D + p % D] : 0.f;
    }
    __syncthreads();
  }
}

// y[r][o] = sum_j Wy[o][j] h[r][j] over the R = B L rows of h_seq: one warp
// per row, lanes over j, a shuffle reduction per output.
__global__ void k_lstm_out(const float *hs, const float *Wy, int64_t R, int H, int O, float *y) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = w0; row < R; row += nw) {
    const float *hr = hs + row * H;
    for (int o = 0; o < O; ++o) {
      float acc = 0.f;
      for (int j = lane; j < H; j += 32) acc = fmaf(Wy[(int64_t)o * H + j], hr[j], acc);
#pragma unroll
      for (int m = 16; m > 0; m >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
      if (lane == 0) y[row * O + o] = acc;
    }
  }
}

// Backward through time, S sequences per CTA.  The element-wise phase runs
// with the unit index fastest over [sequence][unit] state (coalesced global
// loads of the saved gates and cell states) and writes the gate gradients dz
// both to global memory (for the weight-gradient reduction) and, transposed,
// to dzT [G][SP].  The matvec phase computes [dh_{t-1}; dx_t] = [U | W]^T dz
// with thread (u, group) owning GW sequences of output unit u: one weight
// load and GW/4 16-byte loads of dzT feed GW FMAs.
template <int S, bool ST>
__global__ void __launch_bounds__(S >= 16 ? 512 : 1024) k_lstm_bwd_s(LstmBwd a) {
  constexpr bool STG = ST;
  constexpr int SP = S + 4, GW = S >= 16 ? 8 : 4;
  extern __shared__ __align__(16) float sm[];
  const int H = a.H, D = a.D, G = 4 * H, HD = H + D, r = threadIdx.x, nt = blockDim.x;
  const int s0 = blockIdx.x * S;
  float *dzT = sm;               // [G][SP]
  float *dh = dzT + G * SP;      // [S][H]  dh_t from later steps
  float *dcn = dh + S * H;       // [S][H]  dc_t from step t + 1
  float *dhk = dcn + S * H;      // [S][H]  d hks accumulated over steps
  float *kh = dhk + S * H;       // [S][H]
  float *V = kh + S * H;         // [G][HD] rows of [U | W] (staged)
  if (STG)
    for (int p = r; p < G * HD; p += nt) {
      const int g = p / HD, u = p % HD;
      V[p] = u < H ? a.U[(int64_t)g * H + u] : a.W[(int64_t)g * D + (u - H)];
    }
  for (int p = r; p < S * H; p += nt) {
    const int s = p / H, j = p % H, q = s0 + s;
    dh[p] = 0.f;
    dcn[p] = 0.f;
    dhk[p] = 0.f;
    kh[p] = q < a.B ? a.hks[(int64_t)q * H + j] : 0.f;
  }
  __syncthreads();
  const int items = HD * (S / GW);
  // The block has at least 4H threads: a thread owns at most S/4 of the S*H
  // cells.  Their saved gates, cell states and first output gradient for the
  // next step down are fetched into registers before the matvec phase.
  constexpr int CI = S / 4;
  float pf[CI][7];
  auto fetch = [&](int t) {
#pragma unroll
    for (int i = 0; i < CI; ++i) {
      const int p = r + i * nt, s = p / H, j = p % H, q = s0 + s;
      if (p < S * H && q < a.B) {
        const int64_t row = (int64_t)q * a.L + t;
        const float *gr = a.gates + row * G;
        pf[i][0] = gr[j];
        pf[i][1] = gr[H + j];
        pf[i][2] = gr[2 * H + j];
        pf[i][3] = gr[3 * H + j];
        pf[i][4] = a.cs[row * H + j];
        pf[i][5] = t > 0 ? a.cs[(row - 1) * H + j] : 0.f;
        pf[i][6] = a.O > 0 ? a.dy[row * a.O] : 0.f;
      }
    }
  };
  fetch(a.L - 1);
  for (int t = a.L - 1; t >= 0; --t) {
#pragma unroll
    for (int i = 0; i < CI; ++i) {
      const int p = r + i * nt;
      if (p >= S * H) break;
      const int s = p / H, j = p % H, q = s0 + s;
      if (q >= a.B) {
        dzT[j * SP + s] = dzT[(H + j) * SP + s] = dzT[(2 * H + j) * SP + s] = dzT[(3 * H + j) * SP + s] = 0.f;
        continue;
      }
      const int64_t row = (int64_t)q * a.L + t;
      float dht = dh[p];
      if (a.O > 0) dht = fmaf(a.Wy[j], pf[i][6], dht);
      for (int k = 1; k < a.O; ++k) dht = fmaf(a.Wy[(int64_t)k * H + j], a.dy[row * a.O + k], dht);
      const float ig = pf[i][0], fg = pf[i][1], gg = pf[i][2], og = pf[i][3];
      const float cv = pf[i][4], cp = pf[i][5];
      const float tc = tanh_fast(cv);
      const float dc = fmaf(dht * og, 1.f - tc * tc, dcn[p]);
      dhk[p] = fmaf(dc, fmaf(fg, cp, ig * gg), dhk[p]);
      const float din = dc * kh[p];
      const float zi = din * gg * ig * (1.f - ig);
      const float zf = din * cp * fg * (1.f - fg);
      const float zg = din * ig * (1.f - gg * gg);
      const float zo = dht * tc * og * (1.f - og);
      dzT[j * SP + s] = zi;
      dzT[(H + j) * SP + s] = zf;
      dzT[(2 * H + j) * SP + s] = zg;
      dzT[(3 * H + j) * SP + s] = zo;
      float *dzr = a.dz + row * G;
      dzr[j] = zi;
      dzr[H + j] = zf;
      dzr[2 * H + j] = zg;
      dzr[3 * H + j] = zo;
      dcn[p] = din * fg;
    }
    __syncthreads();
    if (t > 0) fetch(t - 1);
    for (int it = r; it < items; it += nt) {
      const int u = it % HD, sb = (it / HD) * GW;
      float acc[GW];
#pragma unroll
      for (int e = 0; e < GW; ++e) acc[e] = 0.f;
#pragma unroll 4
      for (int g = 0; g < G; ++g) {
        const float w = STG ? V[g * HD + u]
                                 : (u < H ? a.U[(int64_t)g * H + u] : a.W[(int64_t)g * D + (u - H)]);
#pragma unroll
        for (int e = 0; e < GW; e += 4) {
          const float4 v = *reinterpret_cast<const float4 *>(dzT + g * SP + sb + e);
          acc[e] = fmaf(w, v.x, acc[e]);
          acc[e + 1] = fmaf(w, v.y, acc[e + 1]);
          acc[e + 2] = fmaf(w, v.z, acc[e + 2]);
          acc[e + 3] = fmaf(w, v.w, acc[e + 3]);
        }
      }
      if (u < H) {
#pragma unroll
        for (int e = 0; e < GW; ++e) dh[(sb + e) * H + u] = acc[e];
      } else {
#pragma unroll
        for (int e = 0; e < GW; ++e)
          if (s0 + sb + e < a.B) a.dx[((int64_t)(s0 + sb + e) * a.L + t) * D + (u - H)] = acc[e];
      }
    }
    __syncthreads();
  }
  for (int p = r; p < S * H; p += nt) {
    const int s = p / H, j = p % H, q = s0 + s;
    if (q < a.B) a.dpre[(int64_t)q * H + j] = dhk[p] * (1.f - kh[p] * kh[p]);
  }
}

// Weight gradients of the gates in one pass over dz:
//   dW[g][d] += sum_r dz[r][g] x[r][d],  dU[g][k] += sum_r dz[r][g] h_{r-1}[k],
//   db[g] += sum_r dz[r][g]
// i.e. out[g][q] = sum_r dz[r][g] Bc[r][q] with Bc[r] = [x_r, h_{r-1}, 1]
// (h_{r-1} = 0 at the first step of a sequence).  A CTA owns a 64 x 80 tile
// of (g, q) over a chunk of rows, staged 32 rows at a time; thread (tg, tq)
// keeps a 4 x 5 register tile.  The next 32 rows are fetched into registers
// while the current ones are multiplied.  Chunks meet in the output by
// atomic adds.
constexpr int kWgG = 64, kWgQ = 80, kWgK = 32;
constexpr int kWgA = kWgK * kWgG / 4 / 256;  // float4 of dz per thread per stage
constexpr int kWgB = kWgK * kWgQ / 256;      // elements of Bc per thread per stage
static_assert(kWgK * kWgG / 4 == kWgA * 256 && kWgK * kWgQ == kWgB * 256, "stage split");

__global__ void __launch_bounds__(256) k_lstm_wgrad(const float *dz, const float *x, const float *hs,
                                                    int64_t R, int L, int D, int H, int64_t rows_per,
                                                    float *dW, float *dU, float *db) {
  __shared__ __align__(16) float As[kWgK][kWgG];
  __shared__ float Bs[kWgK][kWgQ + 1];
  const int G = 4 * H, Q = D + H + 1, tid = threadIdx.x;
  const int tg = tid & 15, tq = tid >> 4;
  const int g0 = blockIdx.x * kWgG, q0 = blockIdx.y * kWgQ;
  const int64_t r0 = blockIdx.z * rows_per, r1 = r0 + rows_per < R ? r0 + rows_per : R;
  float4 an[kWgA];
  float bn[kWgB];
  // rows rb .. rb + 31 into registers; m0 = step index of row rb in its sequence
  auto fetch = [&](int64_t rb, int m0) {
#pragma unroll
    for (int j = 0; j < kWgA; ++j) {
      const int e = tid + j * 256, rr = e / (kWgG / 4), c4 = (e % (kWgG / 4)) * 4;
      const int64_t rw = rb + rr;
      an[j] = (rw < r1 && g0 + c4 < G) ? *reinterpret_cast<const float4 *>(dz + rw * G + g0 + c4)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < kWgB; ++j) {
      const int e = tid + j * 256, rr = e / kWgQ, q = q0 + e % kWgQ;
      const int64_t rw = rb + rr;
      float v = 0.f;
      if (rw < r1 && q < Q) {
        if (q < D) {
          v = x[rw * D + q];
        } else if (q < D + H) {
          int m = m0 + rr;
          while (m >= L) m -= L;
          v = m ? hs[(rw - 1) * H + (q - D)] : 0.f;
        } else {
          v = 1.f;
        }
      }
      bn[j] = v;
    }
  };
  auto stage = [&]() {
#pragma unroll
    for (int j = 0; j < kWgA; ++j) {
      const int e = tid + j * 256;
      *reinterpret_cast<float4 *>(&As[e / (kWgG / 4)][(e % (kWgG / 4)) * 4]) = an[j];
    }
#pragma unroll
    for (int j = 0; j < kWgB; ++j) {
      const int e = tid + j * 256;
      Bs[e / kWgQ][e % kWgQ] = bn[j];
    }
  };
  float acc[4][5];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 5; ++k) acc[i][k] = 0.f;
  int m0 = (int)(r0 % L);
  const int mstep = kWgK % L;
  fetch(r0, m0);
  stage();
  __syncthreads();
  for (int64_t rb = r0; rb < r1; rb += kWgK) {
    const bool more = rb + kWgK < r1;
    m0 += mstep;
    if (m0 >= L) m0 -= L;
    if (more) fetch(rb + kWgK, m0);
#pragma unroll 8
    for (int k = 0; k < kWgK; ++k) {
      const float4 av = *reinterpret_cast<const float4 *>(&As[k][tg * 4]);
      const float a4[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const float bv = Bs[k][tq * 5 + c];
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i][c] = fmaf(a4[i], bv, acc[i][c]);
      }
    }
    __syncthreads();
    if (more) stage();
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int g = g0 + tg * 4 + i;
    if (g >= G) continue;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const int q = q0 + tq * 5 + c;
      if (q < D) atomicAdd(&dW[(int64_t)g * D + q], acc[i][c]);
      else if (q < D + H) atomicAdd(&dU[(int64_t)g * H + (q - D)], acc[i][c]);
      else if (q == D + H) atomicAdd(&db[g], acc[i][c]);
    }
  }
}

// out[p][q] (+)= scale * sum_{r < R} A(r, p) B(r, q), A(r, p) = A[r * lda + p],
// B(r, q) = B[r * ldb + q]; B == nullptr means B(r, q) = 1 (row sums).
// 16 x 16 output tiles, the rows split over gridDim.z slices, atomic adds.
__global__ void __launch_bounds__(256) k_atb(const float *A, int64_t lda, const float *Bp, int64_t ldb,
                                             int P, int Q, int64_t R, float scale,
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

int num_sms() {
  static int v = -1;
  if (v < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  }
  return v;
}

// Dynamic shared memory of the S-sequence kernels (S = 1: the one-sequence
// kernels), with the gate weights staged when they fit.
int fwd_smem(int S, int D, int H, bool staged) {
  const int G = 4 * H, SP = S + 4;
  const int base = S == 1 ? (D + 2 * H + G + H) * 4 : (2 * D * SP + H * SP + 2 * S * H + S * (G + 1)) * 4;
  return base + (staged ? (D + H) * G * 4 : 0);
}
int bwd_smem(int S, int D, int H, bool staged) {
  const int G = 4 * H, SP = S + 4;
  const int base = S == 1 ? (H + G) * 4 : (G * SP + 4 * S * H) * 4;
  return base + (staged ? (D + H) * G * 4 : 0);
}

template <typename K>
int resident(K kernel, int threads, int smem) {
  if (smem > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) n = 0;
  return n;
}

// Sequences per CTA: the S in {1, 4, 8, 16} that minimises waves x (S + 8),
// ties to the larger S.  A wave's time is modelled as a fixed part (barriers,
// the latency of each step's dependent chain, weight staging) worth about
// eight sequences' arithmetic plus a part linear in S; on GB300 at H = 64,
// D = 11 the measured fwd+bwd times for S = 1, 4, 8, 16 over 4,096
// sequences were 15.9, 11.2, 10.8 and 10.8 ms.  Both passes use the same S;
// the forward kernel's residency decides.  MDHP_LSTM_SEQ_PER_CTA (1, 4, 8,
// 16) overrides the choice where that S can run.
int pick_seq_per_cta(int B, int D, int H) {
  const int G = 4 * H, threads = (G + 31) / 32 * 32, lim = max_smem();
  int forced = 0;
  if (const char *e = getenv("MDHP_LSTM_SEQ_PER_CTA")) forced = atoi(e);
  int best = 1;
  double best_cost = 1e300;
  for (int S : {1, 4, 8, 16}) {
    if (S == 16 && threads > 512) continue;  // its register budget assumes <= 512 threads
    const bool stg = fwd_smem(S, D, H, true) <= lim;
    const int smem = fwd_smem(S, D, H, stg);
    if (smem > lim) continue;
    int res = 0;
    switch (S) {
      case 1: res = resident(k_lstm_fwd, threads, smem); break;
      case 4: res = stg ? resident(k_lstm_fwd_s<4, true>, threads, smem)
                        : resident(k_lstm_fwd_s<4, false>, threads, smem); break;
      case 8: res = stg ? resident(k_lstm_fwd_s<8, true>, threads, smem)
                        : resident(k_lstm_fwd_s<8, false>, threads, smem); break;
      default: res = stg ? resident(k_lstm_fwd_s<16, true>, threads, smem)
                         : resident(k_lstm_fwd_s<16, false>, threads, smem); break;
    }
    if (res < 1) continue;
    if (S == forced) return S;
    const int64_t blocks = ((int64_t)B + S - 1) / S, slots = (int64_t)res * num_sms();
    const double cost = (double)((blocks + slots - 1) / slots) * (S + 8);
    if (cost <= best_cost) {
      best_cost = cost;
      best = S;
    }
  }
  return best;
}

template <int S>
void launch_fwd(const LstmFwd &a0, int threads, cudaStream_t st) {
  LstmFwd a = a0;
  a.staged = fwd_smem(S, a.D, a.H, true) <= max_smem() ? 1 : 0;
  const int smem = fwd_smem(S, a.D, a.H, a.staged);
  auto k = a.staged ? k_lstm_fwd_s<S, true> : k_lstm_fwd_s<S, false>;
  if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k<<<(a.B + S - 1) / S, threads, smem, st>>>(a);
}

template <int S>
void launch_bwd(const LstmBwd &a0, int threads, cudaStream_t st) {
  LstmBwd a = a0;
  a.staged = bwd_smem(S, a.D, a.H, true) <= max_smem() ? 1 : 0;
  const int smem = bwd_smem(S, a.D, a.H, a.staged);
  auto k = a.staged ? k_lstm_bwd_s<S, true> : k_lstm_bwd_s<S, false>;
  if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k<<<(a.B + S - 1) / S, threads, smem, st>>>(a);
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
  const int threads = (G + 31) / 32 * 32;
  LstmFwd a{d->B, d->L, d->D, d->H, d->M, d->nb, d->O, 0, x, mu, alpha, beta, T_span, W, U, b, A,
            Bm, C, Wy, y, h_seq, c_seq, gates, hks};
  cudaStream_t st = (cudaStream_t)stream;
  const int S = pick_seq_per_cta(d->B, d->D, d->H);
  if (S > 1) {
    if (S == 4) launch_fwd<4>(a, threads, st);
    else if (S == 8) launch_fwd<8>(a, threads, st);
    else launch_fwd<16>(a, threads, st);
    if (d->O > 0) {
      const int64_t R = (int64_t)d->B * d->L;
      const int64_t want = (R + 7) / 8;
      const int blocks = (int)(want < (int64_t)num_sms() * 16 ? want : (int64_t)num_sms() * 16);
      k_lstm_out<<<blocks, 256, 0, st>>>(h_seq, Wy, R, d->H, d->O, y);
    }
    return launched("k_lstm_fwd_s / k_lstm_out");
  }
  a.staged = fwd_smem(1, d->D, d->H, true) <= max_smem() ? 1 : 0;
  const int smem = fwd_smem(1, d->D, d->H, a.staged);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_lstm_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_lstm_fwd<<<d->B, threads, smem, st>>>(a);
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
  const int threads = (G + 31) / 32 * 32;
  LstmBwd a{d->B, d->L, D, H, O, 0, W, U, Wy, h_seq, c_seq, gates, hks, dy, dz_work, dpre_work, dx};
  switch (pick_seq_per_cta(d->B, D, H)) {
    case 4: launch_bwd<4>(a, threads, st); break;
    case 8: launch_bwd<8>(a, threads, st); break;
    case 16: launch_bwd<16>(a, threads, st); break;
    default: {
      a.staged = bwd_smem(1, D, H, true) <= max_smem() ? 1 : 0;
      const int smem = bwd_smem(1, D, H, a.staged);
      if (smem > 48 * 1024) cudaFuncSetAttribute(k_lstm_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      k_lstm_bwd<<<d->B, threads, smem, st>>>(a);
    }
  }
  mdhp_status s = launched("k_lstm_bwd");
  if (s != MDHP_OK) return s;
  const int64_t R = (int64_t)d->B * d->L;
  auto atb = [&](const float *Ap, int64_t lda, const float *Bp, int64_t ldb, int P, int Q, int64_t rows,
                 float scale, float *out) {
    const int tiles = ((Q + 15) / 16) * ((P + 15) / 16);
    int64_t split = (int64_t)num_sms() * 8 / tiles;  // about 8 CTAs per SM over the rows
    const int64_t most = (rows + 31) / 32;
    split = split < 1 ? 1 : (split > most ? most : split);
    dim3 grid((Q + 15) / 16, (P + 15) / 16, (unsigned)split);
    k_atb<<<grid, 256, 0, st>>>(Ap, lda, Bp, ldb, P, Q, rows, scale, out);
  };
  {  // dW, dU, db in one pass over dz, chunks of rows filling one wave of CTAs
    const int gx = (G + kWgG - 1) / kWgG, gy = (D + H + 1 + kWgQ - 1) / kWgQ;
    int res = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&res, k_lstm_wgrad, 256, 0) != cudaSuccess || res < 1)
      res = 1;
    int64_t split = (int64_t)num_sms() * res / (gx * gy);
    split = split < 1 ? 1 : split;
    const int64_t tiles = (R + kWgK - 1) / kWgK;
    if (split > tiles) split = tiles;
    const int64_t rows_per = (tiles + split - 1) / split * kWgK;
    const dim3 grid(gx, gy, (unsigned)((R + rows_per - 1) / rows_per));
    k_lstm_wgrad<<<grid, 256, 0, st>>>(dz_work, x, h_seq, R, d->L, D, H, rows_per, dW, dU, db);
  }
  if (O > 0) atb(dy, O, h_seq, H, O, H, R, 1.f, dWy);  // dWy = sum_r dy_r^T h_r
  // Hawkes gate: dA, dBm, dC over sequences; d(alpha, beta, mu) per sequence
  atb(dpre_work, H, alpha, MM, H, MM, d->B, 1.f, dA);
  atb(dpre_work, H, mu, M, H, M, d->B, 1.f, dC);
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
  atb(dpre_work, H, dz_work, nb, H, nb, d->B, -1.f, dBm);
  return launched("lstm hawkes gradients");
}
