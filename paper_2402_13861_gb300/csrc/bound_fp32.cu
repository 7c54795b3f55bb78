// Float32 bound path: affine / probabilistic-affine forms propagated layer by layer through a ReLU
// MLP (Sec. III-B and IV-C), one kernel per step, cells processed in chunks.
//
// Per cell the form of the pre-activation z_j of hidden layer j is a centre c (w floats) and a
// coefficient matrix X with S_j = 3 + w (j - 1) rows (one per noise symbol) and w columns, stored
// row-major [cell][row][w] in float32:
//   z_1:  c = W_0 x_c + b_0, X = diag(h) W_0^T                      (input box, Eq. 3 / Eq. 8)
//   ReLU: alpha, beta, gamma per neuron from (c, r) or (mu, sigma)  (Eq. 4 / Eq. 9, Table VII)
//   L_j:  c' = W_j (alpha c + beta) + b_j,
//         X' = [X diag(alpha) W_j^T ; diag(gamma) W_j^T]           (Eq. 3 / Eq. 8)
//   out:  y_i = X diag(alpha) w_out (+ gamma_m w_out,m for the last ReLU's symbols),
//         r = sum |y_i| (Eq. 2) or sigma^2 = sum y_i^2 (Eq. 7), RA-UA: sigma^2 / 3 (Sec. IV-A).
//
// Rounding-error inflation (SOUND, inflate != 0).  The library carries, per neuron, a slack
// delta >= |true z - carried form| and widens the ReLU interval by it; the linearisation error,
// alpha * delta and the rounding of the new centre all go into the neuron's new symbol, so after
// every ReLU the carried form is exact again.  Float32 rounding of each step is bounded by
// standard error analysis: a K-term dot product errs by at most gamma_K sum |a_k b_k| with
// gamma_K = K u / (1 - K u), u = 2^-24; products alpha_k W_nk rounded once more add u.
#include "internal.cuh"

#include <string>
#include "linearise.cuh"
#include "cell_box.cuh"

#include <algorithm>
#include <cmath>

namespace isx {
namespace {

constexpr float kU = 5.9604645e-08f;        // 2^-24, float32 unit roundoff
constexpr float kSafe = 1.0000010f;         // (1 + 2^-20): slack for evaluating error formulas
constexpr float kInvSqrt3 = 0.57735026918962576f;

__host__ __device__ __forceinline__ float gamma_k(int k) { return (k * kU) / (1.0f - k * kU); }

// z_1 = W_0 x + b_0 over the box: centre, 3 coefficient rows, per-neuron reduction, slack.
__global__ void k_input_layer(CellSource src, int64_t first, int nc, const float* __restrict__ W0,
                              const float* __restrict__ b0, int w, int mode, int inflate, float* C,
                              float* X, int S, float* RAD, float* DELTA) {
  int cell = blockIdx.x;
  if (cell >= nc) return;
  float xc[3], h[3];
  cell_box(src, first + cell, inflate, xc, h);
  if (mode == ISX_BOUND_CLT)
    for (int d = 0; d < 3; ++d) h[d] *= kInvSqrt3;   // uniform on [-h, h] has std h / sqrt 3
  float* Xc = X + (size_t)cell * S * w;
  for (int n = threadIdx.x; n < w; n += blockDim.x) {
    float w0 = W0[3 * n], w1 = W0[3 * n + 1], w2 = W0[3 * n + 2];
    float c = fmaf(w2, xc[2], fmaf(w1, xc[1], fmaf(w0, xc[0], b0[n])));
    float x0 = h[0] * w0, x1 = h[1] * w1, x2 = h[2] * w2;
    Xc[n] = x0;
    Xc[w + n] = x1;
    Xc[2 * w + n] = x2;
    float rad;
    if (mode == ISX_BOUND_CLT) rad = sqrtf(x0 * x0 + x1 * x1 + x2 * x2);
    else rad = fabsf(x0) + fabsf(x1) + fabsf(x2);
    C[(size_t)cell * w + n] = c;
    RAD[(size_t)cell * w + n] = rad;
    if (inflate) {
      float e = fabsf(w0 * xc[0]) + fabsf(w1 * xc[1]) + fabsf(w2 * xc[2]) + fabsf(b0[n]);
      DELTA[(size_t)cell * w + n] = (5.0f * kU * e + 3.0f * kU * rad) * kSafe;
    } else {
      DELTA[(size_t)cell * w + n] = 0.0f;
    }
  }
}

// Activation linearisation per (cell, neuron); updates the centre in place, writes alpha and gamma.
__global__ void k_relu(int64_t total, int mode, int inflate, int act, float* C, const float* RAD,
                       const float* DELTA, float* ALPHA, float* GAMMA) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= total) return;
  Lin r = (mode == ISX_BOUND_CLT) ? act_clt(act, C[i], RAD[i])
                                  : relu_sound(C[i], RAD[i], inflate ? DELTA[i] : 0.0f, inflate != 0);
  C[i] = r.center;
  ALPHA[i] = r.alpha;
  GAMMA[i] = r.gamma;
}

// Centre of the next layer, c' = W a + b, and (inflate) the slack of the next pre-activation:
// kappa * sum_k |W_nk| (alpha_k r_k + gamma_k) + gamma_{K+1} (sum_k |W_nk a_k| + |b_n|).
__global__ void k_center_gemv(int nc, int win, int wout, const float* __restrict__ Wt,
                              const float* __restrict__ bias, float* C, const float* ALPHA,
                              const float* RAD, const float* GAMMA, float* DELTA, int inflate,
                              float kappa) {
  extern __shared__ float sh[];
  float* a = sh;             // a-form centre
  float* ra = sh + win;      // a-form radius
  int cell = blockIdx.x;
  if (cell >= nc) return;
  for (int k = threadIdx.x; k < win; k += blockDim.x) {
    size_t i = (size_t)cell * win + k;
    a[k] = C[i];
    ra[k] = inflate ? fmaf(ALPHA[i], RAD[i], GAMMA[i]) : 0.0f;
  }
  __syncthreads();
  for (int n = threadIdx.x; n < wout; n += blockDim.x) {
    float acc = bias[n], e = fabsf(bias[n]), g = 0.0f;
    for (int k = 0; k < win; ++k) {
      float wk = Wt[(size_t)k * wout + n];
      acc = fmaf(wk, a[k], acc);
      if (inflate) {
        e = fmaf(fabsf(wk), fabsf(a[k]), e);
        g = fmaf(fabsf(wk), ra[k], g);
      }
    }
    C[(size_t)cell * wout + n] = acc;
    if (inflate) DELTA[(size_t)cell * wout + n] = (kappa * g + gamma_k(win + 2) * e) * kSafe;
  }
}

// X_out[r] = X_in[r] diag(alpha) W^T for the S_in carried rows: BM x BN output tiles, K step 16,
// TM x TN outputs per thread.  Every output accumulates over K in the same order whatever the tile,
// so all variants give bit-identical results and the autotuner may pick any of them.
template <int BM, int BN, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN)) k_gemm_fp32(const float* __restrict__ Xin,
                                                                     float* __restrict__ Xout, int S_in, int S_out,
                                                                     int w, const float* __restrict__ Wt,
                                                                     const float* __restrict__ ALPHA) {
  constexpr int T = (BM / TM) * (BN / TN), TX = BN / TN;
  static_assert(TN % 4 == 0, "float4 stores");
  __shared__ float As[16][BM + 4];
  __shared__ float Bs[16][BN];
  const int cell = blockIdx.z;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const float* A = Xin + (size_t)cell * S_in * w;
  const float* al = ALPHA + (size_t)cell * w;
  float* Y = Xout + (size_t)cell * S_out * w;
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  float acc[TM][TN] = {};
  for (int k0 = 0; k0 < w; k0 += 16) {
    for (int q = tid; q < BM * 4; q += T) {
      const int row = q >> 2, kq = (q & 3) * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (m0 + row < S_in) v = *reinterpret_cast<const float4*>(A + (size_t)(m0 + row) * w + k0 + kq);
      As[kq + 0][row] = v.x; As[kq + 1][row] = v.y; As[kq + 2][row] = v.z; As[kq + 3][row] = v.w;
    }
    for (int q = tid; q < 4 * BN; q += T) {
      const int kk = q / (BN / 4), nq = (q % (BN / 4)) * 4;
      float4 bv = make_float4(0.f, 0.f, 0.f, 0.f);
      if (n0 + nq < w) bv = *reinterpret_cast<const float4*>(Wt + (size_t)(k0 + kk) * w + n0 + nq);
      const float sc = al[k0 + kk];
      Bs[kk][nq + 0] = bv.x * sc; Bs[kk][nq + 1] = bv.y * sc; Bs[kk][nq + 2] = bv.z * sc; Bs[kk][nq + 3] = bv.w * sc;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int r = m0 + ty * TM + i;
#pragma unroll
    for (int jc = 0; jc < TN; jc += 4) {
      const int c = n0 + tx * TN + jc;
      if (r < S_in && c < w)
        *reinterpret_cast<float4*>(Y + (size_t)r * w + c) =
            make_float4(acc[i][jc], acc[i][jc + 1], acc[i][jc + 2], acc[i][jc + 3]);
    }
  }
}

// Tile variants of the FP32 coefficient GEMM the autotuner chooses from.
struct GemmShape {
  int bm, bn;
  const char* name;
};
constexpr GemmShape kGemmShapes[] = {{64, 64, "64x64/4x4"}, {32, 64, "32x64/2x4"}, {16, 64, "16x64/1x4"},
                                     {128, 64, "128x64/8x4"}, {64, 128, "64x128/4x8"}};
constexpr int kGemmVariants = sizeof(kGemmShapes) / sizeof(kGemmShapes[0]);

void launch_gemm(int v, int nc, int S, int S_out, int w, const float* Xa, float* Xb, const float* Wt,
                 const float* AL, cudaStream_t st) {
  const GemmShape g = kGemmShapes[v];
  const dim3 grid((w + g.bn - 1) / g.bn, (S + g.bm - 1) / g.bm, nc);
  switch (v) {
    case 0: k_gemm_fp32<64, 64, 4, 4><<<grid, 256, 0, st>>>(Xa, Xb, S, S_out, w, Wt, AL); break;
    case 1: k_gemm_fp32<32, 64, 2, 4><<<grid, 256, 0, st>>>(Xa, Xb, S, S_out, w, Wt, AL); break;
    case 2: k_gemm_fp32<16, 64, 1, 4><<<grid, 256, 0, st>>>(Xa, Xb, S, S_out, w, Wt, AL); break;
    case 3: k_gemm_fp32<128, 64, 8, 4><<<grid, 256, 0, st>>>(Xa, Xb, S, S_out, w, Wt, AL); break;
    default: k_gemm_fp32<64, 128, 4, 8><<<grid, 256, 0, st>>>(Xa, Xb, S, S_out, w, Wt, AL); break;
  }
}

// Rows of the symbols created by the last ReLU: X_out[S_in + m][n] = gamma_m W[n][m].
__global__ void k_fresh_rows(float* Xout, int S_in, int S_out, int w, const float* __restrict__ Wt,
                             const float* __restrict__ GAMMA) {
  int cell = blockIdx.y, m = blockIdx.x;
  float g = GAMMA[(size_t)cell * w + m];
  float* Y = Xout + ((size_t)cell * S_out + S_in + m) * w;
  for (int n = threadIdx.x; n < w; n += blockDim.x) Y[n] = g * Wt[(size_t)m * w + n];
}

// Per-neuron reduction over all rows (compensated): r = sum |x| (sound) or sigma = sqrt(sum x^2).
__global__ void k_reduce(const float* X, int S, int w, int mode, float* RAD) {
  int cell = blockIdx.x;
  const float* Xc = X + (size_t)cell * S * w;
  for (int n = threadIdx.x; n < w; n += blockDim.x) {
    float s = 0.0f, comp = 0.0f;
    for (int r = 0; r < S; ++r) {
      float x = Xc[(size_t)r * w + n];
      float v = (mode == ISX_BOUND_CLT) ? x * x : fabsf(x);
      float y = v - comp;
      float t = s + y;
      comp = (t - s) - y;
      s = t;
    }
    RAD[(size_t)cell * w + n] = (mode == ISX_BOUND_CLT) ? sqrtf(s) : s;
  }
}

// Output layer w -> 1 and the read-off.  One block per cell, one warp per coefficient row.
__global__ void __launch_bounds__(256) k_output(const float* X, int S, int w, const float* C,
                                                const float* ALPHA, const float* GAMMA,
                                                const float* RAD, const float* __restrict__ wout,
                                                float bout, int mode, int inflate, float* center,
                                                float* spread, int64_t first) {
  __shared__ float s_aw[1024];
  __shared__ float red[2][8];
  int cell = blockIdx.x;
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float* al = ALPHA + (size_t)cell * w;
  for (int n = threadIdx.x; n < w; n += blockDim.x) s_aw[n] = al[n] * wout[n];
  __syncthreads();
  bool sq = (mode != ISX_BOUND_SOUND);
  // carried rows
  float s = 0.0f, comp = 0.0f;
  const float* Xc = X + (size_t)cell * S * w;
  for (int r = warp; r < S; r += 8) {
    float y = 0.0f;
    for (int n = lane; n < w; n += 32) y = fmaf(Xc[(size_t)r * w + n], s_aw[n], y);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
    float v = sq ? y * y : fabsf(y);
    float yy = v - comp, t = s + yy;
    comp = (t - s) - yy;
    s = t;
  }
  // symbols of the last ReLU: y_m = gamma_m w_m
  float s2 = 0.0f, e = 0.0f, g = 0.0f, y0 = 0.0f;
  for (int m = threadIdx.x; m < w; m += blockDim.x) {
    size_t i = (size_t)cell * w + m;
    float y = GAMMA[i] * wout[m];
    s2 += sq ? y * y : fabsf(y);
    y0 = fmaf(wout[m], C[i], y0);
    if (inflate) {
      e = fmaf(fabsf(wout[m]), fabsf(C[i]), e);
      g = fmaf(fabsf(wout[m]), fmaf(ALPHA[i], RAD[i], GAMMA[i]), g);
    }
  }
  // block reductions (the warp-row sums live in lane 0 of each warp)
  float part = (lane == 0 ? s : 0.0f) + s2;
  float vals[4] = {part, y0, e, g};
  float tot[4];
  for (int q = 0; q < 4; ++q) {
    float v = vals[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[0][warp] = v;
    __syncthreads();
    float acc = 0.0f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) acc += red[0][k];
    tot[q] = acc;
  }
  if (threadIdx.x == 0) {
    float x0 = tot[1] + bout;
    float sp;
    if (mode == ISX_BOUND_SOUND) {
      sp = tot[0];
      if (inflate) {
        float ge = gamma_k(w + 1) + kU;
        sp = __fadd_ru(__fmul_ru(sp, kSafe), (ge * tot[3] + gamma_k(w + 2) * (tot[2] + fabsf(bout))) * 1.01f);
      }
    } else if (mode == ISX_BOUND_CLT) {
      sp = sqrtf(tot[0]);
    } else {
      sp = sqrtf(tot[0] / 3.0f);
    }
    center[first + cell] = x0;
    spread[first + cell] = sp;
  }
}

}  // namespace

isx_status bound_fp32(isx_inr inr, const CellSource& src, int64_t n, isx_bound_mode mode,
                      int inflate, float* d_center, float* d_spread, cudaStream_t st) {
  if (n <= 0) return ISX_OK;
  const int w = inr->w, H = inr->H;
  if (mode != ISX_BOUND_SOUND) inflate = 0;
  const int Smax = 3 + w * (H - 1);
  // chunk so that the two coefficient buffers stay within ~6 GB
  size_t per_cell = 2ull * Smax * w * sizeof(float);
  int64_t nc_max = std::max<int64_t>(1, (int64_t)((6ull << 30) / per_cell));
  nc_max = std::min<int64_t>(nc_max, 1 << 16);
  int64_t nc_alloc = std::min<int64_t>(n, nc_max);
  auto& ws = inr->ws;
  ISX_TRY(ws[WS_X0].ensure((size_t)nc_alloc * Smax * w * sizeof(float), "X0"));
  ISX_TRY(ws[WS_X1].ensure((size_t)nc_alloc * Smax * w * sizeof(float), "X1"));
  for (Slot s : {WS_C, WS_RAD, WS_ALPHA, WS_GAMMA, WS_DELTA})
    ISX_TRY(ws[s].ensure((size_t)nc_alloc * w * sizeof(float), "per-neuron"));
  float* C = ws[WS_C].as<float>();
  float* RAD = ws[WS_RAD].as<float>();
  float* AL = ws[WS_ALPHA].as<float>();
  float* GA = ws[WS_GAMMA].as<float>();
  float* DE = ws[WS_DELTA].as<float>();
  const int bt = std::min(w, 256);
  for (int64_t first = 0; first < n; first += nc_alloc) {
    int nc = (int)std::min<int64_t>(nc_alloc, n - first);
    float* Xa = ws[WS_X0].as<float>();
    float* Xb = ws[WS_X1].as<float>();
    int S = 3;
    {
      prof::Scope _ps(K_INPUT, st, 0, 0);
      k_input_layer<<<nc, bt, 0, st>>>(src, first, nc, inr->W[0], inr->b[0], w, (int)mode, inflate, C, Xa, S,
                                       RAD, DE);
    }
    ISX_LAUNCH_CHECK("k_input_layer");
    int64_t tot = (int64_t)nc * w;
    for (int j = 1; j <= H - 1; ++j) {
      {
        prof::Scope _ps(K_RELU, st, 0, 0);
        k_relu<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(tot, (int)mode, inflate, inr->act, C, RAD, DE, AL, GA);
      }
      ISX_LAUNCH_CHECK("k_relu");
      float kappa = 3.0f * kU + gamma_k(w);
      {
        prof::Scope _ps(K_GEMV, st, 2.0 * nc * w * w, 0);
        k_center_gemv<<<nc, bt, 2 * w * sizeof(float), st>>>(nc, w, w, inr->Wt[j], inr->b[j], C, AL, RAD, GA, DE,
                                                            inflate, kappa);
      }
      ISX_LAUNCH_CHECK("k_center_gemv");
      int S_out = S + w;
      // the coefficient buffers are laid out with the final stride S_out per cell; the tile shape
      // comes from the autotuner (timed once per width and row-count bucket)
      {
        int bucket = 1;
        while (bucket < S) bucket <<= 1;
        const std::string key = "gemm_fp32 w=" + std::to_string(w) + " rows<=" + std::to_string(bucket);
        const float* Wt = inr->Wt[j];
        auto run = [&](int v) -> isx_status {
          launch_gemm(v, nc, S, S_out, w, Xa, Xb, Wt, AL, st);
          ISX_LAUNCH_CHECK("k_gemm_fp32");
          return ISX_OK;
        };
        int v = 0;
        ISX_TRY(tune::pick(key, kGemmVariants, [&](int i) { return kGemmShapes[i].name; }, run, st, &v));
        prof::Scope _ps(K_GEMM_FP32, st, 2.0 * nc * (double)S * w * w, 8.0 * nc * (double)S * w);
        ISX_TRY(run(v));
      }
      {
        prof::Scope _ps(K_FRESH, st, 0, 4.0 * nc * w * w);
        k_fresh_rows<<<dim3(w, nc), bt, 0, st>>>(Xb, S, S_out, w, inr->Wt[j], GA);
      }
      ISX_LAUNCH_CHECK("k_fresh_rows");
      {
        prof::Scope _ps(K_REDUCE, st, 0, 4.0 * nc * (double)S_out * w);
        k_reduce<<<nc, bt, 0, st>>>(Xb, S_out, w, (int)mode, RAD);
      }
      ISX_LAUNCH_CHECK("k_reduce");
      std::swap(Xa, Xb);
      S = S_out;
    }
    {
      prof::Scope _ps(K_RELU, st, 0, 0);
      k_relu<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(tot, (int)mode, inflate, inr->act, C, RAD, DE, AL, GA);
    }
    ISX_LAUNCH_CHECK("k_relu");
    const int L = inr->n_layers - 1;
    float bout = inr->hb[L][0];
    {
      prof::Scope _ps(K_OUTPUT, st, 2.0 * nc * (double)S * w, 4.0 * nc * (double)S * w);
      k_output<<<nc, 256, 0, st>>>(Xa, S, w, C, AL, GA, RAD, inr->W[L], bout, (int)mode, inflate, d_center,
                                   d_spread, first);
    }
    ISX_LAUNCH_CHECK("k_output");
  }
  return ISX_OK;
}

}  // namespace isx
