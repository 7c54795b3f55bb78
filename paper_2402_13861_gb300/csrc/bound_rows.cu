// Row-batched tensor-core bounds: the layer loop of Sec. III-B / IV-C run layer-synchronously over a
// chunk of cells, with the noise-symbol rows of all cells of the chunk in one matrix per layer.
//
// Per cell the pre-activation z_j carries a centre c (w floats), the three input-symbol rows I
// (3 x w, float32) and the rows of the symbols created by earlier activations
// (bfloat16, "G rows").  Through activation j and linear layer j (Eq. 4 / 9, then Eq. 3 / 8):
//   a = alpha c + beta,  c' = W_j a + b_j,  I' = (I diag(alpha)) W_j^T   (tensor cores, two-term bf16)
//   G' = (G diag(alpha)) W_j^T                                          (one tcgen05 GEMM, all cells)
//   new rows gamma_n W_j[:, n] for every neuron with gamma_n != 0       (appended after the cell's G')
// A symbol whose coefficient gamma_n is exactly 0 (a neuron whose interval or Gaussian lies on
// one side of the kink) has an all-zero row in every later layer, so it is never created: the
// result is the full propagation's up to the order of the reductions.  At the finest levels of the
// scientific workload only 6-20 % of the neurons per layer create a symbol.
//
// alpha is applied to the A operand (the rows) while it is staged into shared memory, so the B
// operand is W_j itself, loaded once per CTA and shared by the rows of every cell: rows of many
// cells fill each 128-row MMA tile (rows_gemm.cu).  Per chunk and layer this file runs:
//   k_rows_input_act / k_rows_reduce_act: r = sum |x| (sound) or sigma^2 = sum x^2 (UP) per (cell,
//     neuron) over the stored rows and the input rows, the linearisation of the next activation,
//     the split A operand of the centre GEMM and the next per-cell row count;
//   k_rows_scan_*: row offsets of the next layer (the host reads the total to size the buffers);
//   the row GEMM, k_rows_new (the new rows) and k_rows_split (centre and input rows);
// and, after the last layer, k_rows_output: the output coefficient of every symbol is its row .
// (alpha_H * w_out), read off as sum |y| or sum y^2.
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <cuda_bf16.h>

#include "cell_box.cuh"
#include "linearise.cuh"
#include "tc_ptx.cuh"
#include "rows.cuh"

namespace isx {
namespace {

using namespace tc;

constexpr int64_t kMaxChunkCells = 1 << 19;     // cells per chunk of the layer-synchronous loop
using rows::kRT;
using rows::roff;
using rows::rwait;

// Rounding-error inflation of the sound bound (inflate != 0).  The carried form of a pre-activation
// is exact up to a per-neuron slack d >= |true z - carried form|.  The ReLU interval is widened by it
// and alpha d goes into the neuron's new symbol together with the linearisation error (relu_sound,
// as in the float32 path), so after every ReLU the carried form is exact again and the error symbols
// propagate through W with their signs, like every other symbol.  (Carrying alpha d on as a separate
// bound through |W| would lose the cancellation of every later layer: on a 256-wide net the bound
// then grows by the ratio sum |W| |x| / |sum W x| per layer.)  A neuron on the linear side with
// d > 0 therefore creates a symbol; a dead one (alpha = 0) does not.  A hidden linear layer j makes
// the slack of the next pre-activation
//   d' = |W_j| v,  v = alpha (kappa_g r_G + kappa_i r_I) + kappa_c |a|,
// plus the rounding of the stored result, store * r'_G, and kappa_c |b|.  r_G, r_I are
// the sums of |x| over the stored symbol rows (bf16) and the three input rows; kappa_g bounds the
// symbol-row GEMM (the A operand x alpha rounded to float32 and then bf16, W_j in bf16, tensor-core
// accumulation with unit roundoff u_a), kappa_i the two-term products of the centre and the input
// rows (3 2^-16 per product, u_a accumulation of 3 K products).  With inflation the centre c' = W_j a
// + b_j is computed in float32 on the CUDA cores (k_center_fp32), one fused multiply-add chain per
// output, so its error is kappa_c (sum_k |W_nk a_k| + |b_n|), kappa_c = gamma_{K+1}(u): the tensor
// cores' accumulation bound would give the centre an error that does not shrink with the cell.
// Its |a| term rides in v (v = ... + kappa_c |a|), its |b| term is added by the combine.  |W_j| v is
// itself a tensor-core GEMM
// with both operands rounded up to bf16 (non-negative, so the exact sum is below the rounded one up
// to the accumulation error, the factor gemm_slack).  The output layer adds the float32 dot products'
// errors (see k_rows_output).  Constants as in set_infl; u_a = 2^-17 is a conservative unit roundoff
// for tensor-core float32 accumulation.
struct Infl {
  int on = 0;
  float kappa_g = 0, kappa_i = 0, kappa_c = 0, store = 0, gemm_slack = 1, sum_g = 1;
  float gamma_w = 0;                            // gamma_{w+1}(u): the output layer's float32 dot products
  const float* bias = nullptr;                  // [w] b_j of the layer whose centre the combine reads
  __nv_bfloat16* V = nullptr;                   // [nc][w] v, rounded up: A operand of the bound GEMM
  const float* D = nullptr;                     // [nc][w] |W_j| v of the previous layer
  float* RAD = nullptr;                         // [nc][w] after the last hidden layer: radius bound
  float* SLK = nullptr;                         // [nc][w] after the last hidden layer: alpha d
};
constexpr float kU32 = 5.9604645e-08f;           // 2^-24
inline float gamma_u(double k, double u) { return (float)((k * u) / (1.0 - k * u)); }   // host only
void set_infl(Infl& f, int w) {
  const double ub = 1.0 / 256.0, u = 1.0 / 16777216.0, ua = 1.0 / 131072.0, K = w;
  f.kappa_g = (float)((1.0 + ub + u) * (1.0 + ub) * (1.0 + gamma_u(K, ua)) - 1.0) * 1.0001f;
  f.kappa_i = (float)(3.0 / 65536.0 * (1.0 + 2.0 * ub) + gamma_u(3.0 * K, ua) * (1.0 + ub) * (1.0 + ub) * (1.0 + ub) + u)
              * 1.0001f;
  f.kappa_c = gamma_u(K + 1.0, u) * 1.0001f;
  f.store = (float)(ub / (1.0 - ub) + 2.0 * u) * 1.0001f;
  f.gemm_slack = (float)(1.0 + 2.0 * gamma_u(K, ua)) * 1.0001f;
  f.sum_g = (float)(1.0 + gamma_u(132.0, u) + 8.0 * u);
  f.gamma_w = gamma_u(K + 1.0, u) * 1.0001f;
}
__device__ __forceinline__ __nv_bfloat16 bf16_up(float x) { return __float2bfloat16_ru(x); }

// ---- layer 0 and activation 1: centre c_1, the three input rows I_1 = diag(h) W_0^T (written: the
//      output layer of a one-hidden-layer net reads them), their reduction, the linearisation, the
//      split A operand of the first centre / input-row GEMM (when AH is given) and the row count of
//      the first stored block.  w / 2 threads per cell, two adjacent neurons per thread. ----
__global__ void __launch_bounds__(256) k_rows_input_act(CellSource src, int64_t first, int nc, int w, int mode,
                                                        int act, const float* __restrict__ W0,
                                                        const float* __restrict__ b0, float* I, float* A, float* AL,
                                                        float* GA, int* cnt_out, __nv_bfloat16* AH,
                                                        __nv_bfloat16* ALO, Infl infl) {
  __shared__ int mcount[8];
  const int tpc = w / 2, cpb = blockDim.x / tpc;
  const int sub = threadIdx.x / tpc, n = 2 * (threadIdx.x - sub * tpc);
  const int64_t cell = (int64_t)blockIdx.x * cpb + sub;
  if (threadIdx.x < 8) mcount[threadIdx.x] = 0;
  __syncthreads();
  const bool valid = sub < cpb && cell < nc;
  const bool clt = mode == ISX_BOUND_CLT;
  int m = 0;
  if (valid) {
    float xc[3], h[3];
    cell_box(src, first + cell, infl.on, xc, h);
    if (clt)
      for (int d = 0; d < 3; ++d) h[d] *= 0.57735026918962576f;   // uniform on [-h, h] has std h / sqrt 3
    Lin L[2];
    float iv[2][3];
    for (int e = 0; e < 2; ++e) {
      const int nn = n + e;
      const float w0 = W0[3 * nn], w1 = W0[3 * nn + 1], w2 = W0[3 * nn + 2];
      const float c = fmaf(w2, xc[2], fmaf(w1, xc[1], fmaf(w0, xc[0], b0[nn])));
      iv[e][0] = h[0] * w0;
      iv[e][1] = h[1] * w1;
      iv[e][2] = h[2] * w2;
      const float rad = clt ? sqrtf(iv[e][0] * iv[e][0] + iv[e][1] * iv[e][1] + iv[e][2] * iv[e][2])
                            : fabsf(iv[e][0]) + fabsf(iv[e][1]) + fabsf(iv[e][2]);
      if (infl.on) {
        // c: three fused multiply-adds; the input rows: one product each
        const float ru = __fmul_ru(rad, 1.0f + 4.0f * kU32);
        const float ex = fabsf(w0 * xc[0]) + fabsf(w1 * xc[1]) + fabsf(w2 * xc[2]) + fabsf(b0[nn]);
        const float dl = __fmul_ru(__fadd_ru(__fmul_ru(5.0f * kU32, ex), __fmul_ru(3.0f * kU32, ru)), 1.0000010f);
        L[e] = relu_sound(c, ru, dl, true);          // the slack is folded into the new symbol
        const size_t o = (size_t)cell * w + nn;
        if (infl.V) {
          float v = __fmul_ru(infl.kappa_i, __fmul_ru(L[e].alpha, ru));
          v = __fadd_ru(v, __fmul_ru(infl.kappa_c, fabsf(L[e].center)));
          infl.V[o] = bf16_up(v);
        } else {
          infl.RAD[o] = ru;
          infl.SLK[o] = 0.0f;
        }
      } else {
        L[e] = clt ? act_clt(act, c, rad) : relu_sound(c, rad, 0.0f, false);
      }
    }
    const size_t o = (size_t)cell * w + n;
    for (int d = 0; d < 3; ++d)
      *reinterpret_cast<float2*>(I + ((size_t)cell * 3 + d) * w + n) = make_float2(iv[0][d], iv[1][d]);
    *reinterpret_cast<float2*>(A + o) = make_float2(L[0].center, L[1].center);
    *reinterpret_cast<float2*>(AL + o) = make_float2(L[0].alpha, L[1].alpha);
    *reinterpret_cast<float2*>(GA + o) = make_float2(L[0].gamma, L[1].gamma);
    m = (L[0].gamma != 0.0f) + (L[1].gamma != 0.0f);
    if (AH) {
      auto put = [&](size_t i, float v0, float v1) {
        const __nv_bfloat162 hh = __floats2bfloat162_rn(v0, v1);
        const float2 hf = __bfloat1622float2(hh);
        const __nv_bfloat162 ll = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
        *reinterpret_cast<__nv_bfloat162*>(AH + i) = hh;
        *reinterpret_cast<__nv_bfloat162*>(ALO + i) = ll;
      };
      const size_t r0 = (size_t)cell * 4 * w + n;
      put(r0, L[0].center, L[1].center);
      for (int d = 0; d < 3; ++d) put(r0 + (size_t)(d + 1) * w, L[0].alpha * iv[0][d], L[1].alpha * iv[1][d]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
  if ((threadIdx.x & 31) == 0 && valid) atomicAdd(&mcount[sub], m);   // a warp never spans two cells
  __syncthreads();
  if (valid && threadIdx.x - sub * tpc == 0) cnt_out[cell] = mcount[sub];
}

// Exclusive scan of the per-cell row counts into int64 row offsets, total to *d_total: block sums
// of 1024 counts, one block scanning the sums, then every block's scan plus its offset.
constexpr int kScanB = 1024;
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* wsum, int64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int64_t s = wsum[lane];
    int64_t si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t t = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += t;
    }
    wsum[lane] = si - s;
    if (lane == 31) *total = si;
  }
  __syncthreads();
  return wsum[warp] + incl - v;
}
__global__ void __launch_bounds__(kScanB) k_rows_scan_sums(const int* cnt, int64_t nc, int64_t* bsum) {
  __shared__ int64_t wsum[32];
  __shared__ int64_t total;
  const int64_t i = (int64_t)blockIdx.x * kScanB + threadIdx.x;
  block_excl_scan(i < nc ? cnt[i] : 0, wsum, &total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}
__global__ void __launch_bounds__(kScanB) k_rows_scan_top(int64_t* bsum, int64_t nb, int64_t* d_total) {
  __shared__ int64_t wsum[32];
  __shared__ int64_t total;
  int64_t carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += kScanB) {
    const int64_t i = b0 + threadIdx.x;
    const int64_t v = i < nb ? bsum[i] : 0;
    const int64_t e = block_excl_scan(v, wsum, &total);
    if (i < nb) bsum[i] = carry + e;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) *d_total = carry;
}
__global__ void __launch_bounds__(kScanB) k_rows_scan_apply(const int* cnt, int64_t nc, const int64_t* bsum,
                                                            int64_t* off) {
  __shared__ int64_t wsum[32];
  __shared__ int64_t total;
  const int64_t i = (int64_t)blockIdx.x * kScanB + threadIdx.x;
  const int64_t e = block_excl_scan(i < nc ? cnt[i] : 0, wsum, &total);
  if (i < nc) off[i] = bsum[blockIdx.x] + e;
}

// ---- new rows gamma_n W_j[:, n] (row n of W_j^T) after each cell's transformed rows, in
//      increasing n; the row -> cell map of the whole output; and, per cell and column, the sum of
//      f(x) over the cell's new rows (x = the stored bf16 value; f = x^2 or |x|).  One warp per cell:
//      the neurons with gamma != 0 come from ballots, and each row goes out as one warp-wide store
//      (w / 32 columns per lane, whose sums the lane keeps in registers). ----
constexpr int kNewWarps = 8;
template <int CPL>
struct NewRowIO;
template <>
struct NewRowIO<8> {
  static __device__ __forceinline__ void ld(const float* p, float* v) {
    const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, const uint32_t* h) {
    *reinterpret_cast<uint4*>(p) = make_uint4(h[0], h[1], h[2], h[3]);
  }
};
template <>
struct NewRowIO<16> {
  static __device__ __forceinline__ void ld(const float* p, float* v) {
#pragma unroll
    for (int i = 0; i < 16; i += 4) {
      const float4 a = *reinterpret_cast<const float4*>(p + i);
      v[i] = a.x; v[i + 1] = a.y; v[i + 2] = a.z; v[i + 3] = a.w;
    }
  }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, const uint32_t* h) {
    *reinterpret_cast<uint4*>(p) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(p + 8) = make_uint4(h[4], h[5], h[6], h[7]);
  }
};
template <>
struct NewRowIO<4> {
  static __device__ __forceinline__ void ld(const float* p, float* v) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, const uint32_t* h) {
    *reinterpret_cast<uint2*>(p) = make_uint2(h[0], h[1]);
  }
};
template <>
struct NewRowIO<2> {
  static __device__ __forceinline__ void ld(const float* p, float* v) {
    const float2 a = *reinterpret_cast<const float2*>(p);
    v[0] = a.x; v[1] = a.y;
  }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, const uint32_t* h) { *reinterpret_cast<uint32_t*>(p) = h[0]; }
};
template <int CPL>
__global__ void __launch_bounds__(32 * kNewWarps) k_rows_new(int nc, int sq, const float* __restrict__ GA,
                                                             const float* __restrict__ Wt, const int* cnt_in,
                                                             const int64_t* off_out, const int* cnt_out,
                                                             __nv_bfloat16* xout, int* rowcell_out, float* pnew) {
  constexpr int w = 32 * CPL;
  using IO = NewRowIO<CPL>;
  const int lane = threadIdx.x & 31;
  const int cell = blockIdx.x * kNewWarps + (threadIdx.x >> 5);
  if (cell >= nc) return;
  const int64_t o0 = off_out[cell];
  const int co = cnt_out[cell];
  for (int r = lane; r < co; r += 32) rowcell_out[o0 + r] = cell;
  const int m0 = lane * CPL;                       // this lane's columns m0 .. m0 + CPL - 1
  float acc[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) acc[c] = 0.0f;
  int64_t row = o0 + cnt_in[cell];
  // one new row: x = bf16(gamma_n W_j[m, n]) for this lane's columns m, stored with one vector store
  auto emit = [&](float g, const float* v) {
    uint32_t h[CPL / 2];
#pragma unroll
    for (int c = 0; c < CPL; c += 2) {
      const __nv_bfloat162 x = __floats2bfloat162_rn(g * v[c], g * v[c + 1]);
      h[c / 2] = *reinterpret_cast<const uint32_t*>(&x);
      const float2 f = __bfloat1622float2(x);
      acc[c] += sq ? f.x * f.x : fabsf(f.x);
      acc[c + 1] += sq ? f.y * f.y : fabsf(f.y);
    }
    IO::st(xout + row * w + m0, h);
    ++row;
  };
  // gamma of all w neurons, loaded together into shared memory with one ballot mask per 32; then,
  // group by group, the new rows in increasing neuron order, NF rows' weight loads in flight (the
  // group loop is not unrolled: one copy of the row code keeps the kernel small)
  constexpr int NF = CPL >= 16 ? 2 : 4;
  __shared__ float sgam[kNewWarps][w];
  __shared__ unsigned smask[kNewWarps][CPL];
  const int wi = threadIdx.x >> 5;
#pragma unroll
  for (int g = 0; g < CPL; ++g) {
    const float x = GA[(size_t)cell * w + 32 * g + lane];
    sgam[wi][32 * g + lane] = x;
    const unsigned bm = __ballot_sync(0xffffffffu, x != 0.0f);
    if (lane == 0) smask[wi][g] = bm;
  }
  __syncwarp();
#pragma unroll 1
  for (int g = 0; g < CPL; ++g) {
    unsigned b = smask[wi][g];
    while (b) {
      int l[NF];
#pragma unroll
      for (int q = 0; q < NF; ++q) {
        l[q] = b ? __ffs(b) - 1 : -1;
        b &= b - 1;
      }
      float gg[NF], v[NF][CPL];
#pragma unroll
      for (int q = 0; q < NF; ++q) {
        gg[q] = l[q] >= 0 ? sgam[wi][32 * g + l[q]] : 0.0f;
        if (l[q] >= 0) IO::ld(Wt + (size_t)(32 * g + l[q]) * w + m0, v[q]);
      }
#pragma unroll
      for (int q = 0; q < NF; ++q)
        if (l[q] >= 0) emit(gg[q], v[q]);
    }
  }
#pragma unroll
  for (int c = 0; c < CPL; ++c) pnew[(size_t)cell * w + m0 + c] = acc[c];
}

// ---- c' = W_j a + b_j for every cell of a chunk in float32 on the CUDA cores (sound mode with
//      inflation): output (cell, n) is one fused multiply-add chain over k = 0 .. K-1 starting from
//      b_n, so it errs by at most gamma_{K+1} (sum_k |W_nk a_k| + |b_n|).  64 x 64 output tiles (cells x
//      neurons), K step 16, 4 x 4 outputs per thread. ----
__global__ void __launch_bounds__(256) k_center_fp32(int nc, int w, const float* __restrict__ A,
                                                     const float* __restrict__ Wt, const float* __restrict__ bias,
                                                     float* __restrict__ C) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64];
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float bj = (n0 + tx * 4 + j < w) ? bias[n0 + tx * 4 + j] : 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i][j] = bj;
  }
  for (int k0 = 0; k0 < w; k0 += 16) {
    {
      const int row = tid >> 2, kq = (tid & 3) * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (m0 + row < nc) v = *reinterpret_cast<const float4*>(A + (size_t)(m0 + row) * w + k0 + kq);
      As[kq + 0][row] = v.x; As[kq + 1][row] = v.y; As[kq + 2][row] = v.z; As[kq + 3][row] = v.w;
      const int kk = tid >> 4, nq = (tid & 15) * 4;
      float4 bv = make_float4(0.f, 0.f, 0.f, 0.f);
      if (n0 + nq < w) bv = *reinterpret_cast<const float4*>(Wt + (size_t)(k0 + kk) * w + n0 + nq);
      Bs[kk][nq + 0] = bv.x; Bs[kk][nq + 1] = bv.y; Bs[kk][nq + 2] = bv.z; Bs[kk][nq + 3] = bv.w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = m0 + ty * 4 + i;
    const int c = n0 + tx * 4;
    if (r < nc && c < w) *reinterpret_cast<float4*>(C + (size_t)r * w + c) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
  }
}

// ---- centre and input rows of z_{j+1}: c' = W a + b, I'_d = (I_d diag(alpha)) W^T, at float32-class
//      accuracy on the tensor cores: every operand x is carried as x_hi + x_lo (two bf16 terms) and
//      the product as a_hi w_hi + a_lo w_hi + a_hi w_lo (the dropped a_lo w_lo is below 2^-16 of
//      it), accumulated in float32 in TMEM.  Row r of the A operand is quantity r & 3 (0: a,
//      1-3: alpha I_d) of cell r >> 2; the activation pass writes it, split, to global memory.
//      Warp-specialised and TMA-fed: warp 0 loads A_hi, A_lo, W_hi, W_lo chunk by chunk (64-wide K)
//      into a two-stage ring, warp 1 issues the MMAs into one of two TMEM accumulators, warps 2-5
//      drain the other accumulator to float32 rows (TMEM lane group = warp mod 4). ----
enum { SB_FULL, SB_EMPTY = SB_FULL + 2, SB_TFULL = SB_EMPTY + 2, SB_TEMPTY = SB_TFULL + 2, SB_COUNT = SB_TEMPTY + 2 };
constexpr int kST = 192;                        // threads of the split GEMM: producer, MMA, 4 epilogue warps

struct RowsSplitArgs {
  int64_t nc;
  const float* bias;                            // [W]
  float* Cout;                                  // [nc][W]
  float* Iout;                                  // [nc][3][W]
  float* Dout;                                  // one-product mode: [nc][W], row r of A -> row r
  int* status;
};
struct RowsSplitMaps {
  CUtensorMap ahi, alo;                         // A terms [4 nc][W] bf16, box {64, 128}
  CUtensorMap whi, wlo;                         // W_j terms [W][W] bf16, box {64, W}
};

template <int W>
struct SplitSmem {
  static constexpr int KC = W / 64;
  static constexpr int NHALF = W > 256 ? 2 : 1;            // W = 512: each CTA computes 256 output columns
  static constexpr int NC = W / NHALF;                     // output columns of a CTA
  static constexpr size_t kA = (size_t)kRT * 128;          // one A term of one K chunk
  static constexpr size_t kB = (size_t)NC * 128;           // one W term of one K chunk (NC rows of W)
  static constexpr size_t kStage = 2 * kA + 2 * kB;
  static constexpr size_t bytes() { return 1024 + 2 * kStage + SB_COUNT * 8 + 16; }
};

// ONE = true: the one-product mode, D = A_hi W_hi^T for nc rows of A (no low terms, no bias): the
// GEMM of the rounding-error bound, whose operands are non-negative and rounded up.
template <int W, bool ONE>
__global__ void __launch_bounds__(kST, 1) k_rows_split(const __grid_constant__ RowsSplitArgs args,
                                                        const __grid_constant__ RowsSplitMaps maps) {
  using S = SplitSmem<W>;
  constexpr int KC = S::KC, NHALF = S::NHALF, NC = S::NC;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + 2 * S::kStage);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + SB_COUNT);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int64_t nrows = ONE ? args.nc : 4 * args.nc;
  const int64_t ntiles = (nrows + kRT - 1) / kRT;
  // work items (tile, column half); the grid is a multiple of NHALF, so a CTA keeps its half
  const int hq = blockIdx.x % NHALF;
  const int64_t t0 = blockIdx.x / NHALF, TS = gridDim.x / NHALF;
  if (t == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bar[SB_FULL + i], 1);
      mbar_init(&bar[SB_EMPTY + i], 1);
      mbar_init(&bar[SB_TFULL + i], 1);
      mbar_init(&bar[SB_TEMPTY + i], 4);
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "n"(2 * NC)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  auto stage = [&](int s) { return base + (size_t)s * S::kStage; };

  if (warp == 0) {
    // ---- producer ----
    if (lane == 0) {
      uint32_t it = 0;
      for (int64_t tile = t0; tile < ntiles; tile += TS) {
        for (int c = 0; c < KC; ++c, ++it) {
          const int sidx = it & 1;
          if (!rwait(&bar[SB_EMPTY + sidx], ((it >> 1) & 1) ^ 1, abort, args.status)) break;
          uint8_t* sp = stage(sidx);
          mbar_expect_tx(&bar[SB_FULL + sidx], (uint32_t)(ONE ? S::kA + S::kB : S::kStage));
          tma_load_2d(sp, &maps.ahi, &bar[SB_FULL + sidx], c * 64, (int)(tile * kRT));
          if (!ONE) tma_load_2d(sp + S::kA, &maps.alo, &bar[SB_FULL + sidx], c * 64, (int)(tile * kRT));
          tma_load_2d(sp + 2 * S::kA, &maps.whi, &bar[SB_FULL + sidx], c * 64, hq * NC);
          if (!ONE) tma_load_2d(sp + 2 * S::kA + S::kB, &maps.wlo, &bar[SB_FULL + sidx], c * 64, hq * NC);
        }
        if (*abort) break;
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      const uint32_t id = idesc(NC);
      uint32_t it = 0, tt = 0;
      for (int64_t tile = t0; tile < ntiles && !*abort; tile += TS, ++tt) {
        const uint32_t b = tt & 1;
        if (!rwait(&bar[SB_TEMPTY + b], ((tt >> 1) & 1) ^ 1, abort, args.status)) break;
        tc_fence_after();
        const uint32_t dt = tmem + b * NC;
        for (int c = 0; c < KC; ++c, ++it) {
          const int sidx = it & 1;
          if (!rwait(&bar[SB_FULL + sidx], (it >> 1) & 1, abort, args.status)) break;
          tc_fence_after();
          const uint32_t ah = su32(stage(sidx)), al = ah + (uint32_t)S::kA;
          const uint32_t bh = ah + 2 * (uint32_t)S::kA, bl = bh + (uint32_t)S::kB;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            mma_bf16(dt, sdesc(ah + kk * 32), sdesc(bh + kk * 32), id, (c > 0 || kk > 0) ? 1u : 0u);
            if (!ONE) {
              mma_bf16(dt, sdesc(al + kk * 32), sdesc(bh + kk * 32), id, 1u);
              mma_bf16(dt, sdesc(ah + kk * 32), sdesc(bl + kk * 32), id, 1u);
            }
          }
          mma_commit(&bar[SB_EMPTY + sidx]);
        }
        mma_commit(&bar[SB_TFULL + b]);
      }
    }
  } else {
    // ---- epilogue: TMEM lane group warp % 4, one row per thread ----
    const int row = 32 * (warp & 3) + lane;
    uint32_t tt = 0;
    for (int64_t tile = t0; tile < ntiles; tile += TS, ++tt) {
      const uint32_t b = tt & 1;
      const bool got = rwait(&bar[SB_TFULL + b], (tt >> 1) & 1, abort, args.status);
      if (!__all_sync(0xffffffffu, got)) break;
      tc_fence_after();
      const int64_t r = tile * kRT + row;
      const int64_t cell = ONE ? r : r >> 2;
      const int q = ONE ? 1 : (int)(r & 3);
      const bool valid = cell < args.nc;
      float* dst = nullptr;
      if (valid)
        dst = (ONE ? args.Dout + r * W : (q == 0) ? args.Cout + cell * W : args.Iout + (cell * 3 + q - 1) * W) + hq * NC;
      const uint32_t trow = tmem + b * NC + ((uint32_t)(32 * (warp & 3)) << 16);
#pragma unroll 1
      for (int c0 = 0; c0 < NC; c0 += 32) {
        float v[32];
        tmem_ld32(trow + c0, v);
        if (valid) {
          if (!ONE && q == 0)
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] += args.bias[hq * NC + c0 + i];
          float4* d4 = reinterpret_cast<float4*>(dst + c0);
#pragma unroll
          for (int i = 0; i < 8; ++i) d4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar[SB_TEMPTY + b]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (*abort)
    for (int i = 0; i < 1000; ++i) __nanosleep(1000);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(2 * NC) : "memory");
  }
}

// ---- reductions of z_{j+1} per (cell, neuron): r = sum |x| or sigma = sqrt(sum x^2) over the cell's
//      symbols, from the column sums the row GEMM wrote per (cell, 64-row input block), the new
//      rows' sums of k_rows_new and the three input rows (compensated), fused with activation j+1
//      (alpha, gamma, a,
//      and, when AH is given, the split A operand of the next centre / input-row GEMM (which carries
//      a; otherwise a itself is written, for the output layer) and the next row count
//      cnt_next = cnt_out + #(gamma != 0)).  One warp per cell; PASSES passes over the neurons,
//      CPL consecutive neurons per lane and pass (w = 32 CPL PASSES); every load of a pass is issued
//      before its first use. ----
template <int CPL>
__device__ __forceinline__ void ldv(const float* p, float* v) {
#pragma unroll
  for (int i = 0; i < CPL; i += 2) {
    const float2 x = *reinterpret_cast<const float2*>(p + i);
    v[i] = x.x;
    v[i + 1] = x.y;
  }
}
template <int CPL>
__device__ __forceinline__ void stv(float* p, const float* v) {
#pragma unroll
  for (int i = 0; i < CPL; i += 2) *reinterpret_cast<float2*>(p + i) = make_float2(v[i], v[i + 1]);
}
constexpr int kRedWarps = 4;
template <int CPL, int PASSES>
__global__ void __launch_bounds__(32 * kRedWarps) k_rows_reduce_act(int nc, int mode, int act, const float* part,
                                                                    const float* pnew, const int64_t* off_in,
                                                                    const int* cnt_in, const int* cnt_out,
                                                                    const float* I, const float* C, float* A, float* AL,
                                                                    float* GA, int* cnt_next, __nv_bfloat16* AH,
                                                                    __nv_bfloat16* ALO, Infl infl) {
  constexpr int w = 32 * CPL * PASSES;
  const int lane = threadIdx.x & 31;
  const int cell = blockIdx.x * kRedWarps + (threadIdx.x >> 5);
  if (cell >= nc) return;
  const bool sq = mode == ISX_BOUND_CLT;
  const int rows = cnt_in[cell];
  const int64_t o0 = off_in[cell];
  const int rows_out = cnt_out[cell];
  int m = 0;
#pragma unroll 1
  for (int pass = 0; pass < PASSES; ++pass) {
  const int n0 = (pass * 32 + lane) * CPL;
  float iv[3][CPL], cv[CPL], pv[CPL];
#pragma unroll
  for (int d = 0; d < 3; ++d) ldv<CPL>(I + ((size_t)cell * 3 + d) * w + n0, iv[d]);
  ldv<CPL>(C + (size_t)cell * w + n0, cv);
  ldv<CPL>(pnew + (size_t)cell * w + n0, pv);
  float dv[CPL];
  if (infl.on) ldv<CPL>(infl.D + (size_t)cell * w + n0, dv);
  // s: the symbol rows' sum (column sums of the row GEMM and of the new rows), compensated; sI: the
  // three input rows'
  float s[CPL], e[CPL], sI[CPL];
  auto add = [&](int i, float v) {
    const float y = v - e[i], tt = s[i] + y;
    e[i] = (tt - s[i]) - y;
    s[i] = tt;
  };
#pragma unroll
  for (int i = 0; i < CPL; ++i) {
    s[i] = e[i] = 0.0f;
    sI[i] = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) sI[i] += sq ? iv[d][i] * iv[d][i] : fabsf(iv[d][i]);
    add(i, pv[i]);
  }
  if (rows > 0) {
    const int64_t t0 = o0 / rows::kPT, t1 = (o0 + rows - 1) / rows::kPT;
    for (int64_t t = t0; t <= t1; ++t) {
      float q[CPL];
      ldv<CPL>(part + (size_t)rows::rows_part_slot(cell, t) * w + n0, q);
#pragma unroll
      for (int i = 0; i < CPL; ++i) add(i, q[i]);
    }
  }
  float av[CPL], alv[CPL], gv[CPL];
  const size_t o = (size_t)cell * w + n0;
#pragma unroll
  for (int i = 0; i < CPL; ++i) {
    Lin L;
    if (infl.on) {
      const float sg = s[i];
      const float ru = __fmul_ru(__fadd_ru(sg, sI[i]), infl.sum_g);
      float dl = __fmul_ru(dv[i], infl.gemm_slack);
      dl = __fadd_ru(dl, __fmul_ru(infl.store, __fmul_ru(sg, infl.sum_g)));
      dl = __fadd_ru(dl, __fmul_ru(infl.kappa_c, fabsf(infl.bias[n0 + i])));
      L = relu_sound(cv[i], ru, dl, true);           // the slack is folded into the new symbol
      if (AH) {
        float v = __fmul_ru(L.alpha, __fmul_ru(infl.kappa_g, __fmul_ru(sg, infl.sum_g)));
        v = __fadd_ru(v, __fmul_ru(L.alpha, __fmul_ru(infl.kappa_i, __fmul_ru(sI[i], infl.sum_g))));
        v = __fadd_ru(v, __fmul_ru(infl.kappa_c, fabsf(L.center)));
        infl.V[o + i] = bf16_up(v);
      } else {
        infl.RAD[o + i] = ru;
        infl.SLK[o + i] = 0.0f;
      }
    } else {
      const float tot = s[i] + sI[i];
      const float r = sq ? sqrtf(tot) : tot;
      L = sq ? act_clt(act, cv[i], r) : relu_sound(cv[i], r, 0.0f, false);
    }
    av[i] = L.center;
    alv[i] = L.alpha;
    gv[i] = L.gamma;
    m += L.gamma != 0.0f;
  }
  // the centre a is read back after the last layer, and by the float32 centre GEMM with inflation
  if (!AH || infl.on) stv<CPL>(A + o, av);
  stv<CPL>(AL + o, alv);
  stv<CPL>(GA + o, gv);
  if (AH) {
    auto put = [&](size_t idx, const float* v) {
#pragma unroll
      for (int i = 0; i < CPL; i += 2) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[i], v[i + 1]);
        const float2 hf = __bfloat1622float2(h);
        *reinterpret_cast<__nv_bfloat162*>(AH + idx + i) = h;
        *reinterpret_cast<__nv_bfloat162*>(ALO + idx + i) = __floats2bfloat162_rn(v[i] - hf.x, v[i + 1] - hf.y);
      }
    };
    const size_t q0 = (size_t)cell * 4 * w + n0;
    put(q0, av);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float x[CPL];
#pragma unroll
      for (int i = 0; i < CPL; ++i) x[i] = alv[i] * iv[d][i];
      put(q0 + (size_t)(d + 1) * w, x);
    }
  }
  }
  if (!cnt_next) return;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m += __shfl_xor_sync(0xffffffffu, m, off);
  if (lane == 0) cnt_next[cell] = rows_out + m;
}

// ---- output layer and read-off: x0 = w_out . a + b_out; every symbol's output coefficient is its
//      row . (alpha_H * w_out), or gamma_n w_out,n for the last activation's symbols ----
// With inflation (sound mode) the radius adds the float32 errors of the output layer and the slack:
//   (1 + gamma_S) sum |y_i|  +  gamma_{w+1} sum_n |alpha_n w_n| RAD_n  +  (1 + gamma_w) sum_n |w_n| SLK_n
//   + gamma_{w+1} (sum_n |w_n a_n| + |b|)  +  u sum_n |gamma_n w_n|,
// S the number of symbols: each y_i = row_i . (alpha o w) errs by gamma_{w+1} sum_n |x_in| |alpha_n w_n|
// (summed over i: RAD_n bounds sum_i |x_in|), the centre's dot product by gamma_{w+1} of its terms, the
// last activation's symbols gamma_n w_n by one rounding, and the slack alpha d passes through |w|.
// One warp per cell, CPL = w / 32 consecutive neurons per lane (the vector v = alpha o w_out stays in
// registers); each row is one vector load per lane, four rows' loads in flight, and its dot product
// is reduced across the warp before |y| or y^2 is taken.
constexpr int kOutWarps = 8;
template <int CPL>
__device__ __forceinline__ void ld_row(const __nv_bfloat16* p, float* f) {
  uint32_t h[CPL / 2];
  if constexpr (CPL == 2) {
    h[0] = *reinterpret_cast<const uint32_t*>(p);
  } else if constexpr (CPL == 4) {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    h[0] = u.x; h[1] = u.y;
  } else {
#pragma unroll
    for (int i = 0; i < CPL / 8; ++i) {
      const uint4 u = *reinterpret_cast<const uint4*>(p + 8 * i);
      h[4 * i] = u.x; h[4 * i + 1] = u.y; h[4 * i + 2] = u.z; h[4 * i + 3] = u.w;
    }
  }
#pragma unroll
  for (int i = 0; i < CPL / 2; ++i) {
    const float2 x = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&h[i]));
    f[2 * i] = x.x;
    f[2 * i + 1] = x.y;
  }
}
template <int CPL>
__global__ void __launch_bounds__(32 * kOutWarps) k_rows_output(int nc, int mode, const __nv_bfloat16* X,
                                                                const int64_t* off, const int* cnt, const float* I,
                                                                const float* A, const float* AL, const float* GA,
                                                                const float* __restrict__ wout, float bout,
                                                                int64_t first, float* center, float* spread,
                                                                Infl infl) {
  constexpr int w = 32 * CPL;
  const int lane = threadIdx.x & 31;
  const int cell = blockIdx.x * kOutWarps + (threadIdx.x >> 5);
  if (cell >= nc) return;
  const bool sq = mode != ISX_BOUND_SOUND;
  const int m0 = lane * CPL;
  const size_t o = (size_t)cell * w + m0;
  const int rows = cnt[cell];
  const int64_t o0 = off[cell];
  float v[CPL];
  // per lane: x0 and the last activation's symbols (s), the error terms (ex); sr, the rows' and the
  // input rows' terms, is the same in every lane (their dot products are reduced across the warp)
  float x0 = 0.0f, s = 0.0f, ex = 0.0f, sr = 0.0f;
  {
    float wo[CPL], al[CPL], av[CPL], gv[CPL];
    ldv<CPL>(wout + m0, wo);
    ldv<CPL>(AL + o, al);
    ldv<CPL>(A + o, av);
    ldv<CPL>(GA + o, gv);
    float rad[CPL], slk[CPL];
    if (infl.on) {
      ldv<CPL>(infl.RAD + o, rad);
      ldv<CPL>(infl.SLK + o, slk);
    }
    const float gw = infl.gamma_w;
#pragma unroll
    for (int i = 0; i < CPL; ++i) {
      v[i] = al[i] * wo[i];
      x0 = fmaf(wo[i], av[i], x0);
      const float y = gv[i] * wo[i];
      s += sq ? y * y : fabsf(y);
      if (infl.on) {
        ex = __fadd_ru(ex, __fmul_ru(gw, __fmul_ru(fabsf(v[i]), rad[i])));
        ex = __fadd_ru(ex, __fmul_ru(1.0f + gw, __fmul_ru(fabsf(wo[i]), slk[i])));
        ex = __fadd_ru(ex, __fmul_ru(gw, fabsf(wo[i] * av[i])));
        ex = __fadd_ru(ex, __fmul_ru(kU32, fabsf(y)));
      }
    }
  }
  auto dot = [&](const float* x) {
    float y = 0.0f;
#pragma unroll
    for (int i = 0; i < CPL; ++i) y = fmaf(x[i], v[i], y);
    return y;
  };
  // the three input rows (float32)
  {
    float y[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float iv[CPL];
      ldv<CPL>(I + ((size_t)cell * 3 + d) * w + m0, iv);
      y[d] = dot(iv);
    }
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1)
#pragma unroll
      for (int d = 0; d < 3; ++d) y[d] += __shfl_xor_sync(0xffffffffu, y[d], sh);
#pragma unroll
    for (int d = 0; d < 3; ++d) sr += sq ? y[d] * y[d] : fabsf(y[d]);
  }
  // the stored symbol rows (bf16), four at a time
  const __nv_bfloat16* xp = X + o0 * w + m0;
  int r = 0;
  for (; r + 4 <= rows; r += 4) {
    float y[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float x[CPL];
      ld_row<CPL>(xp + (size_t)(r + q) * w, x);
      y[q] = dot(x);
    }
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1)
#pragma unroll
      for (int q = 0; q < 4; ++q) y[q] += __shfl_xor_sync(0xffffffffu, y[q], sh);
#pragma unroll
    for (int q = 0; q < 4; ++q) sr += sq ? y[q] * y[q] : fabsf(y[q]);
  }
  for (; r < rows; ++r) {
    float x[CPL];
    ld_row<CPL>(xp + (size_t)r * w, x);
    float y = dot(x);
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) y += __shfl_xor_sync(0xffffffffu, y, sh);
    sr += sq ? y * y : fabsf(y);
  }
#pragma unroll
  for (int sh = 16; sh > 0; sh >>= 1) {
    x0 += __shfl_xor_sync(0xffffffffu, x0, sh);
    s += __shfl_xor_sync(0xffffffffu, s, sh);
    ex += __shfl_xor_sync(0xffffffffu, ex, sh);
  }
  if (lane == 0) {
    const float a = x0, b = s + sr;
    center[first + cell] = a + bout;
    if (infl.on) {
      // S symbols summed in float32: a factor 1 + gamma_S, S = rows + 3 + w; the partial sums of the
      // error terms are rounded up and their float32 additions covered by the 1 + 2^-20 factor
      const float su = (float)(rows + 3 + w) * kU32;
      const float gS = __fmul_ru(__fdiv_ru(su, 1.0f - su), 1.0010f);
      float e = ex;
      e = __fadd_ru(e, __fmul_ru(infl.gamma_w, fabsf(bout)));
      e = __fadd_ru(e, 2.0f * kU32 * (fabsf(a) + fabsf(bout)));      // the final add of the centre
      e = __fmul_ru(e, 1.0000050f);
      spread[first + cell] = __fadd_ru(__fmul_ru(b, 1.0f + 2.0f * gS), e);
    } else {
      spread[first + cell] = (mode == ISX_BOUND_SOUND) ? b : sqrtf(mode == ISX_BOUND_RAUA ? b / 3.0f : b);
    }
  }
}

template <int W, bool ONE>
isx_status launch_rows_split(isx_inr inr, const RowsSplitArgs& a, const RowsSplitMaps& maps, cudaStream_t st) {
  const size_t smem = SplitSmem<W>::bytes();
  ISX_CUDA(cudaFuncSetAttribute(k_rows_split<W, ONE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int sms = 148;
  ISX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, inr->device));
  int per_sm = 1;
  ISX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rows_split<W, ONE>, kST, smem));
  constexpr int NHALF = SplitSmem<W>::NHALF;
  per_sm = std::max(1, std::min(per_sm, 512 / (2 * SplitSmem<W>::NC)));
  const int64_t ntiles = ((ONE ? 1 : 4) * a.nc + kRT - 1) / kRT;
  int grid = (int)std::min<int64_t>(ntiles * NHALF, (int64_t)sms * per_sm);
  grid -= grid % NHALF;
  k_rows_split<W, ONE><<<grid, kST, smem, st>>>(a, maps);
  ISX_LAUNCH_CHECK("k_rows_split");
  return ISX_OK;
}
template <bool ONE>
isx_status launch_rows_split_w(isx_inr inr, int w, const RowsSplitArgs& a, const RowsSplitMaps& maps,
                               cudaStream_t st) {
  if (w == 512) return launch_rows_split<512, ONE>(inr, a, maps, st);
  if (w == 256) return launch_rows_split<256, ONE>(inr, a, maps, st);
  if (w == 128) return launch_rows_split<128, ONE>(inr, a, maps, st);
  return launch_rows_split<64, ONE>(inr, a, maps, st);
}

}  // namespace

bool rows_supported(isx_inr inr, isx_bound_mode mode, int inflate) {
  (void)inflate;
  if (!(inr->w == 64 || inr->w == 128 || inr->w == 256 || inr->w == 512) || inr->H < 1) return false;
  return mode == ISX_BOUND_SOUND || mode == ISX_BOUND_CLT || mode == ISX_BOUND_RAUA;
}

isx_status bound_bf16_rows(isx_inr inr, const CellSource& src, int64_t n, isx_bound_mode mode, int inflate,
                           float* d_center, float* d_spread, cudaStream_t st) {
  if (n <= 0) return ISX_OK;
  if (!rows_supported(inr, mode, inflate)) {
    set_error("row-batched tensor-core bounds need hidden width 64, 128, 256 or 512");
    return ISX_ERR_UNSUPPORTED;
  }
  if (mode != ISX_BOUND_SOUND) inflate = 0;
  const int w = inr->w, H = inr->H;
  auto& ws = inr->ws;
  ISX_TRY(ws[WS_TC_STATUS].ensure(64, "tc status"));
  ISX_TRY(ws[WS_R_TOT].ensure(64 + 8 * ((kMaxChunkCells + kScanB - 1) / kScanB), "row total and scan block sums"));
  int* status = ws[WS_TC_STATUS].as<int>();
  int64_t* d_tot = ws[WS_R_TOT].as<int64_t>();
  int64_t* bsum = d_tot + 8;
  ISX_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
  std::vector<CUtensorMap> maps(inr->n_layers), lomaps(inr->n_layers), pmaps(inr->n_layers);
  // TMA boxes are at most 256 rows: the split GEMM reads W_j in 256-row halves and the row GEMM in
  // 128-row quarters at w = 512
  const uint32_t box_split = w > 256 ? 256 : w, box_rows = w > 256 ? 128 : w;
  for (int l = 1; l <= H - 1; ++l) {
    ISX_TRY(tensor_map_bf16(&maps[l], inr->W_bf16[l], w, w, 64, box_split));
    ISX_TRY(tensor_map_bf16(&lomaps[l], inr->Wlo_bf16[l], w, w, 64, box_split));
    ISX_TRY(tensor_map_bf16(&pmaps[l], inr->Wperm_bf16[l] ? inr->Wperm_bf16[l] : inr->W_bf16[l], w, w, 64, box_rows));
  }
  const int sq = mode == ISX_BOUND_CLT ? 1 : 0;
  std::vector<CUtensorMap> absmaps(inr->n_layers);
  if (inflate)
    for (int l = 1; l <= H - 1; ++l) ISX_TRY(tensor_map_bf16(&absmaps[l], inr->Wabsru_bf16[l], w, w, 64, box_split));
  // chunk size: about kRowBudget G rows per chunk, from the rows per cell the previous chunk needed
  const int64_t kRowBudget = inr->row_budget;
  const int64_t kMaxCells = kMaxChunkCells;
  double rows_per_cell = (double)w * (H - 1);
  int64_t first = 0;
  while (first < n) {
    const int64_t want = (int64_t)((double)kRowBudget / std::max(1.0, 1.25 * rows_per_cell));
    const int nc = (int)std::min<int64_t>(n - first, std::max<int64_t>(1024, std::min(kMaxCells, want)));
    const size_t cw = (size_t)nc * w * sizeof(float);
    ISX_TRY(ws[WS_C].ensure(cw, "rows centre"));
    ISX_TRY(ws[WS_R_A].ensure(cw, "rows post-activation centre"));
    ISX_TRY(ws[WS_ALPHA].ensure(cw, "rows alpha"));
    ISX_TRY(ws[WS_GAMMA].ensure(cw, "rows gamma"));
    ISX_TRY(ws[WS_R_I0].ensure(3 * cw, "rows input rows"));
    ISX_TRY(ws[WS_R_I1].ensure(3 * cw, "rows input rows"));
    ISX_TRY(ws[WS_R_PNEW].ensure(cw, "new-row column sums"));
    Infl infl;
    if (inflate) {
      ISX_TRY(ws[WS_R_V].ensure(cw / 2, "rounding-bound operand"));
      ISX_TRY(ws[WS_R_D].ensure(cw, "rounding-bound GEMM result"));
      ISX_TRY(ws[WS_RAD].ensure(cw, "last radius bound"));
      ISX_TRY(ws[WS_DELTA].ensure(cw, "last slack"));
      infl.on = 1;
      set_infl(infl, w);
    }
    ISX_TRY(ws[WS_R_AH].ensure(4 * cw / 2, "split A, high terms"));
    ISX_TRY(ws[WS_R_ALO].ensure(4 * cw / 2, "split A, low terms"));
    for (Slot s : {WS_R_CNT0, WS_R_CNT1}) ISX_TRY(ws[s].ensure((size_t)nc * sizeof(int), "rows counts"));
    for (Slot s : {WS_R_OFF0, WS_R_OFF1}) ISX_TRY(ws[s].ensure((size_t)nc * sizeof(int64_t), "rows offsets"));
    float* C = ws[WS_C].as<float>();
    float* A = ws[WS_R_A].as<float>();
    float* AL = ws[WS_ALPHA].as<float>();
    float* GA = ws[WS_GAMMA].as<float>();
    float* I0 = ws[WS_R_I0].as<float>();
    float* I1 = ws[WS_R_I1].as<float>();
    __nv_bfloat16* AH = ws[WS_R_AH].as<__nv_bfloat16>();
    __nv_bfloat16* ALO = ws[WS_R_ALO].as<__nv_bfloat16>();
    Slot xs[2] = {WS_X0, WS_X1}, cs[2] = {WS_R_CNT0, WS_R_CNT1}, os[2] = {WS_R_OFF0, WS_R_OFF1},
         rs[2] = {WS_R_RC0, WS_R_RC1};
    int cur = 0;
    int64_t R = 0;
    const int act_blocks = (int)((nc + (512 / w) - 1) / (512 / w));   // 512 / w cells per block
    {
      prof::Scope ps(K_ROWS_ACT, st, 2.0 * nc * 3 * w, 0);
      Infl fi = infl;
      if (inflate) {
        fi.V = H > 1 ? ws[WS_R_V].as<__nv_bfloat16>() : nullptr;
        fi.RAD = ws[WS_RAD].as<float>();
        fi.SLK = ws[WS_DELTA].as<float>();
      }
      k_rows_input_act<<<act_blocks, 256, 0, st>>>(src, first, nc, w, (int)mode, inr->act, inr->W[0], inr->b[0], I0,
                                                   A, AL, GA, ws[cs[1]].as<int>(), H > 1 ? AH : nullptr, ALO, fi);
      ISX_LAUNCH_CHECK("k_rows_input_act");
    }
    ISX_CUDA(cudaMemsetAsync(ws[cs[0]].ptr, 0, (size_t)nc * sizeof(int), st));
    ISX_CUDA(cudaMemsetAsync(ws[os[0]].ptr, 0, (size_t)nc * sizeof(int64_t), st));
    for (int j = 1; j <= H - 1; ++j) {
      const int nxt = cur ^ 1;
      int* cnt_in = ws[cs[cur]].as<int>();
      int* cnt_out = ws[cs[nxt]].as<int>();
      int64_t* off_in = ws[os[cur]].as<int64_t>();
      int64_t* off_out = ws[os[nxt]].as<int64_t>();
      {
        prof::Scope ps(K_ROWS_ACT, st, 0, 0);
        const int64_t nb = ((int64_t)nc + kScanB - 1) / kScanB;
        k_rows_scan_sums<<<(unsigned)nb, kScanB, 0, st>>>(cnt_out, nc, bsum);
        k_rows_scan_top<<<1, kScanB, 0, st>>>(bsum, nb, d_tot);
        k_rows_scan_apply<<<(unsigned)nb, kScanB, 0, st>>>(cnt_out, nc, bsum, off_out);
        ISX_LAUNCH_CHECK("k_rows_scan");
      }
      int64_t Rn = 0;
      ISX_CUDA(cudaMemcpyAsync(&Rn, d_tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
      ISX_CUDA(cudaStreamSynchronize(st));
      ISX_TRY(ws[xs[nxt]].ensure((size_t)std::max<int64_t>(Rn, 1) * w * 2, "rows"));
      ISX_TRY(ws[rs[nxt]].ensure((size_t)std::max<int64_t>(Rn, 1) * sizeof(int), "row cells"));
      const int64_t ntiles = (R + rows::kPT - 1) / rows::kPT;     // column-sum blocks of the input rows
      ISX_TRY(ws[WS_R_PART].ensure((size_t)(nc + ntiles) * w * sizeof(float), "row GEMM column sums"));
      __nv_bfloat16* Xin = ws[xs[cur]].as<__nv_bfloat16>();
      __nv_bfloat16* Xout = ws[xs[nxt]].as<__nv_bfloat16>();
      float* part = ws[WS_R_PART].as<float>();
      float* pnew = ws[WS_R_PNEW].as<float>();
      if (R > 0) {
        rows::RowsGemmArgs ga{};
        ga.xin = Xin;
        ga.rowcell = ws[rs[cur]].as<int>();
        ga.off_in = off_in;
        ga.off_out = off_out;
        ga.alpha = AL;
        ga.R = R;
        ga.xout = Xout;
        ga.part = part;
        ga.sq = sq;
        ga.status = status;
        // bytes: rows in and out, the column sums of every (cell, 64-row block) segment
        prof::Scope ps(K_ROWS_GEMM, st, 2.0 * (double)R * w * w, 4.0 * (double)R * w);
        ISX_TRY(rows::launch_rows_gemm(inr, ga, pmaps[j], w, st));
      }
      {
        // bytes: the new rows (bf16) and the row -> cell map written, gamma read, the column sums
        prof::Scope ps(K_ROWS_NEW, st, 0, 2.0 * (double)(Rn - R) * w + 4.0 * (double)Rn + 8.0 * (double)nc * w);
        const unsigned nb = (unsigned)((nc + kNewWarps - 1) / kNewWarps);
        int* rc = ws[rs[nxt]].as<int>();
        if (w == 512)
          k_rows_new<16><<<nb, 32 * kNewWarps, 0, st>>>(nc, sq, GA, inr->Wt[j], cnt_in, off_out, cnt_out, Xout, rc, pnew);
        else if (w == 256)
          k_rows_new<8><<<nb, 32 * kNewWarps, 0, st>>>(nc, sq, GA, inr->Wt[j], cnt_in, off_out, cnt_out, Xout, rc, pnew);
        else if (w == 128)
          k_rows_new<4><<<nb, 32 * kNewWarps, 0, st>>>(nc, sq, GA, inr->Wt[j], cnt_in, off_out, cnt_out, Xout, rc, pnew);
        else
          k_rows_new<2><<<nb, 32 * kNewWarps, 0, st>>>(nc, sq, GA, inr->Wt[j], cnt_in, off_out, cnt_out, Xout, rc, pnew);
        ISX_LAUNCH_CHECK("k_rows_new");
      }
      {
        RowsSplitArgs sa{};
        sa.nc = nc;
        sa.bias = inr->b[j];
        sa.Cout = C;
        sa.Iout = I1;
        sa.status = status;
        RowsSplitMaps sm;
        std::memset(&sm, 0, sizeof(sm));
        ISX_TRY(tensor_map_bf16(&sm.ahi, AH, w, 4 * (uint64_t)nc, 64, kRT));
        ISX_TRY(tensor_map_bf16(&sm.alo, ALO, w, 4 * (uint64_t)nc, 64, kRT));
        sm.whi = maps[j];
        sm.wlo = lomaps[j];
        prof::Scope ps(K_ROWS_SPLIT, st, 2.0 * nc * 4.0 * w * w, 0);
        ISX_TRY(launch_rows_split_w<false>(inr, w, sa, sm, st));
      }
      if (inflate) {
        // the centre in float32 on the CUDA cores, over the tensor cores' two-term one
        prof::Scope pc(K_GEMM_FP32, st, 2.0 * nc * w * w, 0);
        k_center_fp32<<<dim3((unsigned)((w + 63) / 64), (unsigned)((nc + 63) / 64)), 256, 0, st>>>(nc, w, A, inr->Wt[j],
                                                                                                  inr->b[j], C);
        ISX_LAUNCH_CHECK("k_center_fp32");
      }
      if (inflate) {
        // the rounding-error bound's GEMM: D = |W_j| v, operands rounded up
        RowsSplitArgs da{};
        da.nc = nc;
        da.Dout = ws[WS_R_D].as<float>();
        da.status = status;
        RowsSplitMaps dm;
        std::memset(&dm, 0, sizeof(dm));
        ISX_TRY(tensor_map_bf16(&dm.ahi, ws[WS_R_V].ptr, w, (uint64_t)nc, 64, kRT));
        dm.whi = absmaps[j];
        prof::Scope ps(K_ROWS_AUX, st, 2.0 * nc * w * w, 0);
        ISX_TRY(launch_rows_split_w<true>(inr, w, da, dm, st));
      }
      {
        // reductions of z_{j+1} and activation j+1; its row count goes to the buffer of X_j's counts.
        // bytes per cell: the column sums (one vector per 64-row input block the cell spans, and
        // the new rows'), the three input rows and the centre read; a, alpha, gamma and the split
        // operand (4 rows, two bf16 terms) written
        const bool last = j == H - 1;
        const double vecs = (double)(nc + ntiles) + nc + 3.0 * nc + nc + 3.0 * nc + (last ? 0.0 : 4.0 * nc);
        prof::Scope ps(K_ROWS_REDUCE, st, 0, 4.0 * vecs * w);
        const unsigned rb = (unsigned)((nc + kRedWarps - 1) / kRedWarps);
        int* cn = last ? nullptr : cnt_in;
        __nv_bfloat16* ah = last ? nullptr : AH;
        Infl fi = infl;
        if (inflate) {
          fi.bias = inr->b[j];
          fi.D = ws[WS_R_D].as<float>();
          fi.V = last ? nullptr : ws[WS_R_V].as<__nv_bfloat16>();
          fi.RAD = ws[WS_RAD].as<float>();
          fi.SLK = ws[WS_DELTA].as<float>();
        }
        // two neurons per lane and pass: the fewest registers per warp, so the most cells in flight
        // (four neurons per lane took 1.3x as long, eight 1.33x, at w = 256)
        if (w == 512)
          k_rows_reduce_act<2, 8><<<rb, 32 * kRedWarps, 0, st>>>(nc, (int)mode, inr->act, part, pnew, off_in, cnt_in,
                                                                 cnt_out, I1, C, A, AL, GA, cn, ah, ALO, fi);
        else if (w == 256)
          k_rows_reduce_act<2, 4><<<rb, 32 * kRedWarps, 0, st>>>(nc, (int)mode, inr->act, part, pnew, off_in, cnt_in,
                                                                 cnt_out, I1, C, A, AL, GA, cn, ah, ALO, fi);
        else if (w == 128)
          k_rows_reduce_act<2, 2><<<rb, 32 * kRedWarps, 0, st>>>(nc, (int)mode, inr->act, part, pnew, off_in, cnt_in,
                                                                 cnt_out, I1, C, A, AL, GA, cn, ah, ALO, fi);
        else
          k_rows_reduce_act<2, 1><<<rb, 32 * kRedWarps, 0, st>>>(nc, (int)mode, inr->act, part, pnew, off_in, cnt_in,
                                                                 cnt_out, I1, C, A, AL, GA, cn, ah, ALO, fi);
        ISX_LAUNCH_CHECK("k_rows_reduce_act");
      }
      std::swap(I0, I1);
      cur = nxt;
      R = Rn;
    }
    {
      prof::Scope ps(K_ROWS_OUT, st, 2.0 * (double)(R + 3.0 * nc) * w, 2.0 * (double)R * w + 4.0 * 7.0 * nc * w);
      const int L = inr->n_layers - 1;
      Infl fi = infl;
      if (inflate) {
        fi.RAD = ws[WS_RAD].as<float>();
        fi.SLK = ws[WS_DELTA].as<float>();
      }
      const unsigned ob = (unsigned)((nc + kOutWarps - 1) / kOutWarps);
      const __nv_bfloat16* Xl = ws[xs[cur]].as<__nv_bfloat16>();
      const int64_t* ol = ws[os[cur]].as<int64_t>();
      const int* cl = ws[cs[cur]].as<int>();
      const float* wl = inr->W[L];
      const float bl = inr->hb[L][0];
      if (w == 512)
        k_rows_output<16><<<ob, 32 * kOutWarps, 0, st>>>(nc, (int)mode, Xl, ol, cl, I0, A, AL, GA, wl, bl, first,
                                                         d_center, d_spread, fi);
      else if (w == 256)
        k_rows_output<8><<<ob, 32 * kOutWarps, 0, st>>>(nc, (int)mode, Xl, ol, cl, I0, A, AL, GA, wl, bl, first,
                                                        d_center, d_spread, fi);
      else if (w == 128)
        k_rows_output<4><<<ob, 32 * kOutWarps, 0, st>>>(nc, (int)mode, Xl, ol, cl, I0, A, AL, GA, wl, bl, first,
                                                        d_center, d_spread, fi);
      else
        k_rows_output<2><<<ob, 32 * kOutWarps, 0, st>>>(nc, (int)mode, Xl, ol, cl, I0, A, AL, GA, wl, bl, first,
                                                        d_center, d_spread, fi);
      ISX_LAUNCH_CHECK("k_rows_output");
    }
    rows_per_cell = std::max(1.0, (double)R / nc);
    first += nc;
  }
  int stat = 0;
  ISX_CUDA(cudaMemcpyAsync(&stat, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  ISX_CUDA(cudaStreamSynchronize(st));
  if (stat != 0) {
    set_error("row-batched tensor-core kernel gave up waiting (bounded wait expired)");
    return (isx_status)stat;
  }
  return ISX_OK;
}

}  // namespace isx
