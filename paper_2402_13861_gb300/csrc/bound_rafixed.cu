// RA-Fixed bounds (the reduced range-analysis baseline of Sec. V-A.4 and App. A): sound affine
// arithmetic that keeps only the three input symbols and condenses every other coefficient of a
// neuron into one non-negative radius private to that neuron.
//
// Per cell and neuron the carried form is  c + a_1 eps_1 + a_2 eps_2 + a_3 eps_3 + r eta_n:
//   input box:  c = W_0 x_c + b_0,  a_d = h_d W_0[:, d],  r = 0
//   linear:     c' = W c + b,  a_d' = W a_d,  r' = |W| r               (Eq. 3 on the kept symbols)
//   ReLU:       Chebyshev line on [c - s, c + s], s = |a_1| + |a_2| + |a_3| + r   (Eq. 4)
//               c' = alpha c + beta,  a_d' = alpha a_d,  r' = alpha r + gamma
//   output:     [y_c - s_y, y_c + s_y],  s_y = sum_d |w . a_d| + |w| . r   (Eq. 2)
//
// One fused kernel runs the whole network for a tile of cells with the cells' forms resident in
// shared memory: [quantity][cell][neuron] for the quantities c, a_1..3, r.  A layer is a dense
// contraction of the rows c, a_d with W and of r with |W|, computed in float32 by register tiles: a
// thread owns 4 neurons (strided by w / 4,
// so that its W loads coalesce across the warp) of 4 cells and accumulates all quantities of those
// 16 (cell, neuron) pairs over k.  All quantities of one (cell, neuron) sit in one thread, so the
// ReLU is applied in registers and written back in place after a block barrier.
//
// Rounding-error inflation (inflate != 0): every float32 rounding is charged to r, which is a
// private symbol of its neuron, so the carried form stays a sound enclosure.  A K-term dot product
// errs by at most gamma_K sum |a_k b_k| (gamma_K = K u / (1 - K u), u = 2^-24).  Those sums are
// bounded by ||W_n||_1 M, M the largest magnitude m = |c| + sum_d |a_d| + r over the cell's neurons
// (kept per cell in shared memory, rounded up).
#include "internal.cuh"

#include <algorithm>
#include <cmath>

#include "cell_box.cuh"
#include "linearise.cuh"

namespace isx {
namespace {

constexpr int kRaThreads = 256;
constexpr int kRaCellsPerThread = 4;      // cells of one thread's register tile
constexpr int kRaCols = 4;                // neurons of one thread's register tile
constexpr float kRaU = 5.9604645e-08f;    // 2^-24

__host__ __device__ __forceinline__ float ra_gamma(int k) { return (k * kRaU) / (1.0f - k * kRaU); }

struct RaLayers {
  const float* Wt[ISX_MAX_LAYERS];        // hidden layers 1 .. H-1: W^T, [w_in][w_out]
  const float* b[ISX_MAX_LAYERS];
};

// Quantities per (cell, neuron): 0 = c, 1..3 = a_d, 4 = r.
constexpr int kRaQ = 5;

// Sound ReLU on the reduced form of one (cell, neuron); v = {c, a_1, a_2, a_3, r}.  Returns the
// magnitude |c| + sum_d |a_d| + r of the result, rounded up (inflation only).
template <bool INFL>
__device__ __forceinline__ float ra_relu(float* v) {
  if (INFL) {
    const float sa = __fadd_ru(__fadd_ru(fabsf(v[1]), fabsf(v[2])), fabsf(v[3]));
    const float s = __fadd_ru(sa, v[4]);
    Lin L = relu_sound(v[0], s, 0.0f, true);
    v[0] = L.center;
    v[1] *= L.alpha;
    v[2] *= L.alpha;
    v[3] *= L.alpha;
    // r' = alpha r + gamma, plus the rounding of the three products alpha a_d
    float r = __fadd_ru(__fmul_ru(L.alpha, v[4]), L.gamma);
    v[4] = __fadd_ru(r, __fmul_ru(2.0f * kRaU, __fmul_ru(L.alpha, sa)));
    return __fadd_ru(__fadd_ru(__fadd_ru(fabsf(v[0]), fabsf(v[1])), __fadd_ru(fabsf(v[2]), fabsf(v[3]))), v[4]);
  } else {
    const float s = fabsf(v[1]) + fabsf(v[2]) + fabsf(v[3]) + v[4];
    Lin L = relu_sound(v[0], s, 0.0f, false);
    v[0] = L.center;
    v[1] *= L.alpha;
    v[2] *= L.alpha;
    v[3] *= L.alpha;
    v[4] = fmaf(L.alpha, v[4], L.gamma);
    return 0.0f;
  }
}

template <bool INFL>
__global__ void __launch_bounds__(kRaThreads, 2)
k_bound_rafixed(CellSource src, int64_t first, int64_t n, int w, int H, const float* __restrict__ W0,
                const float* __restrict__ b0, RaLayers layers, const float* __restrict__ wout, float bout,
                float* __restrict__ center, float* __restrict__ spread) {
  constexpr int Q = kRaQ;
  constexpr int CPT = kRaCellsPerThread, TN = kRaCols;
  extern __shared__ float4 ra_smem4[];
  float* S = reinterpret_cast<float*>(ra_smem4);
  const int tpg = w / TN;                          // threads per group of CPT cells
  const int G = kRaThreads / tpg;                  // groups per CTA
  const int cells = G * CPT;                       // cells per CTA
  const int t = threadIdx.x;
  const int g = t / tpg, tc = t - g * tpg;
  const bool active = g < G;
  const int64_t cta_first = first + (int64_t)blockIdx.x * cells;
  auto at = [&](int q, int cell, int col) -> float& { return S[((size_t)q * cells + cell) * w + col]; };
  // per-cell largest magnitude, double-buffered across layers (non-negative floats order as ints)
  unsigned* Mx = reinterpret_cast<unsigned*>(S + (size_t)Q * cells * w);
  if (INFL)
    for (int i = t; i < 2 * cells; i += kRaThreads) Mx[i] = 0u;
  __syncthreads();

  // ---- input layer (3 -> w) and first ReLU, written into shared memory ----
  if (active) {
    for (int i = 0; i < CPT; ++i) {
      const int cell = g * CPT + i;
      int64_t gi = cta_first + cell;
      if (gi >= first + n) gi = first + n - 1;     // ragged tile: recompute the last cell, never stored
      float xc[3], h[3];
      cell_box(src, gi, INFL ? 1 : 0, xc, h);
      for (int j = 0; j < TN; ++j) {
        const int col = tc + j * tpg;
        const float w0 = W0[3 * col], w1 = W0[3 * col + 1], w2 = W0[3 * col + 2], bb = b0[col];
        float v[Q];
        v[0] = fmaf(w2, xc[2], fmaf(w1, xc[1], fmaf(w0, xc[0], bb)));
        v[1] = h[0] * w0;
        v[2] = h[1] * w1;
        v[3] = h[2] * w2;
        v[4] = 0.0f;
        if (INFL) {
          // three fused multiply-adds and three products, each rounded once
          const float e = fabsf(w0 * xc[0]) + fabsf(w1 * xc[1]) + fabsf(w2 * xc[2]) + fabsf(bb);
          const float sa = fabsf(v[1]) + fabsf(v[2]) + fabsf(v[3]);
          v[4] = (5.0f * kRaU * e + 3.0f * kRaU * sa) * 1.01f;
        }
        const float mag = ra_relu<INFL>(v);
        if (INFL) atomicMax(&Mx[cell], __float_as_uint(mag));
        for (int q = 0; q < Q; ++q) at(q, cell, col) = v[q];
      }
    }
  }
  __syncthreads();

  // ---- hidden layers 1 .. H-1: contraction with W (rows c, a_d) and |W| (row r), then ReLU ----
  for (int l = 1; l < H; ++l) {
    const float* __restrict__ Wt = layers.Wt[l];
    const float* __restrict__ bias = layers.b[l];
    float acc[Q][CPT][TN];
    float wabs[TN];                                // ||W_n||_1 of the thread's neurons (inflation)
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int i = 0; i < CPT; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[q][i][j] = 0.0f;
#pragma unroll
    for (int j = 0; j < TN; ++j) wabs[j] = 0.0f;
    const unsigned* Mprev = Mx + ((l - 1) & 1) * cells;
    unsigned* Mnext = Mx + (l & 1) * cells;
    if (INFL)
      for (int i = t; i < cells; i += kRaThreads) Mnext[i] = 0u;   // its last reader was layer l - 1
    if (active) {
      const float* rows = S + (size_t)(g * CPT) * w;
      for (int k = 0; k < w; k += 4) {
        float wv[4][TN];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
#pragma unroll
          for (int j = 0; j < TN; ++j) wv[kk][j] = __ldg(Wt + (size_t)(k + kk) * w + tc + j * tpg);
        if (INFL) {
#pragma unroll
          for (int j = 0; j < TN; ++j)
            wabs[j] += (fabsf(wv[0][j]) + fabsf(wv[1][j])) + (fabsf(wv[2][j]) + fabsf(wv[3][j]));
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
#pragma unroll
          for (int i = 0; i < CPT; ++i) {
            const float4 x = *reinterpret_cast<const float4*>(rows + ((size_t)q * cells + i) * w + k);
#pragma unroll
            for (int j = 0; j < TN; ++j) {
              const float m0 = q >= 4 ? fabsf(wv[0][j]) : wv[0][j];
              const float m1 = q >= 4 ? fabsf(wv[1][j]) : wv[1][j];
              const float m2 = q >= 4 ? fabsf(wv[2][j]) : wv[2][j];
              const float m3 = q >= 4 ? fabsf(wv[3][j]) : wv[3][j];
              float a = acc[q][i][j];
              a = fmaf(x.x, m0, a);
              a = fmaf(x.y, m1, a);
              a = fmaf(x.z, m2, a);
              a = fmaf(x.w, m3, a);
              acc[q][i][j] = a;
            }
          }
        }
      }
    }
    __syncthreads();                               // every thread is done reading layer l-1
    if (active) {
      const float gk = ra_gamma(w + 8);
#pragma unroll
      for (int i = 0; i < CPT; ++i) {
        const int cell = g * CPT + i;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          const int col = tc + j * tpg;
          const float bb = bias[col];
          float v[Q];
          v[0] = acc[0][i][j] + bb;
          v[1] = acc[1][i][j];
          v[2] = acc[2][i][j];
          v[3] = acc[3][i][j];
          v[4] = acc[4][i][j];
          if (INFL) {
            // E = ||W_n||_1 M + |b_n| >= sum_k |W_nk| (|c_k| + sum_d |a_dk| + r_k) + |b_n| bounds
            // every row's dot-product error by gamma_K E; four rows (c, a_1..3) are charged, and r'
            // (a sum of non-negative terms) is scaled up by its own relative error
            const float one = 1.0f + 2.0f * gk;
            const float E = __fmul_ru(__fadd_ru(__fmul_ru(wabs[j], __uint_as_float(Mprev[cell])), fabsf(bb)), one);
            v[4] = __fadd_ru(__fmul_ru(v[4], one), __fmul_ru(4.0f * gk, E));
            v[4] = __fadd_ru(v[4], __fmul_ru(kRaU, fabsf(v[0])));      // the bias addition
          }
          const float mag = ra_relu<INFL>(v);
          if (INFL) atomicMax(&Mnext[cell], __float_as_uint(mag));
#pragma unroll
          for (int q = 0; q < Q; ++q) at(q, cell, col) = v[q];
        }
      }
    }
    __syncthreads();
  }

  // ---- output layer (w -> 1) and the read-off: one warp per cell ----
  const int lane = t & 31, warp = t >> 5;
  const unsigned* Mlast = Mx + ((H - 1) & 1) * cells;
  for (int cell = warp; cell < cells; cell += kRaThreads / 32) {
    float y[Q + 1];                                // y[Q] = ||w_out||_1 (inflation)
#pragma unroll
    for (int q = 0; q <= Q; ++q) y[q] = 0.0f;
    for (int col = lane; col < w; col += 32) {
      const float wo = wout[col];
#pragma unroll
      for (int q = 0; q < Q; ++q) y[q] = fmaf(q >= 4 ? fabsf(wo) : wo, at(q, cell, col), y[q]);
      y[Q] += fabsf(wo);
    }
#pragma unroll
    for (int q = 0; q <= Q; ++q)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) y[q] += __shfl_xor_sync(0xffffffffu, y[q], o);
    const int64_t gi = cta_first + cell;
    if (lane == 0 && gi < first + n) {
      const float c = y[0] + bout;
      float s;
      if (INFL) {
        const float gk = ra_gamma(w + 8);
        const float one = 1.0f + 2.0f * gk;
        const float sa = __fadd_ru(__fadd_ru(fabsf(y[1]), fabsf(y[2])), fabsf(y[3]));
        const float E = __fmul_ru(__fadd_ru(__fmul_ru(y[Q], __uint_as_float(Mlast[cell])), fabsf(bout)), one);
        s = __fadd_ru(__fadd_ru(sa, __fmul_ru(y[4], one)), __fmul_ru(4.0f * gk, E));
        s = __fadd_ru(s, __fmul_ru(kRaU, fabsf(c)));
      } else {
        s = fabsf(y[1]) + fabsf(y[2]) + fabsf(y[3]) + y[4];
      }
      center[gi] = c;
      spread[gi] = s;
    }
  }
}

}  // namespace

bool rafixed_supported(isx_inr inr) { return inr->w % (4 * kRaCols) == 0 && inr->w / kRaCols <= kRaThreads; }

size_t rafixed_cells_per_cta(int w) { return (size_t)(kRaThreads / (w / kRaCols)) * kRaCellsPerThread; }

isx_status bound_rafixed(isx_inr inr, const CellSource& src, int64_t n, int inflate, float* d_center,
                         float* d_spread, cudaStream_t st) {
  if (n <= 0) return ISX_OK;
  const int w = inr->w, H = inr->H;
  if (!rafixed_supported(inr)) {
    set_error("RA-Fixed bounds need a hidden width that is a multiple of 16 and at most 1024");
    return ISX_ERR_UNSUPPORTED;
  }
  RaLayers lay{};
  for (int l = 1; l < H; ++l) {
    lay.Wt[l] = inr->Wt[l];
    lay.b[l] = inr->b[l];
  }
  const int L = inr->n_layers - 1;
  const int cells = (int)rafixed_cells_per_cta(w);
  const size_t smem = (size_t)kRaQ * cells * w * sizeof(float) + 2 * cells * sizeof(unsigned);
  // the grid's x dimension is bounded; long lists run in slices
  const int64_t max_ctas = 1 << 30;
  const double flops = 2.0 * 5.0 * w * (double)w * (H - 1) + 2.0 * 3.0 * 4.0 * w + 2.0 * 5.0 * w;
  for (int64_t off = 0; off < n; off += max_ctas * cells) {
    const int64_t m = std::min<int64_t>(n - off, max_ctas * cells);
    const unsigned grid = (unsigned)((m + cells - 1) / cells);
    prof::Scope _ps(K_BOUND_RAFIXED, st, flops * (double)m, 8.0 * (double)m + 4.0 * w * w * (H - 1) * grid);
    if (inflate) {
      ISX_CUDA(cudaFuncSetAttribute(k_bound_rafixed<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_bound_rafixed<true><<<grid, kRaThreads, smem, st>>>(src, off, m, w, H, inr->W[0], inr->b[0], lay, inr->W[L],
                                                            inr->hb[L][0], d_center, d_spread);
    } else {
      ISX_CUDA(cudaFuncSetAttribute(k_bound_rafixed<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_bound_rafixed<false><<<grid, kRaThreads, smem, st>>>(src, off, m, w, H, inr->W[0], inr->b[0], lay,
                                                             inr->W[L], inr->hb[L][0], d_center, d_spread);
    }
    ISX_LAUNCH_CHECK("k_bound_rafixed");
  }
  return ISX_OK;
}

}  // namespace isx
