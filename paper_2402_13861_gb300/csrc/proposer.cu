// Cell-subdivision proposer.  The paper keeps or culls cells by range analysis alone (Algorithm 1);
// this addition scores (cell, iso-value) pairs with a small MLP trained on labels the method itself
// produces (dense evaluation plus the marching-cubes crossing test of Sec. IV-D), so that confident
// pairs skip the affine bound, and range analysis stays the fallback and decides the rest.
//
// Model: 8 -> 64 -> 64 -> 64 -> 1, ReLU hidden layers, sigmoid output, binary cross-entropy.
// Numerics: BF16 weights, BF16 inputs and activations (round to nearest even after every layer),
// FP32 accumulation; FP32 master weights, gradients and Adam moments.  The model costs 17.5 kFLOP
// per pair against 203 MFLOP for one affine bound of the 256-wide 5-layer INR, so it runs on CUDA
// cores: one thread per sample, weights broadcast from shared memory (staged once per block as
// FP32, exact), every thread's activation rows in padded shared memory (row stride 65 floats, so
// the 32 rows a warp touches fall in 32 different banks).
//
// Kernels: k_prop_forward (logits of given feature rows), k_prop_grad (forward + backward of the
// mean BCE, per-block gradient sums in shared memory, one atomic add per parameter per block),
// k_prop_adam (one Adam step over the flat parameter vector, refreshes the BF16 copy),
// k_prop_gate (extraction: builds the features of every (cell, iso) pair in the cell's mask, drops
// confident negatives, keeps confident positives, flags the rest for bounding), k_prop_merge
// (applies the bound of the flagged cells).
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

struct isx_proposer_s {
  int device = 0;
  float* params = nullptr;          // FP32 master weights, packed (isx.h)
  __nv_bfloat16* pb = nullptr;      // BF16 copy used by every forward and backward
  float* m = nullptr;               // Adam first moment
  float* v = nullptr;               // Adam second moment
  float* grad = nullptr;            // gradient accumulator of one step
  float* loss = nullptr;            // device scratch for the loss of one step
  float mu[8], inv_sd[8];
  int64_t t = 0;                    // Adam step count
};

namespace isx {
namespace {

constexpr int kF = 8, kH = 64;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + kH * kF, OFF_W2 = OFF_B1 + kH, OFF_B2 = OFF_W2 + kH * kH,
              OFF_W3 = OFF_B2 + kH, OFF_B3 = OFF_W3 + kH * kH, OFF_W4 = OFF_B3 + kH, OFF_B4 = OFF_W4 + kH,
              kNParam = OFF_B4 + 1;
static_assert(kNParam == ISX_PROPOSER_NPARAM, "packed parameter layout");
static_assert(OFF_W2 % 4 == 0 && OFF_W3 % 4 == 0 && OFF_W4 % 4 == 0, "float4 weight rows");
constexpr int kNParamPad = (kNParam + 3) & ~3;
constexpr int kTB = 128;          // samples per tile = threads per block
constexpr int kRow = kH + 1;      // padded activation row
constexpr int kRow0 = kF + 1;     // padded input row

struct Norm {
  float mu[kF], inv_sd[kF];
};

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void stage_weights(float* sw, const __nv_bfloat16* pb) {
  for (int k = threadIdx.x; k < kNParamPad; k += blockDim.x) sw[k] = k < kNParam ? __bfloat162float(pb[k]) : 0.f;
}

// out_row[o] = bf16(relu(b[o] + sum_i W[o][i] in[i])), o < 64; W row-major [64][IN] in shared memory.
template <int IN>
__device__ __forceinline__ void dense_relu(const float* W, const float* b, const float (&in)[IN], float* out_row) {
#pragma unroll 1
  for (int o = 0; o < kH; ++o) {
    const float4* w4 = reinterpret_cast<const float4*>(W + o * IN);
    float acc = b[o];
#pragma unroll
    for (int i = 0; i < IN / 4; ++i) {
      const float4 w = w4[i];
      acc = fmaf(w.x, in[4 * i], acc);
      acc = fmaf(w.y, in[4 * i + 1], acc);
      acc = fmaf(w.z, in[4 * i + 2], acc);
      acc = fmaf(w.w, in[4 * i + 3], acc);
    }
    out_row[o] = bf16r(fmaxf(acc, 0.f));
  }
}

template <int N>
__device__ __forceinline__ void load_row(const float* row, float (&v)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = row[i];
}

__device__ __forceinline__ void normalise(const Norm& nm, float (&x)[kF]) {
#pragma unroll
  for (int d = 0; d < kF; ++d) x[d] = bf16r((x[d] - nm.mu[d]) * nm.inv_sd[d]);
}

// Logit of one normalised sample; r1, r2, r3 receive the three hidden activation rows (r3 may
// alias r1 when the caller does not keep them).
__device__ __forceinline__ float forward_sample(const float* sw, const float (&x)[kF], float* r1, float* r2,
                                                float* r3) {
  dense_relu<kF>(sw + OFF_W1, sw + OFF_B1, x, r1);
  float h[kH];
  load_row(r1, h);
  dense_relu<kH>(sw + OFF_W2, sw + OFF_B2, h, r2);
  load_row(r2, h);
  dense_relu<kH>(sw + OFF_W3, sw + OFF_B3, h, r3);
  load_row(r3, h);
  float z = sw[OFF_B4];
#pragma unroll
  for (int i = 0; i < kH; ++i) z = fmaf(sw[OFF_W4 + i], h[i], z);
  return z;
}

__global__ void __launch_bounds__(kTB) k_prop_forward(const __nv_bfloat16* pb, Norm nm, const float* feat, int64_t n,
                                                      float* logit) {
  extern __shared__ float sm[];
  float* sw = sm;
  float* rows = sm + kNParamPad;                         // [2][kTB][kRow]
  stage_weights(sw, pb);
  __syncthreads();
  float* rx = rows + threadIdx.x * kRow;
  float* ry = rows + (kTB + threadIdx.x) * kRow;
  for (int64_t s = (int64_t)blockIdx.x * kTB + threadIdx.x; s < n; s += (int64_t)gridDim.x * kTB) {
    float x[kF];
#pragma unroll
    for (int d = 0; d < kF; ++d) x[d] = feat[s * kF + d];
    normalise(nm, x);
    logit[s] = forward_sample(sw, x, rx, ry, rx);
  }
}

// Block sums over the tile's samples of dZ[s][o] * A[s][i] (o < 64, i < IN) and of dZ[s][o],
// added into the block's gradient accumulator g (W at offW, b at offB).
template <int IN, int ROWA>
__device__ __forceinline__ void accumulate_layer(const float* dZ, const float* A, int ns, float* g, int offW,
                                                 int offB) {
  constexpr int PER = IN / 2;
  const int o = threadIdx.x >> 1, half = threadIdx.x & 1;
  float acc[PER];
#pragma unroll
  for (int c = 0; c < PER; ++c) acc[c] = 0.f;
  float accb = 0.f;
  for (int s = 0; s < ns; ++s) {
    const float d = dZ[s * kRow + o];
    const float* ar = A + s * ROWA + PER * half;
#pragma unroll
    for (int c = 0; c < PER; ++c) acc[c] = fmaf(d, ar[c], acc[c]);
    accb += d;
  }
#pragma unroll
  for (int c = 0; c < PER; ++c) g[offW + o * IN + PER * half + c] += acc[c];
  if (half == 0) g[offB + o] += accb;
}

// d_out[i] = mask(A_row[i] > 0) * sum_o W[o][i] dZrow[o]   (W row-major [64][64])
__device__ __forceinline__ void back_through(const float* W, const float* dZrow, const float* Arow, float* out) {
  float d[kH];
#pragma unroll
  for (int i = 0; i < kH; ++i) d[i] = 0.f;
#pragma unroll 1
  for (int o = 0; o < kH; ++o) {
    const float go = dZrow[o];
    const float4* w4 = reinterpret_cast<const float4*>(W + o * kH);
#pragma unroll
    for (int i = 0; i < kH / 4; ++i) {
      const float4 w = w4[i];
      d[4 * i] = fmaf(w.x, go, d[4 * i]);
      d[4 * i + 1] = fmaf(w.y, go, d[4 * i + 1]);
      d[4 * i + 2] = fmaf(w.z, go, d[4 * i + 2]);
      d[4 * i + 3] = fmaf(w.w, go, d[4 * i + 3]);
    }
  }
#pragma unroll
  for (int i = 0; i < kH; ++i) out[i] = Arow[i] > 0.f ? d[i] : 0.f;
}

constexpr size_t kGradSmemFloats = 2 * kNParamPad + kTB * kRow0 + 4 * kTB * kRow + kTB + 32;

// Forward and backward of the mean BCE over n samples: grad += dL/dtheta, loss += L.
__global__ void __launch_bounds__(kTB) k_prop_grad(const __nv_bfloat16* pb, Norm nm, const float* feat,
                                                   const float* label, int64_t n, float inv_n, float* grad,
                                                   float* loss) {
  extern __shared__ float sm[];
  float* sw = sm;
  float* g = sw + kNParamPad;
  float* A0 = g + kNParamPad;
  float* A1 = A0 + kTB * kRow0;
  float* A2 = A1 + kTB * kRow;
  float* A3 = A2 + kTB * kRow;
  float* dZ = A3 + kTB * kRow;
  float* dz4 = dZ + kTB * kRow;
  float* red = dz4 + kTB;
  stage_weights(sw, pb);
  for (int k = threadIdx.x; k < kNParamPad; k += blockDim.x) g[k] = 0.f;
  __syncthreads();
  const int t = threadIdx.x;
  float lsum = 0.f;
  for (int64_t base = (int64_t)blockIdx.x * kTB; base < n; base += (int64_t)gridDim.x * kTB) {
    const int64_t s = base + t;
    const bool valid = s < n;
    const int ns = (int)(n - base < (int64_t)kTB ? n - base : (int64_t)kTB);
    // ---- forward ----
    float x[kF];
#pragma unroll
    for (int d = 0; d < kF; ++d) x[d] = valid ? feat[s * kF + d] : 0.f;
    normalise(nm, x);
    if (!valid)
#pragma unroll
      for (int d = 0; d < kF; ++d) x[d] = 0.f;
#pragma unroll
    for (int d = 0; d < kF; ++d) A0[t * kRow0 + d] = x[d];
    const float z = forward_sample(sw, x, A1 + t * kRow, A2 + t * kRow, A3 + t * kRow);
    const float y = valid ? label[s] : 0.f;
    const float p = 1.f / (1.f + expf(-z));
    if (valid) lsum += fmaxf(z, 0.f) - z * y + log1pf(expf(-fabsf(z)));
    const float dz = valid ? (p - y) * inv_n : 0.f;
    dz4[t] = dz;
    // ---- dZ3 = (dz W4) masked by A3 > 0 ----
#pragma unroll 4
    for (int i = 0; i < kH; ++i) dZ[t * kRow + i] = A3[t * kRow + i] > 0.f ? dz * sw[OFF_W4 + i] : 0.f;
    __syncthreads();
    // ---- dW4, db4 (threads < 64: one input each), dW3, db3 ----
    if (t < kH) {
      float a = 0.f, ab = 0.f;
      for (int q = 0; q < ns; ++q) {
        a = fmaf(dz4[q], A3[q * kRow + t], a);
        ab += dz4[q];
      }
      g[OFF_W4 + t] += a;
      if (t == 0) g[OFF_B4] += ab;
    }
    accumulate_layer<kH, kRow>(dZ, A2, ns, g, OFF_W3, OFF_B3);
    __syncthreads();
    // ---- dZ2 = (W3^T dZ3) masked by A2 > 0 (computed into registers, then stored) ----
    {
      float d[kH];
      back_through(sw + OFF_W3, dZ + t * kRow, A2 + t * kRow, d);
      __syncthreads();
#pragma unroll
      for (int i = 0; i < kH; ++i) dZ[t * kRow + i] = d[i];
    }
    __syncthreads();
    accumulate_layer<kH, kRow>(dZ, A1, ns, g, OFF_W2, OFF_B2);
    __syncthreads();
    // ---- dZ1 = (W2^T dZ2) masked by A1 > 0 ----
    {
      float d[kH];
      back_through(sw + OFF_W2, dZ + t * kRow, A1 + t * kRow, d);
      __syncthreads();
#pragma unroll
      for (int i = 0; i < kH; ++i) dZ[t * kRow + i] = d[i];
    }
    __syncthreads();
    accumulate_layer<kF, kRow0>(dZ, A0, ns, g, OFF_W1, OFF_B1);
    __syncthreads();
  }
  for (int k = threadIdx.x; k < kNParam; k += blockDim.x) atomicAdd(&grad[k], g[k]);
  // ---- loss: block sum, one atomic ----
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if ((t & 31) == 0) red[t >> 5] = lsum;
  __syncthreads();
  if (t == 0) {
    float sacc = 0.f;
    for (int w = 0; w < kTB / 32; ++w) sacc += red[w];
    atomicAdd(loss, sacc * inv_n);
  }
}

__global__ void k_prop_adam(float* params, __nv_bfloat16* pb, float* m, float* v, float* grad, float lr, float b1,
                            float b2, float eps, float bc1, float bc2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kNParam) return;
  const float gk = grad[k];
  const float mk = b1 * m[k] + (1.f - b1) * gk;
  const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  const float p = params[k] - lr * (mk / bc1) / (sqrtf(vk / bc2) + eps);
  params[k] = p;
  pb[k] = __float2bfloat16_rn(p);
  grad[k] = 0.f;
}

__global__ void k_to_bf16(const float* src, __nv_bfloat16* dst, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) dst[k] = __float2bfloat16_rn(src[k]);
}

// Extraction gate: for every cell (packed code at `level`) and every iso q in its mask, the logit of
// the pair's features against the thresholds.  keep[i] = bits with logit >= z_hi (kept without a
// bound); need[i] = 1 if some bit lies strictly between the thresholds (the cell is bounded).
__global__ void __launch_bounds__(kTB) k_prop_gate(const __nv_bfloat16* pb, Norm nm, const uint32_t* codes,
                                                   const uint32_t* masks, const float* anc_c, const float* anc_s,
                                                   const uint8_t* anc_gap, int64_t n, int level, IsoSet iso,
                                                   float z_lo, float z_hi, uint32_t* keep, uint8_t* need) {
  extern __shared__ float sm[];
  float* sw = sm;
  float* rows = sm + kNParamPad;
  stage_weights(sw, pb);
  __syncthreads();
  float* rx = rows + threadIdx.x * kRow;
  float* ry = rows + (kTB + threadIdx.x) * kRow;
  const float h = ldexpf(1.0f, -level);
  for (int64_t i = (int64_t)blockIdx.x * kTB + threadIdx.x; i < n; i += (int64_t)gridDim.x * kTB) {
    const uint32_t code = codes[i];
    uint32_t m = masks[i];
    const float cx = -1.0f + (2.0f * float(code & 1023u) + 1.0f) * h;
    const float cy = -1.0f + (2.0f * float((code >> 10) & 1023u) + 1.0f) * h;
    const float cz = -1.0f + (2.0f * float((code >> 20) & 1023u) + 1.0f) * h;
    const float ac = anc_c[i], as = anc_s[i], gap = (float)anc_gap[i];
    uint32_t kbits = 0;
    bool unsure = false;
    while (m) {
      const int q = __ffs(m) - 1;
      m &= m - 1;
      const float c = iso.c[q];
      float x[kF] = {cx, cy, cz, -(float)level, c, ac - c, as, gap};
      normalise(nm, x);
      const float z = forward_sample(sw, x, rx, ry, rx);
      if (z >= z_hi) kbits |= 1u << q;
      else if (z > z_lo) unsure = true;
      // NaN logits (never expected) fall through to "unsure": the cell is bounded
      else if (!(z <= z_lo)) unsure = true;
    }
    keep[i] = kbits;
    need[i] = unsure ? 1 : 0;
  }
}

}  // namespace

namespace {
// Range-analysis decision of the flagged cells (idx[j], j < nb): their mask becomes
// mask & (cull test of Algorithm 1 on their bound), and that bound becomes the ancestor bound of
// their children (gap 0).
__global__ void k_prop_merge(const uint32_t* idx, int64_t nb, const uint32_t* masks, const float* c_sub,
                             const float* s_sub, IsoSet iso, int mode, float k, int inflate, uint32_t* keep,
                             float* anc_c, float* anc_s, uint8_t* anc_gap) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  const uint32_t i = idx[j];
  const float c = c_sub[j], s = s_sub[j];
  float lo, hi;
  if (sound_readout(mode)) {
    lo = inflate ? __fsub_rd(c, s) : c - s;
    hi = inflate ? __fadd_ru(c, s) : c + s;
  } else {
    lo = c - k * s;
    hi = c + k * s;
  }
  uint32_t bits = 0;
  for (int q = 0; q < iso.n; ++q)
    if (lo <= iso.c[q] && iso.c[q] <= hi) bits |= 1u << q;
  if (!(lo <= hi)) bits = 0xffffffffu;
  keep[i] = masks[i] & bits;
  anc_c[i] = c;
  anc_s[i] = s;
  anc_gap[i] = 0;
}

__global__ void k_gather_codes(const uint32_t* codes, const uint32_t* idx, int64_t nb, uint32_t* out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nb) out[j] = codes[idx[j]];
}

Norm norm_of(isx_proposer p) {
  Norm nm;
  for (int d = 0; d < kF; ++d) {
    nm.mu[d] = p->mu[d];
    nm.inv_sd[d] = p->inv_sd[d];
  }
  return nm;
}

int grid_for(int64_t n, int dev) {
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = (n + kTB - 1) / kTB;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, 4LL * sms));
}

size_t fwd_smem() { return (size_t)(kNParamPad + 2 * kTB * kRow) * sizeof(float); }

isx_status set_smem(const void* fn, size_t bytes) {
  ISX_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return ISX_OK;
}

isx_status check_prop(isx_proposer p) {
  if (!p || !p->params) {
    set_error("null proposer handle");
    return ISX_ERR_ARG;
  }
  return ISX_OK;
}

}  // namespace

isx_status proposer_gate(isx_proposer p, const uint32_t* codes, const uint32_t* masks, const float* anc_c,
                         const float* anc_s, const uint8_t* anc_gap, int64_t n, int level, const IsoSet& iso,
                         float z_lo, float z_hi, uint32_t* keep, uint8_t* need, cudaStream_t st) {
  if (n == 0) return ISX_OK;
  ISX_TRY(set_smem((const void*)k_prop_gate, fwd_smem()));
  {
    prof::Scope _ps(K_PROP_GATE, st, 2.0 * 8768 * (double)n, 0);
    k_prop_gate<<<grid_for(n, p->device), kTB, fwd_smem(), st>>>(p->pb, norm_of(p), codes, masks, anc_c, anc_s,
                                                                  anc_gap, n, level, iso, z_lo, z_hi, keep, need);
  }
  ISX_LAUNCH_CHECK("k_prop_gate");
  return ISX_OK;
}

isx_status proposer_merge(const uint32_t* idx, int64_t nb, const uint32_t* masks, const float* c_sub,
                          const float* s_sub, const IsoSet& iso, isx_bound_mode mode, float k, int inflate,
                          uint32_t* keep, float* anc_c, float* anc_s, uint8_t* anc_gap, cudaStream_t st) {
  if (nb == 0) return ISX_OK;
  {
    prof::Scope _ps(K_PROP_MERGE, st, 0, 0);
    k_prop_merge<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(idx, nb, masks, c_sub, s_sub, iso, (int)mode, k,
                                                               inflate, keep, anc_c, anc_s, anc_gap);
  }
  ISX_LAUNCH_CHECK("k_prop_merge");
  return ISX_OK;
}

isx_status gather_codes(const uint32_t* codes, const uint32_t* idx, int64_t nb, uint32_t* out, cudaStream_t st) {
  if (nb == 0) return ISX_OK;
  {
    prof::Scope _ps(K_PROP_MERGE, st, 0, 0);
    k_gather_codes<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(codes, idx, nb, out);
  }
  ISX_LAUNCH_CHECK("k_gather_codes");
  return ISX_OK;
}

}  // namespace isx

using namespace isx;

extern "C" {

isx_status isx_proposer_create(const float* params, const float* feat_mean, const float* feat_std,
                               isx_proposer* out) {
  if (!params || !feat_mean || !feat_std || !out) {
    set_error("null proposer argument");
    return ISX_ERR_ARG;
  }
  *out = nullptr;
  for (int d = 0; d < kF; ++d)
    if (!(feat_std[d] > 0.f) || !std::isfinite(feat_mean[d])) {
      set_error("feature standard deviations must be positive and means finite");
      return ISX_ERR_ARG;
    }
  isx_proposer p = new isx_proposer_s();
  ISX_CUDA(cudaGetDevice(&p->device));
  for (int d = 0; d < kF; ++d) {
    p->mu[d] = feat_mean[d];
    p->inv_sd[d] = 1.0f / feat_std[d];
  }
  auto fail = [&](cudaError_t e, const char* what) {
    isx_proposer_destroy(p);
    return cuda_fail(e, what, __FILE__, __LINE__);
  };
  cudaError_t e;
  const size_t fb = kNParam * sizeof(float);
  if ((e = cudaMalloc(&p->params, fb)) != cudaSuccess) return fail(e, "proposer params");
  if ((e = cudaMalloc(&p->pb, kNParam * 2)) != cudaSuccess) return fail(e, "proposer bf16");
  if ((e = cudaMalloc(&p->m, fb)) != cudaSuccess || (e = cudaMalloc(&p->v, fb)) != cudaSuccess ||
      (e = cudaMalloc(&p->grad, fb)) != cudaSuccess || (e = cudaMalloc(&p->loss, 16)) != cudaSuccess)
    return fail(e, "proposer optimiser state");
  if ((e = cudaMemcpy(p->params, params, fb, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(p->m, 0, fb)) != cudaSuccess || (e = cudaMemset(p->v, 0, fb)) != cudaSuccess ||
      (e = cudaMemset(p->grad, 0, fb)) != cudaSuccess)
    return fail(e, "proposer upload");
  k_to_bf16<<<(kNParam + 255) / 256, 256>>>(p->params, p->pb, kNParam);
  if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaDeviceSynchronize()) != cudaSuccess)
    return fail(e, "proposer bf16 copy");
  *out = p;
  return ISX_OK;
}

isx_status isx_proposer_destroy(isx_proposer p) {
  if (!p) return ISX_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(p->device);
  for (void* q : {(void*)p->params, (void*)p->pb, (void*)p->m, (void*)p->v, (void*)p->grad, (void*)p->loss})
    if (q) cudaFree(q);
  if (prev >= 0) cudaSetDevice(prev);
  delete p;
  return ISX_OK;
}

isx_status isx_proposer_get_params(isx_proposer p, float* out) {
  ISX_TRY(check_prop(p));
  if (!out) {
    set_error("null output");
    return ISX_ERR_ARG;
  }
  ISX_CUDA(cudaMemcpy(out, p->params, kNParam * sizeof(float), cudaMemcpyDeviceToHost));
  return ISX_OK;
}

isx_status isx_proposer_predict(isx_proposer p, const float* d_feat, int64_t n, float* d_logit, void* stream) {
  ISX_TRY(check_prop(p));
  if (n < 0 || (n > 0 && (!d_feat || !d_logit))) {
    set_error("bad size or null pointer");
    return ISX_ERR_ARG;
  }
  if (n == 0) return ISX_OK;
  cudaStream_t st = (cudaStream_t)stream;
  ISX_TRY(set_smem((const void*)k_prop_forward, fwd_smem()));
  {
    prof::Scope _ps(K_PROP_FWD, st, 2.0 * 8768 * (double)n, 0);
    k_prop_forward<<<grid_for(n, p->device), kTB, fwd_smem(), st>>>(p->pb, norm_of(p), d_feat, n, d_logit);
  }
  ISX_LAUNCH_CHECK("k_prop_forward");
  return ISX_OK;
}

isx_status isx_proposer_grad(isx_proposer p, const float* d_feat, const float* d_label, int64_t n, float* d_grad,
                             float* d_loss, void* stream) {
  ISX_TRY(check_prop(p));
  if (n <= 0 || !d_feat || !d_label || !d_grad || !d_loss) {
    set_error("bad size or null pointer");
    return ISX_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t smem = kGradSmemFloats * sizeof(float);
  ISX_TRY(set_smem((const void*)k_prop_grad, smem));
  ISX_CUDA(cudaMemsetAsync(d_grad, 0, kNParam * sizeof(float), st));
  ISX_CUDA(cudaMemsetAsync(d_loss, 0, sizeof(float), st));
  {
    prof::Scope _ps(K_PROP_GRAD, st, 3.0 * 2.0 * 8768 * (double)n, 0);
    k_prop_grad<<<grid_for(n, p->device), kTB, smem, st>>>(p->pb, norm_of(p), d_feat, d_label, n, 1.0f / (float)n,
                                                           d_grad, d_loss);
  }
  ISX_LAUNCH_CHECK("k_prop_grad");
  return ISX_OK;
}

isx_status isx_proposer_train_step(isx_proposer p, const float* d_feat, const float* d_label, int64_t n, float lr,
                                   float* d_loss, void* stream) {
  ISX_TRY(check_prop(p));
  if (n <= 0 || !d_feat || !d_label || !(lr > 0.f)) {
    set_error("bad size, learning rate or null pointer");
    return ISX_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  ISX_TRY(isx_proposer_grad(p, d_feat, d_label, n, p->grad, d_loss ? d_loss : p->loss, stream));
  p->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = 1.f - (float)std::pow((double)b1, (double)p->t);
  const float bc2 = 1.f - (float)std::pow((double)b2, (double)p->t);
  {
    prof::Scope _ps(K_PROP_ADAM, st, 0, 0);
    k_prop_adam<<<(kNParam + 255) / 256, 256, 0, st>>>(p->params, p->pb, p->m, p->v, p->grad, lr, b1, b2, 1e-8f,
                                                       bc1, bc2);
  }
  ISX_LAUNCH_CHECK("k_prop_adam");
  return ISX_OK;
}

}  // extern "C"
