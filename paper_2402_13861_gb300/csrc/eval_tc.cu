// MLP evaluation at points on the tensor cores (the corner queries of Sec. IV-D and the dense
// baseline of Sec. V-A), with FP32-class accuracy from BF16 operands.
//
// Every operand is split into two BF16 terms, x = x_hi + x_lo with x_hi = bf16(x) and
// x_lo = bf16(x - x_hi) (|x_lo| <= 2^-9 |x|, x_hi + x_lo within 2^-17 |x| of x), and a product is
// taken as a_hi b_hi + a_hi b_lo + a_lo b_hi; the dropped a_lo b_lo term is below 2^-18 |a b|.
// Three tcgen05.mma (kind::f16, BF16 x BF16 -> FP32 in TMEM) per K step, so the tensor cores do 3x
// the algorithmic work, against 1/28 of their BF16 rate for FP32 FMAs on the CUDA cores.
//
// Layout: one CTA (one warpgroup, 128 threads) per 128-point tile, persistent over tiles.  Thread
// t owns point t of the tile = TMEM lane t.  Layer 0 (3 -> w) runs in FP32 on the CUDA cores; its
// activation output is split into A_hi, A_lo in shared memory (K-major, 128-byte swizzle).  Each
// hidden layer W_l (w x w) streams through two 32 KB stages (X: W_hi chunk, Y: W_lo chunk; one
// 64-wide K chunk each) loaded by TMA; thread 0 issues the MMAs into one w-column FP32 accumulator.
// The epilogue reads TMEM, adds the bias, applies the activation (ReLU, ELU or sine) and writes the
// next A_hi, A_lo; after the last hidden layer it contracts with w_out in FP32 instead.  Every wait is bounded (2 s): on timeout
// the kernel records ISX_ERR_TIMEOUT, lets copies land, frees TMEM and returns.
#include "internal.cuh"
#include "tc_ptx.cuh"
#include "linearise.cuh"

#include <algorithm>
#include <cstring>

namespace isx {
namespace {

using namespace tc;

constexpr int kT = 128;                        // points per tile = threads per CTA
constexpr uint64_t kEvWaitNs = 2000000000ull;
enum { EB_XFULL, EB_XEMPTY, EB_YFULL, EB_YEMPTY, EB_DONE, EB_COUNT };

struct EvArgs {
  const float* xyz;
  const uint32_t* ids;
  int R;
  int64_t n;
  float* out;
  int H;                                       // activation layers; hidden GEMMs are layers 1 .. H-1
  const float* W0;                             // [w][3]
  const float* b[ISX_MAX_LAYERS];              // biases of layers 0 .. H-1
  const float* wout;                           // [w]
  float bout;
  int act;                             // isx_activation of the hidden layers
  int* status;
};
struct EvMaps {
  CUtensorMap hi[ISX_MAX_LAYERS];              // W_l high parts, box {64, w}
  CUtensorMap lo[ISX_MAX_LAYERS];              // W_l low parts, box {64, w}
};

template <int W>
struct EvSmem {
  static constexpr int KC = W / 64;
  static constexpr size_t kA = (size_t)kT * W * 2;        // one activation term
  static constexpr size_t kS = (size_t)W * 128;           // one weight stage (64-wide K chunk)
  static constexpr size_t bytes(int H) {
    return 1024 + 2 * kA + 2 * kS + (size_t)(3 * W + (size_t)H * W + W) * 4 + EB_COUNT * 8 + 16;
  }
};

__device__ __forceinline__ uint32_t aoff(int row, int k) {  // byte offset of (row, k..k+7), k % 8 == 0
  return (uint32_t)((k >> 6) * kT * 128 + row * 128 + ((((k & 63) >> 3) ^ (row & 7)) << 4));
}

__device__ __forceinline__ bool ewait(uint64_t* b, uint32_t parity, volatile int* abort, int* status) {
  if (mbar_try(b, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try(b, parity)) return true;
    if ((it & 3) == 0) {
      if (*abort) return false;
      if (global_ns() - t0 > kEvWaitNs) {
        *abort = 1;
        atomicExch(status, (int)ISX_ERR_TIMEOUT);
        return false;
      }
    }
  }
}

// v (after the activation) split into two BF16 terms, 8 consecutive columns, stored at A_hi / A_lo.
__device__ __forceinline__ void store_split8(uint8_t* Ahi, uint8_t* Alo, int row, int k, const float* v) {
  uint32_t ph[4], pl[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float a = v[2 * i], b = v[2 * i + 1];
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    ph[i] = *reinterpret_cast<const uint32_t*>(&h);
    pl[i] = *reinterpret_cast<const uint32_t*>(&l);
  }
  const uint32_t o = aoff(row, k);
  *reinterpret_cast<uint4*>(Ahi + o) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
  *reinterpret_cast<uint4*>(Alo + o) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
}

template <int W>
__global__ void __launch_bounds__(kT, 1) k_eval_tc(const __grid_constant__ EvArgs args,
                                                    const __grid_constant__ EvMaps maps) {
  using S = EvSmem<W>;
  constexpr int KC = S::KC;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* Ahi = base;
  uint8_t* Alo = Ahi + S::kA;
  uint8_t* X = Alo + S::kA;
  uint8_t* Y = X + S::kS;
  float* sW0 = reinterpret_cast<float*>(Y + S::kS);
  float* sb = sW0 + 3 * W;                     // [H][W]: biases of layers 0 .. H-1
  float* swo = sb + (size_t)args.H * W;
  uint64_t* bar = reinterpret_cast<uint64_t*>(swo + W);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + EB_COUNT);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
  const int t = threadIdx.x, warp = t >> 5;
  const int H = args.H;

  if (t == 0) {
    for (int i = 0; i < EB_COUNT; ++i) mbar_init(&bar[i], 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "n"(W)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  for (int i = t; i < 3 * W; i += kT) sW0[i] = args.W0[i];
  for (int l = 0; l < H; ++l)
    for (int i = t; i < W; i += kT) sb[l * W + i] = args.b[l][i];
  for (int i = t; i < W; i += kT) swo[i] = args.wout[i];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t id = idesc(W);
  const int64_t ntiles = (args.n + kT - 1) / kT;
  uint32_t xf = 0, xe = 0, yf = 0, ye = 0, dn = 0;     // phase counters (thread 0 / all)
  // thread 0: weight chunks
  auto load_x = [&](int l, int c) {
    mbar_expect_tx(&bar[EB_XFULL], (uint32_t)S::kS);
    tma_load_2d(X, &maps.hi[l], &bar[EB_XFULL], c * 64, 0);
  };
  auto load_y = [&](int l, int c) {
    mbar_expect_tx(&bar[EB_YFULL], (uint32_t)S::kS);
    tma_load_2d(Y, &maps.lo[l], &bar[EB_YFULL], c * 64, 0);
  };
  bool ok = true;
  if (t == 0 && blockIdx.x < ntiles) {
    load_x(1, 0);
    load_y(1, 0);
  }
  for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int64_t p = tile * kT + t;
    // ---- layer 0 in FP32, split into A_hi / A_lo ----
    float x[3] = {0.f, 0.f, 0.f};
    if (p < args.n) {
      if (args.ids) {
        const uint32_t idv = args.ids[p], n1 = (uint32_t)args.R + 1u;
        const uint32_t ix = idv % n1, iy = (idv / n1) % n1, iz = idv / (n1 * n1);
        const float inv = 2.0f / (float)args.R;
        x[0] = -1.0f + inv * (float)ix;
        x[1] = -1.0f + inv * (float)iy;
        x[2] = -1.0f + inv * (float)iz;
      } else {
        x[0] = args.xyz[3 * p];
        x[1] = args.xyz[3 * p + 1];
        x[2] = args.xyz[3 * p + 2];
      }
    }
    for (int k = 0; k < W; k += 8) {
      float v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int nn = k + i;
        const float z = fmaf(sW0[3 * nn + 2], x[2], fmaf(sW0[3 * nn + 1], x[1], fmaf(sW0[3 * nn], x[0], sb[nn])));
        v[i] = act_fwd(args.act, z);
      }
      store_split8(Ahi, Alo, t, k, v);
    }
    fence_async_shared();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    for (int l = 1; l <= H - 1; ++l) {
      // ---- thread 0: D = A_hi W_hi^T + A_lo W_hi^T + A_hi W_lo^T, K chunk by chunk ----
      if (t == 0) {
        for (int c = 0; c < KC && ok; ++c) {
          if (!ewait(&bar[EB_XFULL], xf & 1, abort, args.status)) { ok = false; break; }
          ++xf;
          tc_fence_after();
          const uint32_t ah = su32(Ahi + (size_t)c * kT * 128), al = su32(Alo + (size_t)c * kT * 128);
          const uint32_t bx = su32(X), by = su32(Y);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            mma_bf16(tmem, sdesc(ah + kk * 32), sdesc(bx + kk * 32), id, (c > 0 || kk > 0) ? 1u : 0u);
            mma_bf16(tmem, sdesc(al + kk * 32), sdesc(bx + kk * 32), id, 1u);
          }
          mma_commit(&bar[EB_XEMPTY]);
          if (!ewait(&bar[EB_YFULL], yf & 1, abort, args.status)) { ok = false; break; }
          ++yf;
          tc_fence_after();
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) mma_bf16(tmem, sdesc(ah + kk * 32), sdesc(by + kk * 32), id, 1u);
          mma_commit(&bar[EB_YEMPTY]);
          // refill the stages: the next chunk of this layer, else chunk 0 of the next layer (or of
          // layer 1 for the next tile)
          int nl = l, nc = c + 1;
          if (nc == KC) {
            nc = 0;
            nl = l + 1;
            if (nl > H - 1) nl = (tile + gridDim.x < ntiles) ? 1 : 0;
          }
          if (!ewait(&bar[EB_XEMPTY], xe & 1, abort, args.status)) { ok = false; break; }
          ++xe;
          if (nl) load_x(nl, nc);
          if (!ewait(&bar[EB_YEMPTY], ye & 1, abort, args.status)) { ok = false; break; }
          ++ye;
          if (nl) load_y(nl, nc);
        }
        if (ok) mma_commit(&bar[EB_DONE]);
      }
      // ---- everyone: epilogue of layer l ----
      if (!ewait(&bar[EB_DONE], dn & 1, abort, args.status)) ok = false;
      ++dn;
      __syncthreads();
      if (*abort) ok = false;
      if (!ok) break;
      tc_fence_after();
      const float* bl = sb + (size_t)l * W;
      const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
      if (l < H - 1) {
        for (int c0 = 0; c0 < W; c0 += 32) {
          float v[32];
          tmem_ld32(trow + c0, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = act_fwd(args.act, v[i] + bl[c0 + i]);
#pragma unroll
          for (int u = 0; u < 4; ++u) store_split8(Ahi, Alo, t, c0 + 8 * u, v + 8 * u);
        }
        fence_async_shared();
      } else {
        float y = 0.f;
        for (int c0 = 0; c0 < W; c0 += 32) {
          float v[32];
          tmem_ld32(trow + c0, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) y = fmaf(swo[c0 + i], act_fwd(args.act, v[i] + bl[c0 + i]), y);
        }
        if (p < args.n) args.out[p] = y + args.bout;
      }
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
    }
  }
  // ---- teardown: let in-flight copies land, free TMEM ----
  __syncthreads();
  if (*abort)
    for (int i = 0; i < 1000; ++i) __nanosleep(1000);
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(W) : "memory");
  }
}

template <int W>
isx_status launch_eval(isx_inr inr, const EvArgs& a, const EvMaps& maps, int64_t ntiles, cudaStream_t st) {
  const size_t smem = EvSmem<W>::bytes(inr->H);
  ISX_CUDA(cudaFuncSetAttribute(k_eval_tc<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 1, sms = 148;
  ISX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, inr->device));
  ISX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eval_tc<W>, kT, smem));
  // TMEM: W columns per CTA out of 512
  per_sm = std::max(1, std::min(per_sm, 512 / W));
  const int grid = (int)std::min<int64_t>(ntiles, (int64_t)sms * per_sm);
  k_eval_tc<W><<<grid, kT, smem, st>>>(a, maps);
  ISX_LAUNCH_CHECK("k_eval_tc");
  return ISX_OK;
}

}  // namespace

bool eval_tc_supported(isx_inr inr) { return (inr->w == 128 || inr->w == 256) && inr->H >= 2 && inr->H <= 12; }

isx_status eval_points_tc(isx_inr inr, const float* xyz, const uint32_t* lattice_ids, int R, int64_t n, float* out,
                          cudaStream_t st) {
  if (!eval_tc_supported(inr)) {
    set_error("tensor-core evaluation supports hidden widths 128 and 256 with 2..12 activation layers");
    return ISX_ERR_UNSUPPORTED;
  }
  if (n <= 0) return ISX_OK;
  const int w = inr->w, H = inr->H;
  EvArgs a{};
  a.xyz = xyz;
  a.ids = lattice_ids;
  a.R = R;
  a.n = n;
  a.out = out;
  a.H = H;
  a.W0 = inr->W[0];
  for (int l = 0; l < H; ++l) a.b[l] = inr->b[l];
  a.wout = inr->W[H];
  a.bout = inr->hb[H][0];
  a.act = inr->act;
  auto& ws = inr->ws;
  ISX_TRY(ws[WS_TC_STATUS].ensure(64, "tc status"));
  a.status = ws[WS_TC_STATUS].as<int>();
  EvMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int l = 1; l <= H - 1; ++l) {
    ISX_TRY(tensor_map_bf16(&maps.hi[l], inr->W_bf16[l], w, w, 64, w));
    ISX_TRY(tensor_map_bf16(&maps.lo[l], inr->Wlo_bf16[l], w, w, 64, w));
  }
  ISX_CUDA(cudaMemsetAsync(a.status, 0, sizeof(int), st));
  const int64_t ntiles = (n + kT - 1) / kT;
  {
    // algorithmic work: 2 (4 w + (H-1) w^2) FLOP per point
    prof::Scope ps(K_EVAL_TC, st, 2.0 * n * (4.0 * w + (H - 1.0) * w * w), 0);
    if (w == 256) {
      ISX_TRY(launch_eval<256>(inr, a, maps, ntiles, st));
    } else {
      ISX_TRY(launch_eval<128>(inr, a, maps, ntiles, st));
    }
  }
  int status = 0;
  ISX_CUDA(cudaMemcpyAsync(&status, a.status, sizeof(int), cudaMemcpyDeviceToHost, st));
  ISX_CUDA(cudaStreamSynchronize(st));
  if (status != 0) {
    set_error("tensor-core evaluation kernel gave up waiting (bounded wait expired)");
    return (isx_status)status;
  }
  return ISX_OK;
}

}  // namespace isx
