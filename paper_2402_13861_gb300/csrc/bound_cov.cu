// CLT bound by covariance propagation on tcgen05 (bf16 operands, f32 accumulation).
//
// In uncertainty propagation the noise symbols are independent with unit variance (Eq. 6) and the
// read-off only needs sigma^2 = sum_i x_i^2 per neuron (Eq. 7).  With the coefficient matrix X of a
// pre-activation z_j, sigma^2 is the diagonal of the Gram matrix C_j = X^T X, and the propagation
// rules (Eq. 8 for the linear layer, Eq. 9 for the activation: X' = [X D; Gamma]) map it exactly to
//   C_1 = W_0 diag(h^2 / 3) W_0^T                      (input box, Sec. IV-C)
//   M_j = D_j C_j D_j + Gamma_j^2                      (ReLU j, Table VII: D = diag(alpha), Gamma = diag(gamma))
//   C_{j+1} = W_j M_j W_j^T                            (linear layer j)
//   sigma_out^2 = w_out^T M_H w_out.
// The centres follow the same rule as in the coefficient form (c' = W (alpha c + beta) + b).  The
// result equals the coefficient propagation up to rounding (the float64 oracle checks the same
// identity in clt_covariance).  Per layer and cell this is two w x w x w GEMMs regardless of depth,
// with no per-symbol reductions and no scratch in global memory.
//
// GB300 mapping (w = 128 or 256).  One CTA per SM walks over cells.  The per-cell w x w operand (M_j,
// then T^T) sits in shared memory as a K-major, 128-byte-swizzled bf16 B operand; the weights W_j
// (shared by all cells, resident in L2) stream through a 4-stage TMA ring as A tiles of 128 rows x
// 64 K; tcgen05.mma (M = 128, N = w, K = 16) accumulates the w x w product in TMEM (w/128 tiles of
// w columns).  Layer j: GEMM1 T^T = W_j M_j, GEMM2 C = W_j (T^T)^T.  8 compute warps move results
// from TMEM to shared memory: T^T after GEMM1; after GEMM2 they read diag(C) for sigma, linearise
// the ReLU with the centre from the 4 math warps (float32 GEMV c' = W a + b), and write
// M_{j+1} = alpha alpha^T * C + diag(gamma^2).  Warps: 0 TMA producer, 1 MMA issuer / TMEM owner,
// 2-9 compute, 10-13 math.  Every wait is bounded (2 s); on timeout the kernel records
// ISX_ERR_TIMEOUT, lets copies land, frees TMEM and returns.
#include "internal.cuh"
#include "linearise.cuh"
#include "tc_ptx.cuh"

#include <algorithm>
#include <cstring>

namespace isx {
namespace {
using namespace tc;

constexpr int kStagesC = 4;
constexpr int kCompWarps = 8;
constexpr int kMathWarpsC = 4;
constexpr int kThreadsC = 32 * (2 + kCompWarps + kMathWarpsC);   // 448
constexpr int kCompThreads = 32 * kCompWarps;                      // 256
constexpr int kCompBase = 64;
constexpr int kMathBaseC = 32 * (2 + kCompWarps);                  // 320
constexpr int kMathThreadsC = 32 * kMathWarpsC;                    // 128
constexpr uint32_t kStageBytesC = 128 * 128;                       // 128 rows x 64 bf16
constexpr uint64_t kWaitNsC = 2000000000ull;

struct CovArgs {
  CellSource src;
  int64_t n;
  int w, H;
  const float* W0;
  const float* b[ISX_MAX_LAYERS];
  const float* Wt[ISX_MAX_LAYERS];
  const float* wout;
  float bout;
  float* center;
  float* spread;
  int* status;
  int act;                             // isx_activation of the hidden layers
};

struct CovMaps {
  CUtensorMap wrow[ISX_MAX_LAYERS];   // W_l bf16 row-major [w][w], box {64, 128}
};

enum { CB_FULL = 0, CB_EMPTY = kStagesC, CB_BREADY = 2 * kStagesC, CB_DFULL, CB_RELU, CB_CENTER, CB_COUNT };

struct CovSmem {
  uint8_t* Bm;      // w/64 chunks of [w rows][128 B]
  uint8_t* A;       // kStagesC x 16 KB
  float* W0;        // [w][3]
  float* cn;        // centre of the next pre-activation (math warps)
  float* sig2;      // diag of C
  float* alpha;
  float* beta;
  float* gamma;
  float* a;         // a-form centre alpha c + beta
  float* aw;        // alpha * w_out (output layer)
  float* red;       // [64]
  uint64_t* bar;
  uint32_t* tmem_slot;
  int* abort;
};

size_t cov_smem_bytes(int w) {
  return (size_t)w * w * 2 + (size_t)kStagesC * kStageBytesC + (size_t)(3 * w + 7 * w + 64) * 4 + CB_COUNT * 8 + 16 +
         1024;
}

__device__ CovSmem cov_carve(uint8_t* raw, int w) {
  uintptr_t base = ((uintptr_t)raw + 1023) & ~(uintptr_t)1023;
  uint8_t* p = (uint8_t*)base;
  CovSmem s;
  s.Bm = p; p += (size_t)w * w * 2;
  s.A = p; p += (size_t)kStagesC * kStageBytesC;
  float* f = (float*)p;
  s.W0 = f; f += 3 * w;
  s.cn = f; f += w;
  s.sig2 = f; f += w;
  s.alpha = f; f += w;
  s.beta = f; f += w;
  s.gamma = f; f += w;
  s.a = f; f += w;
  s.aw = f; f += w;
  s.red = f; f += 64;
  s.bar = (uint64_t*)(((uintptr_t)f + 7) & ~(uintptr_t)7);
  s.tmem_slot = (uint32_t*)(s.bar + CB_COUNT);
  s.abort = (int*)(s.tmem_slot + 1);
  return s;
}

__device__ __forceinline__ void comp_sync() { asm volatile("bar.sync 2, %0;" ::"n"(kCompThreads) : "memory"); }
__device__ __forceinline__ void math_sync_c() { asm volatile("bar.sync 3, %0;" ::"n"(kMathThreadsC) : "memory"); }

__device__ __forceinline__ bool cwait(const CovSmem& s, uint64_t* b, uint32_t parity, int* status) {
  if (mbar_try(b, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try(b, parity)) return true;
    if ((it & 3) == 0) {
      if (*(volatile int*)s.abort) return false;
      if (global_ns() - t0 > kWaitNsC) {
        *(volatile int*)s.abort = 1;
        atomicExch(status, (int)ISX_ERR_TIMEOUT);
        return false;
      }
    }
  }
}

// Write 32 consecutive bf16 values (columns col0 .. col0 + 31 of row p) into the K-major,
// 128-byte-swizzled operand buffer (w/64 chunks of w rows x 128 B).
__device__ __forceinline__ void store_row32(uint8_t* Bm, int w, int p, int col0, const float v[32]) {
  const int c = col0 >> 6, u0 = (col0 & 63) >> 3;
  uint8_t* rowp = Bm + (size_t)c * w * 128 + (size_t)p * 128;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    __nv_bfloat162 h0 = __floats2bfloat162_rn(v[8 * u + 0], v[8 * u + 1]);
    __nv_bfloat162 h1 = __floats2bfloat162_rn(v[8 * u + 2], v[8 * u + 3]);
    __nv_bfloat162 h2 = __floats2bfloat162_rn(v[8 * u + 4], v[8 * u + 5]);
    __nv_bfloat162 h3 = __floats2bfloat162_rn(v[8 * u + 6], v[8 * u + 7]);
    uint4 pk = make_uint4(*reinterpret_cast<uint32_t*>(&h0), *reinterpret_cast<uint32_t*>(&h1),
                          *reinterpret_cast<uint32_t*>(&h2), *reinterpret_cast<uint32_t*>(&h3));
    const int phys = (u0 + u) ^ (p & 7);
    *reinterpret_cast<uint4*>(rowp + phys * 16) = pk;
  }
}

__global__ void __launch_bounds__(kThreadsC, 1) k_bound_cov(const __grid_constant__ CovArgs args,
                                                             const __grid_constant__ CovMaps maps) {
  extern __shared__ uint8_t smem_raw[];
  const int w = args.w, H = args.H;
  CovSmem s = cov_carve(smem_raw, w);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int MT = w / 128, KC = w / 64;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kStagesC; ++i) {
      mbar_init(&s.bar[CB_FULL + i], 1);
      mbar_init(&s.bar[CB_EMPTY + i], 1);
    }
    mbar_init(&s.bar[CB_BREADY], 1);
    mbar_init(&s.bar[CB_DFULL], 1);
    mbar_init(&s.bar[CB_RELU], 1);
    mbar_init(&s.bar[CB_CENTER], 1);
    *s.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = threadIdx.x; i < 3 * w; i += blockDim.x) s.W0[i] = args.W0[i];
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(su32(s.tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s.tmem_slot;

  if (warp == 0) {
    // ================================ TMA producer: W_j tiles, twice per layer =========================
    if (lane == 0) {
      uint32_t stage = 0, phase = 0;
      bool ok = true;
      for (int64_t cell = blockIdx.x; cell < args.n && ok; cell += gridDim.x)
        for (int j = 1; j <= H - 1 && ok; ++j)
          for (int g = 0; g < 2 && ok; ++g)
            for (int mt = 0; mt < MT && ok; ++mt)
              for (int c = 0; c < KC; ++c) {
                if (!cwait(s, &s.bar[CB_EMPTY + stage], phase ^ 1, args.status)) { ok = false; break; }
                mbar_expect_tx(&s.bar[CB_FULL + stage], kStageBytesC);
                tma_load_2d(s.A + (size_t)stage * kStageBytesC, &maps.wrow[j], &s.bar[CB_FULL + stage], c * 64,
                            mt * 128);
                if (++stage == kStagesC) { stage = 0; phase ^= 1; }
              }
    }
  } else if (warp == 1) {
    // ================================ MMA issuer ================================
    if (lane == 0) {
      uint32_t stage = 0, phase = 0, bready_n = 0;
      const uint32_t id = idesc(w);
      bool ok = true;
      for (int64_t cell = blockIdx.x; cell < args.n && ok; cell += gridDim.x)
        for (int j = 1; j <= H - 1 && ok; ++j)
          for (int g = 0; g < 2 && ok; ++g) {
            if (!cwait(s, &s.bar[CB_BREADY], bready_n & 1, args.status)) { ok = false; break; }
            ++bready_n;
            tc_fence_after();
            for (int mt = 0; mt < MT && ok; ++mt)
              for (int c = 0; c < KC; ++c) {
                if (!cwait(s, &s.bar[CB_FULL + stage], phase, args.status)) { ok = false; break; }
                tc_fence_after();
                const uint32_t a0 = su32(s.A + (size_t)stage * kStageBytesC);
                const uint32_t b0 = su32(s.Bm + (size_t)c * w * 128);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                  mma_bf16(tmem + mt * 256, sdesc(a0 + kk * 32), sdesc(b0 + kk * 32), id, (c > 0 || kk > 0) ? 1u : 0u);
                mma_commit(&s.bar[CB_EMPTY + stage]);
                if (++stage == kStagesC) { stage = 0; phase ^= 1; }
              }
            if (ok) mma_commit(&s.bar[CB_DFULL]);
          }
    }
  } else if (warp < 2 + kCompWarps) {
    // ================================ compute warps ================================
    const int ct = threadIdx.x - kCompBase;   // 0 .. 255
    const int q = warp & 3;                   // TMEM lane quarter
    const int hf = (warp - 2) >> 2;           // column half
    const int half = w / 2, nch = half / 32;
    uint32_t dfull_n = 0;
    // warp-uniform bounded wait (lane 0 polls)
    auto wwait = [&](uint64_t* b, uint32_t parity) -> bool {
      int good = 1;
      if (lane == 0) good = cwait(s, b, parity, args.status) ? 1 : 0;
      return __shfl_sync(0xffffffffu, good, 0) != 0;
    };
    // group-uniform wait (thread 0 polls, the compute warps sync)
    auto gwait = [&](uint64_t* b, uint32_t parity) -> bool {
      if (ct == 0) {
        cwait(s, b, parity, args.status);
        s.red[63] = *(volatile int*)s.abort ? 1.f : 0.f;
      }
      comp_sync();
      return s.red[63] == 0.f;
    };
    uint32_t center_n = 0;
    for (int64_t cell = blockIdx.x; cell < args.n; cell += gridDim.x) {
      if (ct == 0) s.red[63] = *(volatile int*)s.abort ? 1.f : 0.f;
      comp_sync();
      if (s.red[63] != 0.f) break;
      // ---- input box, z_1 centre, sigma_1, ReLU 1 ----
      float xc[3], h23[3];
      {
        const CellSource& src = args.src;
        float hh[3];
        if (src.codes) {
          uint32_t code = src.codes[cell];
          int ijk[3] = {int(code & 1023u), int((code >> 10) & 1023u), int((code >> 20) & 1023u)};
          for (int d = 0; d < 3; ++d) {
            const float size = ldexpf(2.0f, -axis_level(src, d));
            hh[d] = 0.5f * size;
            xc[d] = -1.0f + size * float(ijk[d]) + hh[d];
          }
        } else {
          for (int d = 0; d < 3; ++d) {
            float lo = src.lo[3 * cell + d], hi = src.hi[3 * cell + d];
            xc[d] = 0.5f * (lo + hi);
            hh[d] = 0.5f * (hi - lo);
          }
        }
        for (int d = 0; d < 3; ++d) h23[d] = hh[d] * hh[d] * (1.0f / 3.0f);   // variance of U[-h, h]
      }
      for (int p = ct; p < w; p += kCompThreads) {
        const float w0 = s.W0[3 * p], w1 = s.W0[3 * p + 1], w2 = s.W0[3 * p + 2];
        const float c1 = fmaf(w2, xc[2], fmaf(w1, xc[1], fmaf(w0, xc[0], args.b[0][p])));
        const float s2 = w0 * w0 * h23[0] + w1 * w1 * h23[1] + w2 * w2 * h23[2];
        Lin L = act_clt(args.act, c1, sqrtf(s2));
        s.alpha[p] = L.alpha;
        s.beta[p] = L.beta;
        s.gamma[p] = L.gamma;
        s.a[p] = L.center;
      }
      comp_sync();
      if (ct == 0) mbar_arrive(&s.bar[CB_RELU]);
      // ---- M_1 = D C_1 D + Gamma^2, C_1 = W_0 diag(h^2/3) W_0^T (rank 3), rows into Bm ----
      for (int p = ct; p < w; p += kCompThreads) {
        const float ap = s.alpha[p];
        const float u0 = ap * s.W0[3 * p] * h23[0], u1 = ap * s.W0[3 * p + 1] * h23[1], u2 = ap * s.W0[3 * p + 2] * h23[2];
        const float gp2 = s.gamma[p] * s.gamma[p];
        for (int col0 = 0; col0 < w; col0 += 32) {
          float v[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int qq = col0 + i;
            const float cq = u0 * s.W0[3 * qq] + u1 * s.W0[3 * qq + 1] + u2 * s.W0[3 * qq + 2];
            v[i] = s.alpha[qq] * cq + (qq == p ? gp2 : 0.0f);
          }
          store_row32(s.Bm, w, p, col0, v);
        }
      }
      fence_async_shared();
      tc_fence_before();
      comp_sync();
      if (ct == 0) mbar_arrive(&s.bar[CB_BREADY]);
      bool ok = true;
      for (int j = 1; j <= H - 1 && ok; ++j) {
        // ---- GEMM1 done: T^T = W_j M_j -> Bm (B operand of GEMM2) ----
        if (!wwait(&s.bar[CB_DFULL], dfull_n & 1)) { ok = false; break; }
        ++dfull_n;
        tc_fence_after();
        for (int mt = 0; mt < MT; ++mt) {
          const int p = mt * 128 + 32 * q + lane;
          const uint32_t tb = tmem + mt * 256 + ((uint32_t)(32 * q) << 16);
          for (int ch = 0; ch < nch; ++ch) {
            const int col0 = hf * half + ch * 32;
            float v[32];
            tmem_ld32(tb + col0, v);
            store_row32(s.Bm, w, p, col0, v);
          }
        }
        fence_async_shared();
        tc_fence_before();
        comp_sync();
        if (ct == 0) mbar_arrive(&s.bar[CB_BREADY]);
        // ---- GEMM2 done: C_{j+1} = W_j M_j W_j^T in TMEM ----
        if (!wwait(&s.bar[CB_DFULL], dfull_n & 1)) { ok = false; break; }
        ++dfull_n;
        tc_fence_after();
        for (int mt = 0; mt < MT; ++mt) {
          const int dcol = mt * 128 + 32 * q;           // diagonal block of this warp's rows
          if (dcol / half == hf) {
            float v[32];
            tmem_ld32(tmem + mt * 256 + ((uint32_t)(32 * q) << 16) + dcol, v);
            float d = 0.f;
#pragma unroll
            for (int i = 0; i < 32; ++i) d = (i == lane) ? v[i] : d;
            s.sig2[mt * 128 + 32 * q + lane] = fmaxf(d, 0.0f);
          }
        }
        // centre of z_{j+1} from the math warps, then ReLU j+1
        if (!gwait(&s.bar[CB_CENTER], center_n & 1)) { ok = false; break; }
        ++center_n;
        for (int p = ct; p < w; p += kCompThreads) {
          Lin L = act_clt(args.act, s.cn[p], sqrtf(s.sig2[p]));
          s.alpha[p] = L.alpha;
          s.beta[p] = L.beta;
          s.gamma[p] = L.gamma;
          s.a[p] = L.center;
          if (j == H - 1) s.aw[p] = L.alpha * args.wout[p];
        }
        comp_sync();
        if (j + 1 <= H - 1) {
          if (ct == 0) mbar_arrive(&s.bar[CB_RELU]);
          // M_{j+1} = alpha alpha^T * C + diag(gamma^2) -> Bm
          for (int mt = 0; mt < MT; ++mt) {
            const int p = mt * 128 + 32 * q + lane;
            const float ap = s.alpha[p], gp2 = s.gamma[p] * s.gamma[p];
            const uint32_t tb = tmem + mt * 256 + ((uint32_t)(32 * q) << 16);
            for (int ch = 0; ch < nch; ++ch) {
              const int col0 = hf * half + ch * 32;
              float v[32];
              tmem_ld32(tb + col0, v);
#pragma unroll
              for (int i = 0; i < 32; ++i) v[i] = ap * s.alpha[col0 + i] * v[i] + ((col0 + i) == p ? gp2 : 0.0f);
              store_row32(s.Bm, w, p, col0, v);
            }
          }
          fence_async_shared();
          tc_fence_before();
          comp_sync();
          if (ct == 0) mbar_arrive(&s.bar[CB_BREADY]);
        } else {
          // output layer: sigma^2 = sum_pq (alpha w)_p C_pq (alpha w)_q + sum_p (gamma_p w_p)^2, mu = w . a + b
          float part = 0.f;
          for (int mt = 0; mt < MT; ++mt) {
            const int p = mt * 128 + 32 * q + lane;
            const uint32_t tb = tmem + mt * 256 + ((uint32_t)(32 * q) << 16);
            float rowsum = 0.f;
            for (int ch = 0; ch < nch; ++ch) {
              const int col0 = hf * half + ch * 32;
              float v[32];
              tmem_ld32(tb + col0, v);
#pragma unroll
              for (int i = 0; i < 32; ++i) rowsum = fmaf(s.aw[col0 + i], v[i], rowsum);
            }
            part = fmaf(s.aw[p], rowsum, part);
            if (hf == 0) {
              const float gw = s.gamma[p] * args.wout[p];
              part = fmaf(gw, gw, part);
            }
          }
          float mu = 0.f;
          for (int p = ct; p < w; p += kCompThreads) mu = fmaf(args.wout[p], s.a[p], mu);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            part += __shfl_xor_sync(0xffffffffu, part, o);
            mu += __shfl_xor_sync(0xffffffffu, mu, o);
          }
          tc_fence_before();
          comp_sync();
          if (lane == 0) {
            s.red[2 * (warp - 2)] = part;
            s.red[2 * (warp - 2) + 1] = mu;
          }
          comp_sync();
          if (ct == 0) {
            float sg = 0.f, m = 0.f;
            for (int i = 0; i < kCompWarps; ++i) {
              sg += s.red[2 * i];
              m += s.red[2 * i + 1];
            }
            args.center[cell] = m + args.bout;
            args.spread[cell] = sqrtf(fmaxf(sg, 0.0f));
          }
        }
      }
      if (!ok) break;
    }
  } else {
    // ================================ math warps: c_{j+1} = W_j a_j + b_j ================================
    const int mt_ = threadIdx.x - kMathBaseC;   // 0 .. 127
    uint32_t relu_n = 0;
    for (int64_t cell = blockIdx.x; cell < args.n; cell += gridDim.x) {
      bool ok = true;
      for (int j = 1; j <= H - 1; ++j) {
        if (mt_ == 0) {
          cwait(s, &s.bar[CB_RELU], relu_n & 1, args.status);
          s.red[62] = *(volatile int*)s.abort ? 1.f : 0.f;
        }
        math_sync_c();
        if (s.red[62] != 0.f) { ok = false; break; }
        ++relu_n;
        const int LG = w / 4, grp = mt_ / LG, ln = mt_ % LG, kh = w / 2;
        float4 cc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (mt_ < 2 * LG) {
          const float4* Wp = reinterpret_cast<const float4*>(args.Wt[j]) + ln;
          const int kb = grp * kh;
          for (int k0 = kb; k0 < kb + kh; k0 += 16) {
            float4 wv[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) wv[u] = __ldg(Wp + (size_t)(k0 + u) * LG);
#pragma unroll
            for (int u = 0; u < 16; ++u) {
              const float ak = s.a[k0 + u];
              cc.x = fmaf(wv[u].x, ak, cc.x);
              cc.y = fmaf(wv[u].y, ak, cc.y);
              cc.z = fmaf(wv[u].z, ak, cc.z);
              cc.w = fmaf(wv[u].w, ak, cc.w);
            }
          }
          if (grp == 1) reinterpret_cast<float4*>(s.cn)[ln] = cc;
        }
        math_sync_c();
        if (mt_ < LG) {
          const float4 t = reinterpret_cast<const float4*>(s.cn)[ln];
          const float4 bb = reinterpret_cast<const float4*>(args.b[j])[ln];
          reinterpret_cast<float4*>(s.cn)[ln] =
              make_float4(cc.x + t.x + bb.x, cc.y + t.y + bb.y, cc.z + t.z + bb.z, cc.w + t.w + bb.w);
        }
        math_sync_c();
        if (mt_ == 0) mbar_arrive(&s.bar[CB_CENTER]);
      }
      if (!ok) break;
    }
  }

  __syncthreads();
  if (*(volatile int*)s.abort) {
    for (int i = 0; i < 1000; ++i) __nanosleep(1000);
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

}  // namespace

isx_status bound_bf16_clt_cov(isx_inr inr, const CellSource& src, int64_t n, float* d_center, float* d_spread,
                              cudaStream_t st) {
  if (n <= 0) return ISX_OK;
  const int w = inr->w, H = inr->H;
  if (!((w == 128 || w == 256) && H >= 2 && H <= ISX_MAX_LAYERS - 1)) {
    set_error("covariance CLT kernel supports hidden widths 128 and 256");
    return ISX_ERR_UNSUPPORTED;
  }
  int sms = 0;
  ISX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, inr->device));
  const int grid = (int)std::min<int64_t>(n, sms);
  auto& ws = inr->ws;
  ISX_TRY(ws[WS_TC_STATUS].ensure(64, "tc status"));
  CovArgs a{};
  a.src = src;
  a.n = n;
  a.w = w;
  a.H = H;
  a.act = inr->act;
  a.W0 = inr->W[0];
  for (int l = 0; l < inr->n_layers; ++l) {
    a.b[l] = inr->b[l];
    a.Wt[l] = inr->Wt[l];
  }
  a.wout = inr->W[inr->n_layers - 1];
  a.bout = inr->hb[inr->n_layers - 1][0];
  a.center = d_center;
  a.spread = d_spread;
  a.status = ws[WS_TC_STATUS].as<int>();
  CovMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int l = 1; l < inr->n_layers - 1; ++l) ISX_TRY(tensor_map_bf16(&maps.wrow[l], inr->W_bf16[l], w, w, 64, 128));
  ISX_CUDA(cudaMemsetAsync(a.status, 0, sizeof(int), st));
  const size_t smem = cov_smem_bytes(w);
  ISX_CUDA(cudaFuncSetAttribute(k_bound_cov, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  {
    // algorithmic work of the coefficient form (the method as printed): 2 w^2 (3 (H-1) + w (H-1)(H-2)/2)
    const double flops = (double)n * 2.0 * w * w * (3.0 * (H - 1) + (double)w * (H - 1) * (H - 2) / 2.0);
    prof::Scope ps(K_BOUND_COV, st, flops, 0);
    k_bound_cov<<<grid, kThreadsC, smem, st>>>(a, maps);
  }
  ISX_LAUNCH_CHECK("k_bound_cov");
  int status = 0;
  ISX_CUDA(cudaMemcpyAsync(&status, a.status, sizeof(int), cudaMemcpyDeviceToHost, st));
  ISX_CUDA(cudaStreamSynchronize(st));
  if (status != 0) {
    set_error("covariance bound kernel gave up waiting (bounded wait expired)");
    return (isx_status)status;
  }
  return ISX_OK;
}

}  // namespace isx
