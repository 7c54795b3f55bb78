// Tensor-core bound path: one persistent kernel bounds whole cells, all layers, on tcgen05.
//
// Structure of the coefficient matrix (Sec. III-B / IV-C).  For the pre-activation z_j of hidden
// layer j the rows (noise symbols) form blocks: I (the 3 input symbols) and G_k (the w symbols
// created by ReLU k), k < j.  Through ReLU j and linear layer j (Eq. 4 / 9 then Eq. 3 / 8):
//   I' = I D_j W_j^T,   G_k' = G_k D_j W_j^T (k < j),   G_j' = diag(gamma_j) W_j^T,   D_j = diag(alpha_j).
// G_j' is never materialised ("implicit"): its reductions are GEMVs with |W_j| (or W_j^2), and at
// the next layer it enters the product as A = W_j^T (shared by all cells) with the rows scaled by
// gamma_j in the epilogue.  Layer j is therefore one GEMM with M = w (j - 1) rows of G blocks,
// K = N = w, B = D_j W_j^T; the 3 I rows, the centre and all GEMVs run on CUDA cores.
// The last hidden GEMM only feeds the reductions of the last ReLU and is not stored; the output
// layer is rewritten through the previous layer: y = X_{H-1} (alpha_{H-1} * v) with
// v = W_{H-1}^T (alpha_H * w_out), which a short N = 16 tensor-core pass computes.
//
// GB300 mapping.  One CTA per SM walks over cells.  The cell's stored G blocks live in a private
// global scratch slice (<= w (H - 3) rows of bfloat16, 256 KB at w = 256, H = 5), updated in place,
// small enough across 148-152 CTAs to stay resident in the 126 MB L2.  Per layer, B = D_j W_j^T
// is staged once in shared memory (TMA load of W_j in bfloat16, then scaled by alpha_j in place),
// A tiles (128 rows x 64 K, 128-byte swizzle) stream through a TMA ring, tcgen05.mma (M = 128,
// N = w, K = 16, bf16 x bf16 -> f32) accumulates in TMEM (two 256-column accumulators), and the
// epilogue (8 warps) reads TMEM, scales implicit rows by gamma, rounds to bfloat16, stores the
// rows back to scratch and reduces every column (sum |x| or sum x^2) with a warp-transpose
// butterfly (pairwise summation), compensated across tiles.  4 math warps do the ReLU
// linearisation, the bfloat16 scaling of B, the I rows, the centre and all GEMVs.
//
// Warp roles: 0 = TMA producer, 1 = MMA issuer (and TMEM owner), 2-9 = epilogue, 10-13 = math.
// Every wait is bounded: on timeout the kernel records ISX_ERR_TIMEOUT, lets copies in flight
// land, frees its TMEM and returns.
//
// Rounding-error inflation (SOUND, inflate != 0): stored coefficients and B are bfloat16
// (unit roundoff u_b = 2^-8; B is rounded twice: W to bf16, then alpha * W), tensor-core
// accumulation is bounded with a conservative unit roundoff u_a = 2^-17 per addition, CUDA-core
// float32 with u = 2^-24.  The slack of neuron n of z_{j+1} is
//   kappa * sum_k |W_j[n,k]| (alpha_k r_k + gamma_k) + u_b/(1-u_b) * (sum of stored |x|)
//   + gamma_{K+2} (sum_k |W_j[n,k] a_k| + |b_n|),  kappa = (1+u_b)^3 (1+gamma_K(u_a)) (1+u) - 1,
// and the output radius adds kappa_out times the matching absolute sums.
#include "internal.cuh"
#include "linearise.cuh"
#include "tc_ptx.cuh"

#include <cuda.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace isx {
namespace {

constexpr int kStages = 3;
constexpr int kEpiWarps = 8;
constexpr int kMathWarps = 4;
constexpr int kThreads = 32 * (2 + kEpiWarps + kMathWarps);   // 448
constexpr int kMathThreads = 32 * kMathWarps;
constexpr int kMathBase = 32 * (2 + kEpiWarps);                // first math thread
constexpr uint32_t kStageBytes = 128 * 128;                    // 128 rows x 64 bf16
constexpr uint64_t kWaitNs = 2000000000ull;                    // 2 s per wait
constexpr float kUb = 0.00390625f;                             // 2^-8
constexpr float kUa = 7.62939453125e-06f;                      // 2^-17

struct TcArgs {
  CellSource src;
  int64_t n;
  int mode, inflate, w, H;
  const float* W[ISX_MAX_LAYERS];
  const float* Wt[ISX_MAX_LAYERS];
  const float* b[ISX_MAX_LAYERS];
  float bout;
  __nv_bfloat16* scratch;
  int rows_per_cta;
  float* center;
  float* spread;
  int* status;
  float kappa, kappa_out;
  long long* trace;     // optional per-phase clock64 stamps of CTA 0 (ISX_TRACE=1)
};

using namespace tc;
__device__ __forceinline__ void math_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kMathThreads) : "memory"); }

struct TcMaps {
  CUtensorMap scratch;                 // [rows][w] bf16, box {64, 128}
  CUtensorMap wt[ISX_MAX_LAYERS];      // W_l^T bf16 [w][w], box {64, 128}: implicit-block A
  CUtensorMap wrow[ISX_MAX_LAYERS];    // W_l bf16 [w][w], box {64, w}: source of B
};

// ---- shared-memory layout ------------------------------------------------------------------------------
struct Smem {
  uint8_t* B;        // w/64 chunks of [w rows][128 B]
  uint8_t* A;        // kStages x 16 KB
  uint8_t* Bout;     // w/64 chunks of [16 rows][128 B]
  float* alpha;      // [3][w] (slot = layer % 3)
  float* gamma;      // [3][w]
  float* c;          // centre of the current z
  float* r;          // radius / sigma of the current z (all rows)
  float* delta;      // slack of the current z
  float* a;          // a-form centre
  float* rada;       // a-form radius (sound)
  float* red;        // [4][w] epilogue partial reductions
  float* I;          // [3][w] input-symbol rows of the current z
  float* Ia;         // [3][w] I rows times alpha
  float* Inew;       // [3][w] next layer's I rows
  float* rprev;      // radius of the previous z
  float* rpart;      // CUDA-core part of the next radius
  float* spart;      // CUDA-core part of the next slack
  float* v;          // [w]
  float* u;          // [w]
  float* tmp;        // [w]
  float* scal;       // [64] block-reduction scratch
  uint64_t* bar;     // barriers
  uint32_t* tmem_slot;
  int* abort;
};

enum Bars { BAR_FULL = 0, BAR_EMPTY = kStages, BAR_TFULL = 2 * kStages, BAR_TEMPTY = 2 * kStages + 2,
            BAR_BREADY = 2 * kStages + 4, BAR_BFREE, BAR_WLOADED, BAR_RED, BAR_BOUTREADY, BAR_COUNT };

__host__ __device__ inline size_t smem_bytes(int w) {
  size_t off = 0;
  off += (size_t)w * w * 2;                 // B
  off += (size_t)kStages * kStageBytes;     // A
  off += (size_t)16 * w * 2;                // Bout
  off += (size_t)(3 + 3 + 5 + 4 + 3 + 3 + 3 + 3 + 3) * w * 4 + 64 * 4;
  off += BAR_COUNT * 8 + 16;
  return off + 1024;                        // alignment slack
}

__device__ Smem carve(uint8_t* raw, int w) {
  uintptr_t base = ((uintptr_t)raw + 1023) & ~(uintptr_t)1023;
  uint8_t* p = (uint8_t*)base;
  Smem s;
  s.B = p; p += (size_t)w * w * 2;
  s.A = p; p += (size_t)kStages * kStageBytes;
  s.Bout = p; p += (size_t)16 * w * 2;
  float* f = (float*)p;
  s.alpha = f; f += 3 * w;
  s.gamma = f; f += 3 * w;
  s.c = f; f += w;
  s.r = f; f += w;
  s.delta = f; f += w;
  s.a = f; f += w;
  s.rada = f; f += w;
  s.red = f; f += 4 * w;
  s.I = f; f += 3 * w;
  s.Ia = f; f += 3 * w;
  s.Inew = f; f += 3 * w;
  s.rprev = f; f += w;
  s.rpart = f; f += w;
  s.spart = f; f += w;
  s.v = f; f += w;
  s.u = f; f += w;
  s.tmp = f; f += w;
  s.scal = f; f += 64;
  s.bar = (uint64_t*)(((uintptr_t)f + 7) & ~(uintptr_t)7);
  s.tmem_slot = (uint32_t*)(s.bar + BAR_COUNT);
  s.abort = (int*)(s.tmem_slot + 1);
  return s;
}

// Bounded wait (kWaitNs of wall time); on timeout raises the CTA-wide abort flag and the global
// status and returns false.  Also returns false as soon as another role has aborted.
__device__ __forceinline__ bool wait_bar(const Smem& s, uint64_t* b, uint32_t parity, int* status) {
  if (mbar_try(b, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try(b, parity)) return true;
    if ((it & 3) == 0) {
      if (*(volatile int*)s.abort) return false;
      if (global_ns() - t0 > kWaitNs) {
        *(volatile int*)s.abort = 1;
        atomicExch(status, (int)ISX_ERR_TIMEOUT);
        return false;
      }
    }
  }
}

// Trace slots: [role][cell < kTraceCells][event < kTraceEvents]
constexpr int kTraceCells = 4, kTraceEvents = 48;
__device__ __forceinline__ void trace(const TcArgs& a, int role, int64_t cell, int ev) {
  if (a.trace && blockIdx.x == 0 && cell < kTraceCells && ev < kTraceEvents)
    a.trace[(role * kTraceCells + cell) * kTraceEvents + ev] = clock64();
}

__device__ __forceinline__ int tiles_per_block(int w) { return w / 128; }
// TC layers are j = 2 .. H-1; layer j has (j - 1) blocks of w rows.
__device__ __forceinline__ int layer_tiles(int j, int w) { return (j - 1) * tiles_per_block(w); }
__device__ __forceinline__ int out_tiles(int H, int w) { return H >= 4 ? (H - 3) * tiles_per_block(w) : 0; }

// ---- the kernel ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 1) k_bound_tc(const __grid_constant__ TcArgs args,
                                                           const __grid_constant__ TcMaps maps) {
  extern __shared__ uint8_t smem_raw[];
  const int w = args.w, H = args.H;
  Smem s = carve(smem_raw, w);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkc = w / 64;                  // 64-wide K chunks
  const int mode = args.mode;
  const bool clt = mode == ISX_BOUND_CLT;
  const bool infl = args.inflate != 0 && mode == ISX_BOUND_SOUND;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&s.bar[BAR_FULL + i], 1);
      mbar_init(&s.bar[BAR_EMPTY + i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&s.bar[BAR_TFULL + i], 1);
      mbar_init(&s.bar[BAR_TEMPTY + i], kEpiWarps);
    }
    mbar_init(&s.bar[BAR_BREADY], 1);
    mbar_init(&s.bar[BAR_BFREE], 1);
    mbar_init(&s.bar[BAR_WLOADED], 1);
    mbar_init(&s.bar[BAR_RED], kEpiWarps);
    mbar_init(&s.bar[BAR_BOUTREADY], 1);
    *s.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // zero Bout (rows 1..15 stay zero)
  for (int i = threadIdx.x; i < 16 * w * 2 / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(s.Bout)[i] = make_uint4(0, 0, 0, 0);
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(su32(s.tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_shared();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s.tmem_slot;
  __nv_bfloat16* scratch = args.scratch + (size_t)blockIdx.x * args.rows_per_cta * w;
  const int scratch_row0 = blockIdx.x * args.rows_per_cta;

  if (warp == 0) {
    // ================================ TMA producer ================================
    if (lane == 0) {
      uint32_t stage = 0, sphase = 0, bfree_n = 0, red_n = 0;
      for (int64_t cell = blockIdx.x; cell < args.n && !*(volatile int*)s.abort; cell += gridDim.x) {
        for (int j = 2; j <= H - 1; ++j) {
          // B source: W_j (bf16) into the B buffer once the previous B is no longer read
          if (!wait_bar(s, &s.bar[BAR_BFREE], (bfree_n & 1) ^ 1, args.status)) break;
          ++bfree_n;
          mbar_expect_tx(&s.bar[BAR_WLOADED], (uint32_t)(w * w * 2));
          for (int c = 0; c < nkc; ++c) tma_load_2d(s.B + (size_t)c * w * 128, &maps.wrow[j], &s.bar[BAR_WLOADED], c * 64, 0);
          // rows written by the previous layer must be complete before they are read
          if (j >= 3) {
            if (!wait_bar(s, &s.bar[BAR_RED], red_n & 1, args.status)) break;
            ++red_n;
          }
          const int T = layer_tiles(j, w), tb = tiles_per_block(w);
          for (int t = 0; t < T; ++t) {
            const int blk = t / tb + 1, sub = t % tb;      // G_blk
            const bool implicit = (blk == j - 1);
            for (int c = 0; c < nkc; ++c) {
              if (!wait_bar(s, &s.bar[BAR_EMPTY + stage], sphase ^ 1, args.status)) break;
              mbar_expect_tx(&s.bar[BAR_FULL + stage], kStageBytes);
              uint8_t* dst = s.A + (size_t)stage * kStageBytes;
              if (implicit) tma_load_2d(dst, &maps.wt[j - 1], &s.bar[BAR_FULL + stage], c * 64, sub * 128);
              else tma_load_2d(dst, &maps.scratch, &s.bar[BAR_FULL + stage], c * 64, scratch_row0 + (blk - 1) * w + sub * 128);
              if (++stage == kStages) { stage = 0; sphase ^= 1; }
            }
          }
        }
        // red_ready of the last TC layer (not waited above) keeps the phase count in step
        if (H >= 3) {
          if (!wait_bar(s, &s.bar[BAR_RED], red_n & 1, args.status)) break;
          ++red_n;
        }
        const int TO = out_tiles(H, w);
        for (int t = 0; t < TO; ++t) {
          for (int c = 0; c < nkc; ++c) {
            if (!wait_bar(s, &s.bar[BAR_EMPTY + stage], sphase ^ 1, args.status)) break;
            mbar_expect_tx(&s.bar[BAR_FULL + stage], kStageBytes);
            tma_load_2d(s.A + (size_t)stage * kStageBytes, &maps.scratch, &s.bar[BAR_FULL + stage], c * 64,
                        scratch_row0 + t * 128);
            if (++stage == kStages) { stage = 0; sphase ^= 1; }
          }
        }
        if (TO > 0) {
          if (!wait_bar(s, &s.bar[BAR_RED], red_n & 1, args.status)) break;
          ++red_n;
        }
      }
    }
  } else if (warp == 1) {
    // ================================ MMA issuer ================================
    if (lane == 0) {
      uint32_t stage = 0, sphase = 0, bready_n = 0, bout_n = 0, tiles_done = 0;
      const uint32_t id_main = idesc(w), id_out = idesc(16);
      for (int64_t cell = blockIdx.x; cell < args.n && !*(volatile int*)s.abort; cell += gridDim.x) {
        bool ok = true;
        for (int j = 2; j <= H - 1 && ok; ++j) {
          if (!wait_bar(s, &s.bar[BAR_BREADY], bready_n & 1, args.status)) { ok = false; break; }
          ++bready_n;
          trace(args, 1, cell / gridDim.x, 2 * j);
          tc_fence_after();
          const int T = layer_tiles(j, w);
          for (int t = 0; t < T && ok; ++t) {
            const uint32_t acc = tiles_done & 1;
            if (!wait_bar(s, &s.bar[BAR_TEMPTY + acc], ((tiles_done >> 1) & 1) ^ 1, args.status)) { ok = false; break; }
            tc_fence_after();
            const uint32_t d = tmem + acc * 256;
            for (int c = 0; c < nkc; ++c) {
              if (!wait_bar(s, &s.bar[BAR_FULL + stage], sphase, args.status)) { ok = false; break; }
              tc_fence_after();
              const uint32_t a0 = su32(s.A + (size_t)stage * kStageBytes);
              const uint32_t b0 = su32(s.B + (size_t)c * w * 128);
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)
                mma_bf16(d, sdesc(a0 + kk * 32), sdesc(b0 + kk * 32), id_main, (c > 0 || kk > 0) ? 1u : 0u);
              mma_commit(&s.bar[BAR_EMPTY + stage]);
              if (++stage == kStages) { stage = 0; sphase ^= 1; }
            }
            mma_commit(&s.bar[BAR_TFULL + acc]);
            ++tiles_done;
          }
          mma_commit(&s.bar[BAR_BFREE]);
          trace(args, 1, cell / gridDim.x, 2 * j + 1);
        }
        if (!ok) break;
        const int TO = out_tiles(H, w);
        if (TO > 0) {
          if (!wait_bar(s, &s.bar[BAR_BOUTREADY], bout_n & 1, args.status)) break;
          ++bout_n;
          tc_fence_after();
          for (int t = 0; t < TO && ok; ++t) {
            const uint32_t acc = tiles_done & 1;
            if (!wait_bar(s, &s.bar[BAR_TEMPTY + acc], ((tiles_done >> 1) & 1) ^ 1, args.status)) { ok = false; break; }
            tc_fence_after();
            const uint32_t d = tmem + acc * 256;
            for (int c = 0; c < nkc; ++c) {
              if (!wait_bar(s, &s.bar[BAR_FULL + stage], sphase, args.status)) { ok = false; break; }
              tc_fence_after();
              const uint32_t a0 = su32(s.A + (size_t)stage * kStageBytes);
              const uint32_t b0 = su32(s.Bout + (size_t)c * 16 * 128);
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)
                mma_bf16(d, sdesc(a0 + kk * 32), sdesc(b0 + kk * 32), id_out, (c > 0 || kk > 0) ? 1u : 0u);
              mma_commit(&s.bar[BAR_EMPTY + stage]);
              if (++stage == kStages) { stage = 0; sphase ^= 1; }
            }
            mma_commit(&s.bar[BAR_TFULL + acc]);
            ++tiles_done;
          }
        }
      }
    }
  } else if (warp < 2 + kEpiWarps) {
    // ================================ epilogue ================================
    const int q = warp & 3;                    // TMEM lane quarter this warp may access
    const int hf = (warp - 2) >> 2;            // column half
    const int half = w / 2, nch = half / 32;   // columns and 32-column chunks per half
    uint32_t tiles_done = 0;
    for (int64_t cell = blockIdx.x; cell < args.n; cell += gridDim.x) {
      if (__shfl_sync(0xffffffffu, *(volatile int*)s.abort, 0)) break;
      bool ok = true;
      const int TO = out_tiles(H, w);
      for (int j = 2; j <= H && ok; ++j) {
        const bool outpass = (j == H);
        if (outpass && TO == 0) break;
        const bool store = !outpass && (j < H - 1);
        const int T = outpass ? TO : layer_tiles(j, w);
        const int tb = tiles_per_block(w);
        float p[4] = {0.f, 0.f, 0.f, 0.f}, comp[4] = {0.f, 0.f, 0.f, 0.f};
        float pout = 0.f;
        const float* gprev = s.gamma + ((j - 1) % 3) * w;   // gamma_{j-1}: scale of implicit rows
        for (int t = 0; t < T; ++t) {
          const uint32_t acc = tiles_done & 1;
          {
            int good = 1;
            if (lane == 0) good = wait_bar(s, &s.bar[BAR_TFULL + acc], (tiles_done >> 1) & 1, args.status) ? 1 : 0;
            good = __shfl_sync(0xffffffffu, good, 0);
            if (!good) { ok = false; break; }
          }
          tc_fence_after();
          const uint32_t tbase = tmem + acc * 256 + ((uint32_t)(32 * q) << 16);
          const int row = 32 * q + lane;                     // row within the tile
          if (outpass) {
            if (hf == 0) {
              float y = tmem_ld1(tbase);
              float x = clt || mode == ISX_BOUND_RAUA ? y * y : fabsf(y);
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
              pout += x;
            }
          } else {
            const int blk = t / tb + 1, sub = t % tb;
            const bool implicit = (blk == j - 1);
            const float rs = implicit ? gprev[sub * 128 + row] : 1.0f;
            __nv_bfloat16* dst = scratch + (size_t)((blk - 1) * w + sub * 128 + row) * w;
            for (int ch = 0; ch < nch; ++ch) {
              const int col0 = hf * half + ch * 32;
              float v[32];
              tmem_ld32(tbase + col0, v);
              if (store) {
                uint32_t pk[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                  __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * i] * rs, v[2 * i + 1] * rs);
                  pk[i] = *reinterpret_cast<uint32_t*>(&h2);
                  float2 f2 = __bfloat1622float2(h2);
                  v[2 * i] = f2.x;
                  v[2 * i + 1] = f2.y;
                }
                uint4* d4 = reinterpret_cast<uint4*>(dst + col0);
#pragma unroll
                for (int i = 0; i < 4; ++i) d4[i] = make_uint4(pk[4 * i], pk[4 * i + 1], pk[4 * i + 2], pk[4 * i + 3]);
              } else {
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] *= rs;
              }
#pragma unroll
              for (int i = 0; i < 32; ++i) v[i] = clt ? v[i] * v[i] : fabsf(v[i]);
              float sum = transpose_reduce32(v);
              // compensated accumulation across tiles
              float y = sum - comp[ch];
              float tt = p[ch] + y;
              comp[ch] = (tt - p[ch]) - y;
              p[ch] = tt;
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&s.bar[BAR_TEMPTY + acc]);
          ++tiles_done;
        }
        if (!ok) break;
        if (warp == 2 && lane == 0) trace(args, 2, cell / gridDim.x, j);
        if (store) fence_async_global();
        if (outpass) {
          if (hf == 0 && lane == 0) s.red[q * w] = pout;
        } else {
          for (int ch = 0; ch < nch; ++ch) s.red[q * w + hf * half + ch * 32 + lane] = p[ch];
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&s.bar[BAR_RED]);
      }
      if (!ok) break;
    }
  } else {
    // ================================ math ================================
    const int mt = threadIdx.x - kMathBase;    // 0..127
    uint32_t wl_n = 0, red_n = 0;
    const float kap = args.kappa;
    const bool sq = clt || mode == ISX_BOUND_RAUA;
    // uniform decisions: thread 0 of the group waits / reads the abort flag, the group syncs
    auto group_wait = [&](uint64_t* b, uint32_t parity) -> bool {
      if (mt == 0) {
        wait_bar(s, b, parity, args.status);
        s.scal[63] = *(volatile int*)s.abort ? 1.f : 0.f;
      }
      math_sync();
      return s.scal[63] == 0.f;
    };
    for (int64_t cell = blockIdx.x; cell < args.n; cell += gridDim.x) {
      if (mt == 0) s.scal[63] = *(volatile int*)s.abort ? 1.f : 0.f;
      math_sync();
      if (s.scal[63] != 0.f) break;
      bool ok = true;
      if (mt == 0) trace(args, 0, cell / gridDim.x, 0);
      // ---- input layer z_1 = W_0 x + b_0 over the box (Sec. III-B / IV-C) ----
      float xc[3], h[3];
      {
        const CellSource& src = args.src;
        if (src.codes) {
          uint32_t code = src.codes[cell];
          float size = ldexpf(2.0f, -src.level);
          int ijk[3] = {int(code & 1023u), int((code >> 10) & 1023u), int((code >> 20) & 1023u)};
          for (int d = 0; d < 3; ++d) {
            h[d] = 0.5f * size;
            xc[d] = -1.0f + size * float(ijk[d]) + h[d];
          }
        } else {
          for (int d = 0; d < 3; ++d) {
            float lo = src.lo[3 * cell + d], hi = src.hi[3 * cell + d];
            xc[d] = 0.5f * (lo + hi);
            h[d] = infl ? __fadd_ru(__fmul_ru(__fsub_ru(hi, lo), 0.5f), fabsf(xc[d]) * 1.2e-7f) : 0.5f * (hi - lo);
          }
        }
        if (clt)
          for (int d = 0; d < 3; ++d) h[d] *= 0.57735026918962576f;
      }
      const float* W0 = args.W[0];
      for (int nn = mt; nn < w; nn += kMathThreads) {
        float w0 = W0[3 * nn], w1 = W0[3 * nn + 1], w2 = W0[3 * nn + 2], b0 = args.b[0][nn];
        float c = fmaf(w2, xc[2], fmaf(w1, xc[1], fmaf(w0, xc[0], b0)));
        float x0 = h[0] * w0, x1 = h[1] * w1, x2 = h[2] * w2;
        s.I[nn] = x0;
        s.I[w + nn] = x1;
        s.I[2 * w + nn] = x2;
        s.c[nn] = c;
        float r = clt ? sqrtf(x0 * x0 + x1 * x1 + x2 * x2) : fabsf(x0) + fabsf(x1) + fabsf(x2);
        s.r[nn] = r;
        s.rprev[nn] = r;
        s.delta[nn] = infl ? (5.0f * kLinU * (fabsf(w0 * xc[0]) + fabsf(w1 * xc[1]) + fabsf(w2 * xc[2]) + fabsf(b0)) +
                              3.0f * kLinU * r) * kLinSafe
                           : 0.0f;
      }
      math_sync();
      if (mt == 0) trace(args, 0, cell / gridDim.x, 1);
      for (int j = 1; j <= H - 1; ++j) {
        float* al = s.alpha + (j % 3) * w;
        float* ga = s.gamma + (j % 3) * w;
        // ---- ReLU j (Eq. 4 / Eq. 9) ----
        for (int nn = mt; nn < w; nn += kMathThreads) {
          Lin L = clt ? relu_clt(s.c[nn], s.r[nn]) : relu_sound(s.c[nn], s.r[nn], s.delta[nn], infl);
          al[nn] = L.alpha;
          ga[nn] = L.gamma;
          s.a[nn] = L.center;
          s.rada[nn] = infl ? fmaf(L.alpha, s.r[nn], L.gamma) : 0.0f;
          for (int rr = 0; rr < 3; ++rr) s.Ia[rr * w + nn] = s.I[rr * w + nn] * L.alpha;
        }
        if (j >= 2) {
          // ---- B = D_j W_j^T in place: scale the bf16 rows of W_j (K-major, 128-byte swizzle) ----
          if (!group_wait(&s.bar[BAR_WLOADED], wl_n & 1)) { ok = false; break; }
          ++wl_n;
          const int units = nkc * w * 8;   // 16-byte units
          for (int uidx = mt; uidx < units; uidx += kMathThreads) {
            const int c = uidx / (w * 8), rem = uidx % (w * 8), nrow = rem >> 3, pu = rem & 7;
            const int k0 = c * 64 + 8 * (pu ^ (nrow & 7));
            uint4* ptr = reinterpret_cast<uint4*>(s.B + (size_t)c * w * 128 + nrow * 128 + pu * 16);
            uint4 val = *ptr;
            __nv_bfloat162* hv = reinterpret_cast<__nv_bfloat162*>(&val);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              float2 f = __bfloat1622float2(hv[i]);
              hv[i] = __floats2bfloat162_rn(f.x * al[k0 + 2 * i], f.y * al[k0 + 2 * i + 1]);
            }
            *ptr = val;
          }
          fence_async_shared();
          math_sync();
          if (mt == 0) mbar_arrive(&s.bar[BAR_BREADY]);
        } else {
          math_sync();
        }
        if (mt == 0) trace(args, 0, cell / gridDim.x, 2 + 4 * (j - 1));
        // ---- CUDA-core part of linear layer j: centre, I rows, implicit block G_j, slack ----
        // Every thread owns 4 consecutive neurons (float4 loads of W_j^T rows) for one half of
        // the k range; the two halves are combined through shared memory.
        {
          const float* Wt = args.Wt[j];
          const int LG = w / 4, grp = mt / LG, ln = mt % LG, kh = w / 2;
          float4 cc = make_float4(0.f, 0.f, 0.f, 0.f), i0 = cc, i1 = cc, i2 = cc, imp = cc, ee = cc, gg = cc;
          if (mt < 2 * LG) {
            const float4* Wp = reinterpret_cast<const float4*>(Wt) + ln;
            const int kb = grp * kh;
#pragma unroll 16
            for (int k = kb; k < kb + kh; ++k) {
              const float4 wk = __ldg(Wp + (size_t)k * LG);
              const float ak = s.a[k], gk = ga[k], q0 = s.Ia[k], q1 = s.Ia[w + k], q2 = s.Ia[2 * w + k];
              cc.x = fmaf(wk.x, ak, cc.x); cc.y = fmaf(wk.y, ak, cc.y); cc.z = fmaf(wk.z, ak, cc.z); cc.w = fmaf(wk.w, ak, cc.w);
              i0.x = fmaf(wk.x, q0, i0.x); i0.y = fmaf(wk.y, q0, i0.y); i0.z = fmaf(wk.z, q0, i0.z); i0.w = fmaf(wk.w, q0, i0.w);
              i1.x = fmaf(wk.x, q1, i1.x); i1.y = fmaf(wk.y, q1, i1.y); i1.z = fmaf(wk.z, q1, i1.z); i1.w = fmaf(wk.w, q1, i1.w);
              i2.x = fmaf(wk.x, q2, i2.x); i2.y = fmaf(wk.y, q2, i2.y); i2.z = fmaf(wk.z, q2, i2.z); i2.w = fmaf(wk.w, q2, i2.w);
              if (clt) {
                const float tx = wk.x * gk, ty = wk.y * gk, tz = wk.z * gk, tw = wk.w * gk;
                imp.x = fmaf(tx, tx, imp.x); imp.y = fmaf(ty, ty, imp.y); imp.z = fmaf(tz, tz, imp.z); imp.w = fmaf(tw, tw, imp.w);
              } else {
                imp.x = fmaf(fabsf(wk.x), gk, imp.x); imp.y = fmaf(fabsf(wk.y), gk, imp.y);
                imp.z = fmaf(fabsf(wk.z), gk, imp.z); imp.w = fmaf(fabsf(wk.w), gk, imp.w);
                if (infl) {
                  const float aa = fabsf(ak), ra = s.rada[k];
                  ee.x = fmaf(fabsf(wk.x), aa, ee.x); ee.y = fmaf(fabsf(wk.y), aa, ee.y);
                  ee.z = fmaf(fabsf(wk.z), aa, ee.z); ee.w = fmaf(fabsf(wk.w), aa, ee.w);
                  gg.x = fmaf(fabsf(wk.x), ra, gg.x); gg.y = fmaf(fabsf(wk.y), ra, gg.y);
                  gg.z = fmaf(fabsf(wk.z), ra, gg.z); gg.w = fmaf(fabsf(wk.w), ra, gg.w);
                }
              }
            }
          }
          // group 1 hands its partial sums over (v, u, tmp, rpart, spart, Inew as staging)
          float* stg[7] = {s.tmp, s.Inew, s.Inew + w, s.Inew + 2 * w, s.rpart, s.v, s.u};
          const float4 mine[7] = {cc, i0, i1, i2, imp, ee, gg};
          if (mt < 2 * LG && grp == 1)
            for (int q = 0; q < 7; ++q) reinterpret_cast<float4*>(stg[q])[ln] = mine[q];
          math_sync();
          if (mt < LG) {
            float4 o[7];
            for (int q = 0; q < 7; ++q) {
              const float4 t = reinterpret_cast<const float4*>(stg[q])[ln];
              o[q] = make_float4(mine[q].x + t.x, mine[q].y + t.y, mine[q].z + t.z, mine[q].w + t.w);
            }
            const float4 bb = reinterpret_cast<const float4*>(args.b[j])[ln];
            const float bv[4] = {bb.x, bb.y, bb.z, bb.w};
            const float cv[4] = {o[0].x, o[0].y, o[0].z, o[0].w};
            const float v0[4] = {o[1].x, o[1].y, o[1].z, o[1].w}, v1[4] = {o[2].x, o[2].y, o[2].z, o[2].w},
                        v2[4] = {o[3].x, o[3].y, o[3].z, o[3].w}, im[4] = {o[4].x, o[4].y, o[4].z, o[4].w},
                        ev[4] = {o[5].x, o[5].y, o[5].z, o[5].w}, gv[4] = {o[6].x, o[6].y, o[6].z, o[6].w};
            for (int e4 = 0; e4 < 4; ++e4) {
              const int nn = 4 * ln + e4;
              s.tmp[nn] = cv[e4] + bv[e4];
              s.Inew[nn] = v0[e4];
              s.Inew[w + nn] = v1[e4];
              s.Inew[2 * w + nn] = v2[e4];
              s.rpart[nn] = im[e4] + (clt ? v0[e4] * v0[e4] + v1[e4] * v1[e4] + v2[e4] * v2[e4]
                                          : fabsf(v0[e4]) + fabsf(v1[e4]) + fabsf(v2[e4]));
              s.spart[nn] = infl ? (kap * gv[e4] + gamma_k(w + 2, kLinU) * (ev[e4] + fabsf(bv[e4]))) * kLinSafe : 0.0f;
            }
          }
        }
        // ---- the G rows' reductions from the epilogue ----
        if (mt == 0) trace(args, 0, cell / gridDim.x, 3 + 4 * (j - 1));
        if (j >= 2) {
          if (!group_wait(&s.bar[BAR_RED], red_n & 1)) { ok = false; break; }
          ++red_n;
        } else {
          math_sync();
        }
        if (mt == 0) trace(args, 0, cell / gridDim.x, 4 + 4 * (j - 1));
        const bool stored = (j >= 2) && (j < H - 1);
        for (int nn = mt; nn < w; nn += kMathThreads) {
          float tc = 0.f;
          if (j >= 2) tc = s.red[nn] + s.red[w + nn] + s.red[2 * w + nn] + s.red[3 * w + nn];
          float tot = s.rpart[nn] + tc;
          s.rprev[nn] = s.r[nn];
          s.r[nn] = clt ? sqrtf(tot) : tot;
          s.delta[nn] = infl ? s.spart[nn] + (stored ? kUb / (1.0f - kUb) * tc * kLinSafe : 0.f) : 0.f;
          s.c[nn] = s.tmp[nn];
          s.I[nn] = s.Inew[nn];
          s.I[w + nn] = s.Inew[w + nn];
          s.I[2 * w + nn] = s.Inew[2 * w + nn];
        }
        math_sync();
        if (mt == 0) trace(args, 0, cell / gridDim.x, 5 + 4 * (j - 1));
      }
      if (!ok) break;
      // ---- ReLU H, then the output layer (through layer H-1 for the G rows) ----
      float* al = s.alpha + (H % 3) * w;
      float* ga = s.gamma + (H % 3) * w;
      for (int nn = mt; nn < w; nn += kMathThreads) {
        Lin L = clt ? relu_clt(s.c[nn], s.r[nn]) : relu_sound(s.c[nn], s.r[nn], s.delta[nn], infl);
        al[nn] = L.alpha;
        ga[nn] = L.gamma;
        s.a[nn] = L.center;
      }
      math_sync();
      const float* wout = args.W[H];
      if (mt == 0) trace(args, 0, cell / gridDim.x, 40);
      const float* WHm1 = args.W[H - 1];                 // row-major [n][k]
      const float* alm1 = s.alpha + ((H - 1) % 3) * w;
      // v = W_{H-1}^T (alpha_H * w_out), |v|abs, u = alpha_{H-1} * v  (4 k per thread, n split in halves)
      {
        const int LG = w / 4, grp = mt / LG, ln = mt % LG, nh = w / 2;
        float4 vv = make_float4(0.f, 0.f, 0.f, 0.f), va = vv;
        if (mt < 2 * LG) {
          const float4* Wp = reinterpret_cast<const float4*>(WHm1) + ln;
#pragma unroll 8
          for (int nn = grp * nh; nn < grp * nh + nh; ++nn) {
            const float4 wv = __ldg(Wp + (size_t)nn * LG);
            const float aw = al[nn] * wout[nn], awa = fabsf(aw);
            vv.x = fmaf(wv.x, aw, vv.x); vv.y = fmaf(wv.y, aw, vv.y); vv.z = fmaf(wv.z, aw, vv.z); vv.w = fmaf(wv.w, aw, vv.w);
            va.x = fmaf(fabsf(wv.x), awa, va.x); va.y = fmaf(fabsf(wv.y), awa, va.y);
            va.z = fmaf(fabsf(wv.z), awa, va.z); va.w = fmaf(fabsf(wv.w), awa, va.w);
          }
          if (grp == 1) {
            reinterpret_cast<float4*>(s.v)[ln] = vv;
            reinterpret_cast<float4*>(s.tmp)[ln] = va;
          }
        }
        math_sync();
        if (mt < LG) {
          const float4 t1 = reinterpret_cast<const float4*>(s.v)[ln], t2 = reinterpret_cast<const float4*>(s.tmp)[ln];
          const float x[4] = {vv.x + t1.x, vv.y + t1.y, vv.z + t1.z, vv.w + t1.w};
          const float y[4] = {va.x + t2.x, va.y + t2.y, va.z + t2.z, va.w + t2.w};
          for (int e4 = 0; e4 < 4; ++e4) {
            const int k = 4 * ln + e4;
            s.v[k] = x[e4];
            s.tmp[k] = y[e4];
            s.u[k] = alm1[k] * x[e4];
          }
        }
      }
      math_sync();
      const int TO = out_tiles(H, w);
      if (TO > 0) {
        // Bout row 0 = bf16(u) in the 128-byte-swizzled K-major layout (row 0 is not permuted)
        for (int k = mt; k < w; k += kMathThreads) {
          const int c = k / 64, unit = (k % 64) / 8;
          __nv_bfloat16* p = reinterpret_cast<__nv_bfloat16*>(s.Bout + (size_t)c * 16 * 128 + unit * 16) + (k % 8);
          *p = __float2bfloat16_rn(s.u[k]);
        }
        fence_async_shared();
        math_sync();
        if (mt == 0) mbar_arrive(&s.bar[BAR_BOUTREADY]);
      }
      // implicit G_{H-2} at z_{H-1} (through u): y_m = gamma_{H-2,m} sum_n W_{H-2}[n][m] u_n
      if (H >= 3) {
        const int LG = w / 4, grp = mt / LG, ln = mt % LG, nh = w / 2;
        float4 dd = make_float4(0.f, 0.f, 0.f, 0.f);
        if (mt < 2 * LG) {
          const float4* Wp = reinterpret_cast<const float4*>(args.W[H - 2]) + ln;
#pragma unroll 8
          for (int nn = grp * nh; nn < grp * nh + nh; ++nn) {
            const float4 wv = __ldg(Wp + (size_t)nn * LG);
            const float un = s.u[nn];
            dd.x = fmaf(wv.x, un, dd.x); dd.y = fmaf(wv.y, un, dd.y); dd.z = fmaf(wv.z, un, dd.z); dd.w = fmaf(wv.w, un, dd.w);
          }
          if (grp == 1) reinterpret_cast<float4*>(s.rpart)[ln] = dd;
        }
        math_sync();
        if (mt < LG) {
          const float4 t = reinterpret_cast<const float4*>(s.rpart)[ln];
          s.spart[4 * ln] = dd.x + t.x;
          s.spart[4 * ln + 1] = dd.y + t.y;
          s.spart[4 * ln + 2] = dd.z + t.z;
          s.spart[4 * ln + 3] = dd.w + t.w;
        }
        math_sync();
      }
      // CUDA-core rows: G_{H-2} at z_{H-1} (above), G_{H-1} at z_H (v), fresh G_H, and the I rows of
      // z_H (through alpha_H * w_out)
      float acc = 0.f, eabs = 0.f, x0p = 0.f, cen = 0.f;
      const float* gam1 = s.gamma + ((H - 1) % 3) * w;
      for (int m = mt; m < w; m += kMathThreads) {
        if (H >= 3) {
          const float* gam2 = s.gamma + ((H - 2) % 3) * w;
          const float y = gam2[m] * s.spart[m];
          acc += sq ? y * y : fabsf(y);
        }
        const float y1 = gam1[m] * s.v[m];
        const float y2 = ga[m] * wout[m];
        acc += sq ? y1 * y1 + y2 * y2 : fabsf(y1) + fabsf(y2);
        x0p = fmaf(wout[m], s.a[m], x0p);
        if (infl) {
          eabs += s.rprev[m] * alm1[m] * s.tmp[m] + gam1[m] * s.tmp[m] + (s.r[m] * al[m] + ga[m]) * fabsf(wout[m]);
          cen = fmaf(fabsf(wout[m]), fabsf(s.a[m]), cen);
        }
      }
      if (mt < 3) {
        float y = 0.f;
        for (int k = 0; k < w; ++k) y = fmaf(s.I[mt * w + k], al[k] * wout[k], y);
        acc += sq ? y * y : fabsf(y);
      }
      float vals[4] = {acc, eabs, x0p, cen};
      for (int qv = 0; qv < 4; ++qv) {
        float x = vals[qv];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) s.scal[qv * 4 + (mt >> 5)] = x;
      }
      if (mt == 0) trace(args, 0, cell / gridDim.x, 41);
      if (TO > 0) {
        if (!group_wait(&s.bar[BAR_RED], red_n & 1)) break;
        ++red_n;
      } else {
        math_sync();
      }
      if (mt == 0) trace(args, 0, cell / gridDim.x, 42);
      if (mt == 0) {
        float tot = 0.f, ea = 0.f, xp = 0.f, ce = 0.f;
        for (int i = 0; i < 4; ++i) {
          tot += s.scal[i];
          ea += s.scal[4 + i];
          xp += s.scal[8 + i];
          ce += s.scal[12 + i];
        }
        if (TO > 0) tot += s.red[0] + s.red[w] + s.red[2 * w] + s.red[3 * w];
        const float x0 = xp + args.bout;
        float sp;
        if (mode == ISX_BOUND_SOUND) {
          sp = tot;
          if (infl)
            sp = __fadd_ru(__fmul_ru(sp, kLinSafe),
                           (args.kappa_out * ea + gamma_k(w + 2, kLinU) * (ce + fabsf(args.bout))) * 1.01f);
        } else if (mode == ISX_BOUND_CLT) {
          sp = sqrtf(tot);
        } else {
          sp = sqrtf(tot / 3.0f);
        }
        args.center[cell] = x0;
        args.spread[cell] = sp;
      }
      math_sync();
    }
  }

  // ---- teardown: let in-flight copies land, free TMEM ----
  __syncthreads();
  if (*(volatile int*)s.abort) {
    for (int i = 0; i < 1000; ++i) __nanosleep(1000);
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// ---- host side ---------------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

isx_status make_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint32_t box_inner,
                    uint32_t box_outer) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available");
    return ISX_ERR_CUDA;
  }
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
    return ISX_ERR_CUDA;
  }
  return ISX_OK;
}

}  // namespace

isx_status tensor_map_bf16(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint32_t box_inner,
                           uint32_t box_outer) {
  return make_map(m, base, inner, outer, box_inner, box_outer);
}

bool bf16_supported(isx_inr inr) { return (inr->w == 128 || inr->w == 256) && inr->H >= 2 && inr->H <= 12; }

isx_status bound_bf16(isx_inr inr, const CellSource& src, int64_t n, isx_bound_mode mode, int inflate,
                      float* d_center, float* d_spread, cudaStream_t st) {
  if (!bf16_supported(inr)) {
    set_error("BF16 tensor-core propagation supports hidden widths 128 and 256");
    return ISX_ERR_UNSUPPORTED;
  }
  if (n <= 0) return ISX_OK;
  // ISX_CLT_COV=1 selects the covariance (Gram-matrix) propagation of bound_cov.cu for CLT: faster,
  // but its bf16 rounding error grows with the square of the output-layer cancellation ratio, so
  // the coefficient propagation below stays the default
  if (mode == ISX_BOUND_CLT && std::getenv("ISX_CLT_COV") != nullptr)
    return bound_bf16_clt_cov(inr, src, n, d_center, d_spread, st);
  const int w = inr->w, H = inr->H;
  int dev = inr->device, sms = 0;
  ISX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = (int)std::min<int64_t>(n, sms);
  const int rows = std::max(1, w * std::max(0, H - 3));
  auto& ws = inr->ws;
  ISX_TRY(ws[WS_TC_SCRATCH].ensure((size_t)sms * rows * w * 2, "tc scratch"));
  ISX_TRY(ws[WS_TC_STATUS].ensure(64, "tc status"));
  TcArgs a{};
  a.src = src;
  a.n = n;
  a.mode = (int)mode;
  a.inflate = (mode == ISX_BOUND_SOUND) ? inflate : 0;
  a.w = w;
  a.H = H;
  for (int l = 0; l < inr->n_layers; ++l) {
    a.W[l] = inr->W[l];
    a.Wt[l] = inr->Wt[l];
    a.b[l] = inr->b[l];
  }
  a.bout = inr->hb[inr->n_layers - 1][0];
  a.scratch = ws[WS_TC_SCRATCH].as<__nv_bfloat16>();
  a.rows_per_cta = rows;
  a.center = d_center;
  a.spread = d_spread;
  a.status = ws[WS_TC_STATUS].as<int>();
  const float ub = kUb, ua = kUa, u = kLinU;
  const float gK = (w * ua) / (1.0f - w * ua), gK32 = (w * u) / (1.0f - w * u);
  a.kappa = (1 + ub) * (1 + ub) * (1 + ub) * (1 + gK) * (1 + u) - 1;
  a.kappa_out = (1 + ub) * (1 + gK) * (1 + gK32) * (1 + gK32) * (1 + u) * (1 + u) - 1;
  TcMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  ISX_TRY(make_map(&maps.scratch, a.scratch, w, (uint64_t)sms * rows, 64, 128));
  for (int l = 1; l < inr->n_layers - 1; ++l) {
    ISX_TRY(make_map(&maps.wt[l], inr->Wt_bf16[l], w, w, 64, 128));
    ISX_TRY(make_map(&maps.wrow[l], inr->W_bf16[l], w, w, 64, w));
  }
  ISX_CUDA(cudaMemsetAsync(a.status, 0, sizeof(int), st));
  const bool tracing = std::getenv("ISX_TRACE") != nullptr;
  a.trace = nullptr;
  if (tracing) {
    ISX_TRY(ws[WS_AUX].ensure(3 * kTraceCells * kTraceEvents * sizeof(long long), "trace"));
    a.trace = ws[WS_AUX].as<long long>();
    ISX_CUDA(cudaMemsetAsync(a.trace, 0, 3 * kTraceCells * kTraceEvents * sizeof(long long), st));
  }
  const size_t smem = smem_bytes(w);
  ISX_CUDA(cudaFuncSetAttribute(k_bound_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  {
    const double cells = (double)n;
    const double rows_gemm = (double)w * (H - 1) * (H - 2) / 2.0;   // G rows over layers 2..H-1
    prof::Scope ps(K_BOUND_TC, st, cells * 2.0 * w * w * (3.0 * (H - 1) + rows_gemm), 0);
    k_bound_tc<<<grid, kThreads, smem, st>>>(a, maps);
  }
  ISX_LAUNCH_CHECK("k_bound_tc");
  int status = 0;
  ISX_CUDA(cudaMemcpyAsync(&status, a.status, sizeof(int), cudaMemcpyDeviceToHost, st));
  ISX_CUDA(cudaStreamSynchronize(st));
  if (status != 0) {
    set_error("tensor-core bound kernel gave up waiting (bounded wait expired)");
    return (isx_status)status;
  }
  if (tracing) {
    std::vector<long long> h(3 * kTraceCells * kTraceEvents);
    ISX_CUDA(cudaMemcpy(h.data(), a.trace, h.size() * sizeof(long long), cudaMemcpyDeviceToHost));
    const long long t0 = h[0];
    for (int role = 0; role < 3; ++role)
      for (int c = 0; c < kTraceCells; ++c) {
        std::fprintf(stderr, "isx trace n=%lld role=%d cell=%d:", (long long)n, role, c);
        for (int e = 0; e < kTraceEvents; ++e) {
          long long v = h[(role * kTraceCells + c) * kTraceEvents + e];
          if (v) std::fprintf(stderr, " %d:%lld", e, v - t0);
        }
        std::fprintf(stderr, "\n");
      }
  }
  return ISX_OK;
}

}  // namespace isx

// ---- allocation-free variant ---------------------------------------------------------------------------
// isx_bound_cells_noalloc runs the same tensor-core kernel, but takes its per-CTA coefficient
// slices and its status word from a fixed array compiled into this file instead of the INR's
// workspace, so the call itself never allocates device memory.
namespace isx {
namespace {

constexpr size_t kStaticScratchBytes = 16ull << 20;   // 16 MiB, held by every device that loads the library
constexpr size_t kStaticStatusBytes = 256;            // status word, padded to keep the slices aligned
static __device__ __align__(256) uint8_t g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_addr[64] = {};

// Device address of g_static_scratch on the current device, looked up once per device.
isx_status static_scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (dev < 0 || dev >= 64) {
    set_error("device index out of range for the static scratch table");
    return ISX_ERR_ARG;
  }
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                                                 "cudaGetSymbolAddress(g_static_scratch)", __FILE__, __LINE__);
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return ISX_OK;
}

}  // namespace
}  // namespace isx

extern "C" isx_status isx_bound_cells_noalloc(isx_inr inr, const float* d_lo, const float* d_hi, int64_t n,
                                             isx_bound_mode mode, int inflate, float* d_center, float* d_spread,
                                             void* stream) {
  using namespace isx;
  if (!inr) {
    set_error("null INR handle");
    return ISX_ERR_ARG;
  }
  if (n < 0 || (n > 0 && (!d_lo || !d_hi || !d_center || !d_spread))) {
    set_error("bad size or null pointer");
    return ISX_ERR_ARG;
  }
  if (mode < ISX_BOUND_SOUND || mode > ISX_BOUND_RAUA) {
    set_error("bad mode");
    return ISX_ERR_ARG;
  }
  int dev = -1;
  ISX_CUDA(cudaGetDevice(&dev));
  if (dev != inr->device) {
    set_error("the INR was created on another device than the current one");
    return ISX_ERR_ARG;
  }
  if (!bf16_supported(inr)) {
    set_error("isx_bound_cells_noalloc supports the bf16 tensor-core path only (hidden width 128 or 256)");
    return ISX_ERR_UNSUPPORTED;
  }
  if (n == 0) return ISX_OK;
  const int w = inr->w, H = inr->H;
  const int rows = std::max(1, w * std::max(0, H - 3));
  const size_t per_cta = (((size_t)rows * w * 2) + 255) & ~size_t(255);
  if (per_cta > kStaticScratchBytes - kStaticStatusBytes) {
    set_error("isx_bound_cells_noalloc: this network needs " + std::to_string(per_cta) +
              " bytes of scratch per CTA, more than the 16 MiB static scratch array holds");
    return ISX_ERR_CAPACITY;
  }
  void* base = nullptr;
  ISX_TRY(static_scratch_address(dev, &base));
  int sms = 0;
  ISX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t fit = (int64_t)((kStaticScratchBytes - kStaticStatusBytes) / per_cta);
  const int grid = (int)std::min<int64_t>(std::min<int64_t>(n, sms), fit);
  cudaStream_t st = (cudaStream_t)stream;
  TcArgs a{};
  a.src.lo = d_lo;
  a.src.hi = d_hi;
  a.n = n;
  a.mode = (int)mode;
  a.inflate = (mode == ISX_BOUND_SOUND) ? inflate : 0;
  a.w = w;
  a.H = H;
  for (int l = 0; l < inr->n_layers; ++l) {
    a.W[l] = inr->W[l];
    a.Wt[l] = inr->Wt[l];
    a.b[l] = inr->b[l];
  }
  a.bout = inr->hb[inr->n_layers - 1][0];
  a.status = reinterpret_cast<int*>(base);
  a.scratch = reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<uint8_t*>(base) + kStaticStatusBytes);
  a.rows_per_cta = (int)(per_cta / (w * 2));
  a.center = d_center;
  a.spread = d_spread;
  a.trace = nullptr;
  const float ub = kUb, ua = kUa, u = kLinU;
  const float gK = (w * ua) / (1.0f - w * ua), gK32 = (w * u) / (1.0f - w * u);
  a.kappa = (1 + ub) * (1 + ub) * (1 + ub) * (1 + gK) * (1 + u) - 1;
  a.kappa_out = (1 + ub) * (1 + gK) * (1 + gK32) * (1 + gK32) * (1 + u) * (1 + u) - 1;
  TcMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  ISX_TRY(make_map(&maps.scratch, a.scratch, w, (uint64_t)grid * a.rows_per_cta, 64, 128));
  for (int l = 1; l < inr->n_layers - 1; ++l) {
    ISX_TRY(make_map(&maps.wt[l], inr->Wt_bf16[l], w, w, 64, 128));
    ISX_TRY(make_map(&maps.wrow[l], inr->W_bf16[l], w, w, 64, w));
  }
  // the status word must start at zero on every call; the slices need no clearing (every row is
  // written before it is read)
  ISX_CUDA(cudaMemsetAsync(a.status, 0, sizeof(int), st));
  const size_t smem = smem_bytes(w);
  ISX_CUDA(cudaFuncSetAttribute(k_bound_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  {
    const double rows_gemm = (double)w * (H - 1) * (H - 2) / 2.0;
    prof::Scope ps(K_BOUND_TC, st, (double)n * 2.0 * w * w * (3.0 * (H - 1) + rows_gemm), 0);
    k_bound_tc<<<grid, kThreads, smem, st>>>(a, maps);
  }
  ISX_LAUNCH_CHECK("k_bound_tc (static scratch)");
  int status = 0;
  ISX_CUDA(cudaMemcpyAsync(&status, a.status, sizeof(int), cudaMemcpyDeviceToHost, st));
  ISX_CUDA(cudaStreamSynchronize(st));
  if (status != 0) {
    set_error("tensor-core bound kernel gave up waiting (bounded wait expired)");
    return (isx_status)status;
  }
  return ISX_OK;
}
