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
#include <type_traits>
#include <vector>

namespace isx {
namespace {

constexpr int kStages = 3;
constexpr int kEpiWarps = 8;
constexpr int kMathWarps = 4;
constexpr int kRingWarp = 2 + kEpiWarps + kMathWarps;              // 14: producer of the math ring
constexpr int kThreads = 32 * (kRingWarp + 1);                     // 480
constexpr int kMathThreads = 32 * kMathWarps;
constexpr int kMathBase = 32 * (2 + kEpiWarps);                    // first math thread
constexpr uint32_t kStageBytes = 128 * 128;                        // 128 rows x 64 bf16
constexpr uint32_t kRingBytes = 8192;                              // one stage of float32 weight rows
constexpr int kRingStages = 2;
constexpr int kBigStages = 4;                                      // the B buffer as a ring while B is idle
constexpr uint64_t kWaitNs = 2000000000ull;                        // 2 s per wait
constexpr float kUb = 0.00390625f;                                 // 2^-8
constexpr float kUa = 7.62939453125e-06f;                          // 2^-17
constexpr float kGemvSafe = 1.015625f;                             // 1 + 2^-6: bf16 GEMV results bounded above

// One network of a launch: its weights and the tensor maps of its BF16 copies (device memory,
// 64-byte aligned; written by the host before the launch).
struct TcNet {
  CUtensorMap wt[ISX_MAX_LAYERS];      // W_l^T bf16, box {64, 128}: A of implicit blocks
  CUtensorMap wrow[ISX_MAX_LAYERS];    // W_l bf16, box {64, w}: source of B = D W^T
  CUtensorMap wabs[ISX_MAX_LAYERS];    // |W_l| bf16, box {64, 128}: A of the sound reduction pass
  CUtensorMap wsq[ISX_MAX_LAYERS];     // W_l^2 bf16, box {64, 128}: A of the CLT reduction pass
  const float* W[ISX_MAX_LAYERS];
  const float* Wt[ISX_MAX_LAYERS];
  const float* b[ISX_MAX_LAYERS];
  float bout;
  int H;
  int w;                               // cells of networks of another width are skipped
  int act;                             // isx_activation of the hidden layers (CLT rule)
};

struct TcArgs {
  CellSource src;
  int64_t n;
  int mode, inflate, w;
  const TcNet* nets;                   // device descriptor of the network
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
};

// ---- shared-memory layout ------------------------------------------------------------------------------
struct Smem {
  uint8_t* B;        // w/64 chunks of [w rows][128 B]: D_j W_j^T
  uint8_t* A;        // kStages x 16 KB
  uint8_t* Bs;       // w/64 chunks of [16 rows][128 B]: small B (GEMV columns, then u)
  float* ring;       // kRingStages x 8 KB of float32 weight rows
  float* alpha;      // [3][w] (slot = layer % 3)
  float* gamma;      // [3][w]
  float* c;          // centre of the current z
  float* r;          // radius / sigma of the current z (all rows)
  float* delta;      // slack of the current z
  float* a;          // a-form centre
  float* rada;       // a-form radius (sound)
  float* rprev;      // radius of the previous z
  float* red;        // [4][w] epilogue partial reductions
  float* I;          // [3][w] input-symbol rows of the current z
  float* Inew;       // [3][w] next layer's I rows (small pass 1), later G_{H-2} output values
  float* imp;        // implicit-block reduction (small pass 2); output: v
  float* ig;         // sum |W| rad_a (small pass 2); output: u
  float* ie;         // sum |W| |a| (small pass 2); output: |v|abs
  float* scal;       // [64] block-reduction scratch
  uint64_t* bar;
  uint32_t* tmem_slot;
  int* abort;
};

enum Bars {
  BAR_FULL = 0, BAR_EMPTY = kStages, BAR_TFULL = 2 * kStages, BAR_TEMPTY = 2 * kStages + 2,
  BAR_BREADY = 2 * kStages + 4, BAR_BFREE, BAR_WLOADED, BAR_RED, BAR_BOUTREADY,
  BAR_MFULL, BAR_MEMPTY = BAR_MFULL + kRingStages, BAR_BMFULL = BAR_MEMPTY + kRingStages,
  BAR_BMEMPTY = BAR_BMFULL + kBigStages, BAR_RINGBFREE = BAR_BMEMPTY + kBigStages, BAR_COUNT
};

__host__ __device__ inline size_t smem_bytes(int w) {
  size_t off = 0;
  off += (size_t)w * w * 2;                       // B
  off += (size_t)kStages * kStageBytes;           // A
  off += (size_t)16 * w * 2;                      // Bs
  off += (size_t)kRingStages * kRingBytes;        // ring
  off += (size_t)(25 * w + 64) * 4;               // floats
  off += BAR_COUNT * 8 + 16;
  return off + 1024;                              // alignment slack (carve aligns the base to 1024)
}

__device__ Smem carve(uint8_t* raw, int w) {
  const uintptr_t base = ((uintptr_t)raw + 1023) & ~(uintptr_t)1023;   // swizzled operands need 1024-byte alignment
  uint8_t* p = (uint8_t*)base;
  Smem s;
  s.B = p; p += (size_t)w * w * 2;
  s.A = p; p += (size_t)kStages * kStageBytes;
  s.Bs = p; p += (size_t)16 * w * 2;
  s.ring = (float*)p; p += (size_t)kRingStages * kRingBytes;
  float* f = (float*)p;
  s.alpha = f; f += 3 * w;
  s.gamma = f; f += 3 * w;
  s.c = f; f += w;
  s.r = f; f += w;
  s.delta = f; f += w;
  s.a = f; f += w;
  s.rada = f; f += w;
  s.rprev = f; f += w;
  s.red = f; f += 4 * w;
  s.I = f; f += 3 * w;
  s.Inew = f; f += 3 * w;
  s.imp = f; f += w;
  s.ig = f; f += w;
  s.ie = f; f += w;
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

// TC layers are j = 2 .. H-1; layer j has (j - 1) blocks of w rows.
__device__ __forceinline__ int out_tiles(int H, int w) { return H >= 4 ? (H - 3) * (w / 128) : 0; }

// Element (row, k) of a K-major, 128-byte-swizzled operand of `rows` rows: byte offset.
__device__ __forceinline__ uint32_t swz(int rows, int row, int k) {
  return (uint32_t)((k >> 6) * rows * 128 + row * 128 + ((((k & 63) >> 3) ^ (row & 7)) << 4) + (k & 7) * 2);
}

// One weight matrix streamed through the math ring (rows k in the bulk producer's order):
// acc[v][e] += sum_k row_k[col_e] * x_v[k] for col_e = mt + e * 128 and NX vectors x_v, where
// x_0 = x and, with NX == 4, x_{1..3}[k] = I[r][k] * al[k] (the input-symbol rows times alpha);
// with `with_abs`, aacc[e] += sum_k |row_k[col_e]| |x[k]|.
// Two rings carry the rows: the small one (kRingStages x 8 KB) and, while B is idle (the first
// layer's GEMV and the output GEMVs), the B buffer itself (kBigStages stages of W W / 2 bytes).
struct Ring {
  const float* base;
  int stage_floats, nstages, full, empty;
};
template <int W, bool BIG>
__device__ __forceinline__ Ring ring_of(const Smem& s) {
  if constexpr (BIG) return Ring{reinterpret_cast<const float*>(s.B), W * W / 8, kBigStages, BAR_BMFULL, BAR_BMEMPTY};
  else return Ring{s.ring, (int)(kRingBytes / 4), kRingStages, BAR_MFULL, BAR_MEMPTY};
}

template <int W, int NX, int NPT, bool BIG>
__device__ __forceinline__ bool ring_gemv(const Smem& s, int* status, uint32_t& ms, uint32_t& mph, int mt, int lane,
                                          const float* x, const float* al, float (&acc)[NX][NPT], float (&aacc)[NPT],
                                          bool with_abs) {
  const Ring rg = ring_of<W, BIG>(s);
  constexpr int R = BIG ? W / 8 : (int)(kRingBytes / (4 * W));   // rows per stage
  for (int r0 = 0; r0 < W; r0 += R) {
    if (!wait_bar(s, &s.bar[rg.full + ms], mph, status)) return false;
    const float* rows = rg.base + (size_t)ms * rg.stage_floats;
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      const int k = r0 + rr;
      float xv[NX];
      xv[0] = x[k];
      if constexpr (NX == 4) {
        const float ak = al[k];
        xv[1] = s.I[k] * ak;
        xv[2] = s.I[W + k] * ak;
        xv[3] = s.I[2 * W + k] * ak;
      }
#pragma unroll
      for (int e = 0; e < NPT; ++e) {
        const float wv = rows[rr * W + mt + e * kMathThreads];
#pragma unroll
        for (int vq = 0; vq < NX; ++vq) acc[vq][e] = fmaf(wv, xv[vq], acc[vq][e]);
        if (with_abs) aacc[e] = fmaf(fabsf(wv), fabsf(xv[0]), aacc[e]);
      }
    }
    // The stage is refilled by the bulk copy engine (async proxy) once every math warp has
    // released it; the proxy fence orders this thread's generic reads of the stage before that
    // write.  Without it, reads still queued behind heavy global-store traffic (the epilogue
    // writing stored G rows) were observed to return the next stage's rows.
    fence_async_shared();
    __syncwarp();
    if (lane == 0) mbar_arrive(&s.bar[rg.empty + ms]);
    if (++ms == (uint32_t)rg.nstages) { ms = 0; mph ^= 1; }
  }
  return true;
}

// B = D_j W_j^T in place, by the math warps: every thread owns one logical 8-column K chunk (its 8
// alphas stay in registers) and walks W / 4 / (4 / KC) rows of it; the 8 lanes that share a row cover
// its whole swizzled 128-byte row, so each warp access touches 4 rows x 128 contiguous bytes.
template <int W>
__device__ __forceinline__ void scale_b_rows(const Smem& s, const float* al, int mt) {
  constexpr int KC = W / 64, WPC = 4 / KC, ROWS = W / WPC;   // warps per K chunk, rows per warp
  const int mw = mt >> 5, l = mt & 31;
  const int c = mw % KC, part = mw / KC, L = l & 7, roff = l >> 3;
  const int k0 = c * 64 + 8 * L;
  const float4 a0 = *reinterpret_cast<const float4*>(al + k0);
  const float4 a1 = *reinterpret_cast<const float4*>(al + k0 + 4);
  uint8_t* base = s.B + (size_t)c * W * 128;
#pragma unroll 4
  for (int i = 0; i < ROWS / 4; ++i) {
    const int n = part * ROWS + roff + 4 * i;
    uint4* pu = reinterpret_cast<uint4*>(base + (size_t)n * 128 + ((L ^ (n & 7)) << 4));
    uint4 v = *pu;
    __nv_bfloat162* hv = reinterpret_cast<__nv_bfloat162*>(&v);
    const float2 f0 = __bfloat1622float2(hv[0]), f1 = __bfloat1622float2(hv[1]);
    const float2 f2 = __bfloat1622float2(hv[2]), f3 = __bfloat1622float2(hv[3]);
    hv[0] = __floats2bfloat162_rn(f0.x * a0.x, f0.y * a0.y);
    hv[1] = __floats2bfloat162_rn(f1.x * a0.z, f1.y * a0.w);
    hv[2] = __floats2bfloat162_rn(f2.x * a1.x, f2.y * a1.y);
    hv[3] = __floats2bfloat162_rn(f3.x * a1.z, f3.y * a1.w);
    *pu = v;
  }
}

// ---- the kernel ------------------------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kThreads, 1) k_bound_tc(const __grid_constant__ TcArgs args,
                                                           const __grid_constant__ TcMaps maps) {
  extern __shared__ uint8_t smem_raw[];
  constexpr int MT = W / 128;              // 128-row tiles per block of w rows
  constexpr int KC = W / 64;               // 64-wide K chunks
  const int64_t ncell = args.n;
  Smem s = carve(smem_raw, W);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
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
    for (int i = 0; i < kRingStages; ++i) {
      mbar_init(&s.bar[BAR_MFULL + i], 1);
      mbar_init(&s.bar[BAR_MEMPTY + i], kMathWarps);
    }
    for (int i = 0; i < kBigStages; ++i) {
      mbar_init(&s.bar[BAR_BMFULL + i], 1);
      mbar_init(&s.bar[BAR_BMEMPTY + i], kMathWarps);
    }
    mbar_init(&s.bar[BAR_RINGBFREE], 1);
    mbar_init(&s.bar[BAR_BREADY], 1);
    mbar_init(&s.bar[BAR_BFREE], 1);
    mbar_init(&s.bar[BAR_WLOADED], 1);
    mbar_init(&s.bar[BAR_RED], kEpiWarps);
    mbar_init(&s.bar[BAR_BOUTREADY], 1);
    *s.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = threadIdx.x; i < 16 * W * 2 / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(s.Bs)[i] = make_uint4(0, 0, 0, 0);
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
  __nv_bfloat16* scratch = args.scratch + (size_t)blockIdx.x * args.rows_per_cta * W;

  if (warp == 0) {
    // ============================ TMA producer: B source and A tiles ============================
    if (lane == 0) {
      uint32_t stage = 0, sphase = 0, bfree_n = 0, red_n = 0, rb_n = 0;
      bool ok = true;
      auto load_a = [&](const CUtensorMap* m, int x, int y) -> bool {
        if (!wait_bar(s, &s.bar[BAR_EMPTY + stage], sphase ^ 1, args.status)) return false;
        mbar_expect_tx(&s.bar[BAR_FULL + stage], kStageBytes);
        tma_load_2d(s.A + (size_t)stage * kStageBytes, m, &s.bar[BAR_FULL + stage], x, y);
        if (++stage == kStages) { stage = 0; sphase ^= 1; }
        return true;
      };
      // a 128-row tile of this CTA's stored rows (unit-major scratch), K chunk c: lands in the
      // stage as 8 x [128 rows x 16 bytes] core-matrix columns (no swizzle)
      auto load_s = [&](int row, int c) -> bool {
        if (!wait_bar(s, &s.bar[BAR_EMPTY + stage], sphase ^ 1, args.status)) return false;
        mbar_expect_tx(&s.bar[BAR_FULL + stage], kStageBytes);
        tma_load_3d(s.A + (size_t)stage * kStageBytes, &maps.scratch, &s.bar[BAR_FULL + stage], 0, row,
                    (int)blockIdx.x * (W / 8) + c * 8);
        if (++stage == kStages) { stage = 0; sphase ^= 1; }
        return true;
      };
      for (int64_t cell = blockIdx.x; cell < ncell && ok; cell += gridDim.x) {
        const TcNet& N = args.nets[0];
        const int H = N.H;
        if (N.w != W) continue;
        for (int j = 1; j <= H - 1 && ok; ++j) {
          if (j >= 2) {
            // B source: W_j once the previous layer's MMAs no longer read B, and (for W_2) once the
            // math warps' first-layer GEMV no longer reads B as its ring
            if (!wait_bar(s, &s.bar[BAR_BFREE], (bfree_n & 1) ^ 1, args.status)) { ok = false; break; }
            ++bfree_n;
            if (j == 2 && !wait_bar(s, &s.bar[BAR_RINGBFREE], rb_n & 1, args.status)) { ok = false; break; }
            mbar_expect_tx(&s.bar[BAR_WLOADED], (uint32_t)(W * W * 2));
            for (int c = 0; c < KC; ++c) tma_load_2d(s.B + (size_t)c * W * 128, &N.wrow[j], &s.bar[BAR_WLOADED], c * 64, 0);
            // the previous layer is complete (its stored rows are read below); the proxy fence
            // orders the epilogue's generic stores, acquired through RED, before this thread's TMA reads
            if (!wait_bar(s, &s.bar[BAR_RED], red_n & 1, args.status)) { ok = false; break; }
            ++red_n;
            fence_async_global();
          }
          // reduction pass: A = |W_j| (sound) or W_j^2 (CLT) against the small B columns
          {
            const CUtensorMap* m = clt ? &N.wsq[j] : &N.wabs[j];
            for (int mt = 0; mt < MT && ok; ++mt)
              for (int c = 0; c < KC; ++c)
                if (!load_a(m, c * 64, mt * 128)) { ok = false; break; }
          }
          if (j >= 2) {
            const int T = (j - 1) * MT;
            for (int t = 0; t < T && ok; ++t) {
              const int blk = t / MT + 1, sub = t % MT;      // G_blk
              const bool implicit = (blk == j - 1);
              for (int c = 0; c < KC; ++c) {
                bool good = implicit ? load_a(&N.wt[j - 1], c * 64, sub * 128)
                                     : load_s((blk - 1) * W + sub * 128, c);
                if (!good) { ok = false; break; }
              }
            }
          }
        }
        if (!ok) break;
        ++rb_n;                           // the math warps release B once per cell (after GEMV 1)
        if (!wait_bar(s, &s.bar[BAR_RED], red_n & 1, args.status)) break;   // layer H-1
        ++red_n;
        fence_async_global();
        const int TO = out_tiles(H, W);
        for (int t = 0; t < TO && ok; ++t)
          for (int c = 0; c < KC; ++c)
            if (!load_s(t * 128, c)) { ok = false; break; }
        if (ok && TO > 0) {
          if (!wait_bar(s, &s.bar[BAR_RED], red_n & 1, args.status)) break;
          ++red_n;
        }
      }
    }
  } else if (warp == kRingWarp) {
    // ============================ bulk producer: float32 weight rows for the math warps ============================
    if (lane == 0) {
      uint32_t ms = 0, mph = 0, bms = 0, bmph = 0;
      uint64_t bfree_total = 0;           // B releases (one per layer >= 2) of the cells so far
      bool ok = true;
      auto push = [&](const float* src, bool big) -> bool {
        const int stage_bytes = big ? W * W / 2 : (int)kRingBytes, rows = stage_bytes / (4 * W);
        const int nst = big ? kBigStages : kRingStages, full = big ? BAR_BMFULL : BAR_MFULL,
                  empty = big ? BAR_BMEMPTY : BAR_MEMPTY;
        float* base = big ? reinterpret_cast<float*>(s.B) : s.ring;
        uint32_t& st = big ? bms : ms;
        uint32_t& ph = big ? bmph : mph;
        for (int r0 = 0; r0 < W; r0 += rows) {
          if (!wait_bar(s, &s.bar[empty + st], ph ^ 1, args.status)) return false;
          mbar_expect_tx(&s.bar[full + st], (uint32_t)stage_bytes);
          bulk_load(base + (size_t)st * (stage_bytes / 4), src + (size_t)r0 * W, (uint32_t)stage_bytes, &s.bar[full + st]);
          if (++st == (uint32_t)nst) { st = 0; ph ^= 1; }
        }
        return true;
      };
      for (int64_t cell = blockIdx.x; cell < ncell && ok; cell += gridDim.x) {
        const TcNet& N = args.nets[0];
        const int H = N.H;
        if (N.w != W) continue;
        // layer 1: B is idle (the previous cell's MMAs released it, this cell's W_2 waits for this GEMV)
        ok = push(N.Wt[1], true);                                        // centre of z_2
        for (int j = 2; j <= H - 1 && ok; ++j) ok = push(N.Wt[j], false); // centre of z_{j+1}
        if (!ok) break;
        if (H >= 3) {
          // the output GEMVs reuse B once the last layer's MMAs have released it
          bfree_total += (uint64_t)(H - 2);
          if (!wait_bar(s, &s.bar[BAR_BFREE], (uint32_t)((bfree_total - 1) & 1), args.status)) break;
        }
        ok = push(N.W[H - 1], true);                                     // v
        if (ok && H >= 3) ok = push(N.W[H - 2], true);                   // implicit G_{H-2}
      }
    }
  } else if (warp == 1) {
    // ============================ MMA issuer ============================
    if (lane == 0) {
      uint32_t stage = 0, sphase = 0, bready_n = 0, bout_n = 0, tiles_done = 0;
      const uint32_t id_main = idesc(W), id_small = idesc(16);
      bool ok = true;
      // one 128-row tile: K chunks from the A ring against B (bsmem, rows of the B operand)
      auto tile = [&](uint8_t* bsm, int brows, uint32_t id, bool a_noswz) -> bool {
        const uint32_t acc = tiles_done & 1;
        if (!wait_bar(s, &s.bar[BAR_TEMPTY + acc], ((tiles_done >> 1) & 1) ^ 1, args.status)) return false;
        tc_fence_after();
        const uint32_t d = tmem + acc * 256;
        for (int c = 0; c < KC; ++c) {
          if (!wait_bar(s, &s.bar[BAR_FULL + stage], sphase, args.status)) return false;
          tc_fence_after();
          const uint32_t a0 = su32(s.A + (size_t)stage * kStageBytes);
          const uint32_t b0 = su32(bsm + (size_t)c * brows * 128);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            // A: 128-byte swizzled rows (weight tiles) or unit-major core matrices (stored rows:
            // 16 K-elements = 2 core-matrix columns of 128 x 16 bytes)
            const uint64_t ad = a_noswz ? sdesc_noswz(a0 + kk * 2 * 2048, 2048, 128) : sdesc(a0 + kk * 32);
            mma_bf16(d, ad, sdesc(b0 + kk * 32), id, (c > 0 || kk > 0) ? 1u : 0u);
          }
          mma_commit(&s.bar[BAR_EMPTY + stage]);
          if (++stage == kStages) { stage = 0; sphase ^= 1; }
        }
        mma_commit(&s.bar[BAR_TFULL + acc]);
        ++tiles_done;
        return true;
      };
      for (int64_t cell = blockIdx.x; cell < ncell && ok; cell += gridDim.x) {
        const TcNet& N = args.nets[0];
        const int H = N.H;
        if (N.w != W) continue;
        for (int j = 1; j <= H - 1 && ok; ++j) {
          if (!wait_bar(s, &s.bar[BAR_BREADY], bready_n & 1, args.status)) { ok = false; break; }
          ++bready_n;
          trace(args, 1, cell / gridDim.x, 2 * j);
          tc_fence_after();
          for (int t = 0; t < MT && ok; ++t) ok = tile(s.Bs, 16, id_small, false);
          if (j >= 2) {
            const int T = (j - 1) * MT;
            for (int t = 0; t < T && ok; ++t) ok = tile(s.B, W, id_main, t / MT + 1 != j - 1);
            if (ok) mma_commit(&s.bar[BAR_BFREE]);
          }
          trace(args, 1, cell / gridDim.x, 2 * j + 1);
        }
        if (!ok) break;
        const int TO = out_tiles(H, W);
        if (TO > 0) {
          if (!wait_bar(s, &s.bar[BAR_BOUTREADY], bout_n & 1, args.status)) break;
          ++bout_n;
          tc_fence_after();
          for (int t = 0; t < TO && ok; ++t) ok = tile(s.Bs, 16, id_small, true);
        }
      }
    }
  } else if (warp < 2 + kEpiWarps) {
    // ============================ epilogue ============================
    const int q = warp & 3;                    // TMEM lane quarter this warp may access
    const int hf = (warp - 2) >> 2;            // column half
    constexpr int HALF = W / 2, NCH = HALF / 32;
    uint32_t tiles_done = 0;
    auto wait_tile = [&](uint32_t acc) -> bool {
      int good = 1;
      if (lane == 0) good = wait_bar(s, &s.bar[BAR_TFULL + acc], (tiles_done >> 1) & 1, args.status) ? 1 : 0;
      return __shfl_sync(0xffffffffu, good, 0) != 0;
    };
    auto release = [&](uint32_t acc) {
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&s.bar[BAR_TEMPTY + acc]);
      ++tiles_done;
    };
    for (int64_t cell = blockIdx.x; cell < ncell; cell += gridDim.x) {
      const TcNet& N = args.nets[0];
      const int H = N.H;
      if (N.w != W) continue;
      if (__shfl_sync(0xffffffffu, *(volatile int*)s.abort, 0)) break;
      bool ok = true;
      for (int j = 1; j <= H - 1 && ok; ++j) {
        // ---- the reduction pass: 16-column results per output neuron ----
        for (int mt = 0; mt < MT; ++mt) {
          const uint32_t acc = tiles_done & 1;
          if (!wait_tile(acc)) { ok = false; break; }
          tc_fence_after();
          if (hf == 0) {
            float v[16];
            tmem_ld16(tmem + acc * 256 + ((uint32_t)(32 * q) << 16), v);
            const int p = mt * 128 + 32 * q + lane;
            s.imp[p] = v[3];
            s.ig[p] = v[4];
            s.ie[p] = v[5];
          }
          release(acc);
        }
        if (!ok) break;
        // ---- main tiles: G rows of z_{j+1} ----
        if (j >= 2) {
          const bool store = j < H - 1;
          const int T = (j - 1) * MT;
          float p[NCH], comp[NCH];
#pragma unroll
          for (int ch = 0; ch < NCH; ++ch) p[ch] = comp[ch] = 0.f;
          const float* gprev = s.gamma + ((j - 1) % 3) * W;   // gamma_{j-1}: scale of implicit rows
          for (int t = 0; t < T; ++t) {
            const uint32_t acc = tiles_done & 1;
            if (!wait_tile(acc)) { ok = false; break; }
            tc_fence_after();
            const uint32_t tbase = tmem + acc * 256 + ((uint32_t)(32 * q) << 16);
            const int row = 32 * q + lane;
            const int blk = t / MT + 1, sub = t % MT;
            const bool implicit = (blk == j - 1);
            const float rs = implicit ? gprev[sub * 128 + row] : 1.0f;
            // unit-major slice: 16-byte unit u (columns 8u .. 8u+7) of slice row r at [u * rows + r], so the
            // 32 lanes (consecutive rows) of every store below write 512 contiguous bytes
            const int rowg = (blk - 1) * W + sub * 128 + row;
            uint4* slice4 = reinterpret_cast<uint4*>(scratch);
#pragma unroll
            for (int ch = 0; ch < NCH; ++ch) {
              const int col0 = hf * HALF + ch * 32;
              float v[32];
              tmem_ld32(tbase + col0, v);
              if (store) {
                uint32_t pk[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                  __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * i] * rs, v[2 * i + 1] * rs);
                  pk[i] = *reinterpret_cast<uint32_t*>(&h2);
                  const float2 f2 = __bfloat1622float2(h2);
                  v[2 * i] = f2.x;
                  v[2 * i + 1] = f2.y;
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
                  slice4[(size_t)(col0 / 8 + i) * args.rows_per_cta + rowg] =
                      make_uint4(pk[4 * i], pk[4 * i + 1], pk[4 * i + 2], pk[4 * i + 3]);
              } else {
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] *= rs;
              }
#pragma unroll
              for (int i = 0; i < 32; ++i) v[i] = clt ? v[i] * v[i] : fabsf(v[i]);
              const float sum = transpose_reduce32(v);
              const float y = sum - comp[ch];
              const float tt = p[ch] + y;
              comp[ch] = (tt - p[ch]) - y;
              p[ch] = tt;
            }
            release(acc);
          }
          if (!ok) break;
          if (store) {
            // the next layer's TMA reads these rows: make the stores visible at GPU scope, then
            // order them before the async proxy
            __threadfence();
            fence_async_global();
          }
#pragma unroll
          for (int ch = 0; ch < NCH; ++ch) s.red[q * W + hf * HALF + ch * 32 + lane] = p[ch];
        }
        if (warp == 2 && lane == 0) trace(args, 2, cell / gridDim.x, j);
        __syncwarp();
        if (lane == 0) mbar_arrive(&s.bar[BAR_RED]);
      }
      if (!ok) break;
      // ---- output pass: y rows of the stored blocks of z_{H-1} (column 0) ----
      const int TO = out_tiles(H, W);
      if (TO > 0) {
        float pout = 0.f;
        for (int t = 0; t < TO; ++t) {
          const uint32_t acc = tiles_done & 1;
          if (!wait_tile(acc)) { ok = false; break; }
          tc_fence_after();
          if (hf == 0) {
            float v[16];
            tmem_ld16(tmem + acc * 256 + ((uint32_t)(32 * q) << 16), v);
            float x = (clt || mode == ISX_BOUND_RAUA) ? v[0] * v[0] : fabsf(v[0]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            pout += x;
          }
          release(acc);
        }
        if (!ok) break;
        if (hf == 0 && lane == 0) s.red[q * W] = pout;
        __syncwarp();
        if (lane == 0) mbar_arrive(&s.bar[BAR_RED]);
      }
    }
  } else if (warp < kRingWarp) {
    // ============================ math ============================
    const int mt = threadIdx.x - kMathBase;    // 0..127
    const int mwarp = mt >> 5;
    constexpr int NPT = W / kMathThreads;      // neurons per thread (1 or 2)
    uint32_t wl_n = 0, red_n = 0, ms = 0, mph = 0, bms = 0, bmph = 0;
    const float kap = args.kappa;
    const bool sq = clt || mode == ISX_BOUND_RAUA;
    auto group_wait = [&](uint64_t* b, uint32_t parity) -> bool {
      if (mt == 0) {
        wait_bar(s, b, parity, args.status);
        s.scal[63] = *(volatile int*)s.abort ? 1.f : 0.f;
      }
      math_sync();
      return s.scal[63] == 0.f;
    };
    for (int64_t cell = blockIdx.x; cell < ncell; cell += gridDim.x) {
      const TcNet& N = args.nets[0];
      const int H = N.H;
      if (N.w != W) continue;
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
          int ijk[3] = {int(code & 1023u), int((code >> 10) & 1023u), int((code >> 20) & 1023u)};
          for (int d = 0; d < 3; ++d) {
            const float size = ldexpf(2.0f, -axis_level(src, d));
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
      const float* W0 = N.W[0];
      for (int nn = mt; nn < W; nn += kMathThreads) {
        float w0 = W0[3 * nn], w1 = W0[3 * nn + 1], w2 = W0[3 * nn + 2], b0 = N.b[0][nn];
        float c = fmaf(w2, xc[2], fmaf(w1, xc[1], fmaf(w0, xc[0], b0)));
        float x0 = h[0] * w0, x1 = h[1] * w1, x2 = h[2] * w2;
        s.I[nn] = x0;
        s.I[W + nn] = x1;
        s.I[2 * W + nn] = x2;
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
        float* al = s.alpha + (j % 3) * W;
        float* ga = s.gamma + (j % 3) * W;
        // ---- ReLU j (Eq. 4 / Eq. 9) ----
        for (int nn = mt; nn < W; nn += kMathThreads) {
          Lin L = clt ? act_clt(N.act, s.c[nn], s.r[nn]) : relu_sound(s.c[nn], s.r[nn], s.delta[nn], infl);
          al[nn] = L.alpha;
          ga[nn] = L.gamma;
          s.a[nn] = L.center;
          s.rada[nn] = infl ? fmaf(L.alpha, s.r[nn], L.gamma) : 0.0f;
        }
        math_sync();
        // ---- small B: columns of the two GEMV passes (rows 0-2: I alpha, 3: gamma or gamma^2,
        //      4: alpha r + gamma, 5: |a|), K-major 128-byte swizzle ----
        for (int k = mt; k < W; k += kMathThreads) {
          __nv_bfloat16* bs = reinterpret_cast<__nv_bfloat16*>(s.Bs);
          const float ak = al[k];
          (void)ak;
          bs[swz(16, 3, k) / 2] = __float2bfloat16_rn(clt ? ga[k] * ga[k] : ga[k]);
          bs[swz(16, 4, k) / 2] = __float2bfloat16_rn(s.rada[k]);
          bs[swz(16, 5, k) / 2] = __float2bfloat16_rn(infl ? fabsf(s.a[k]) : 0.0f);
        }
        if (mt == 0) trace(args, 0, cell / gridDim.x, 24 + 2 * (j - 1));
        if (j >= 2) {
          // ---- B = D_j W_j^T: scale the bf16 rows of W_j in place by alpha_j ----
          if (!group_wait(&s.bar[BAR_WLOADED], wl_n & 1)) { ok = false; break; }
          ++wl_n;
          if (mt == 0) trace(args, 0, cell / gridDim.x, 25 + 2 * (j - 1));
          scale_b_rows<W>(s, al, mt);
          fence_async_shared();
          math_sync();
        } else {
          fence_async_shared();
          math_sync();
        }
        if (mt == 0) mbar_arrive(&s.bar[BAR_BREADY]);
        if (mt == 0) trace(args, 0, cell / gridDim.x, 2 + 4 * (j - 1));
        // ---- centre and I rows of z_{j+1} in float32: W_j a_j + b_j and I_j D_j W_j^T (weights via the ring) ----
        {
          float acc[4][NPT], dummy[NPT];
#pragma unroll
          for (int e = 0; e < NPT; ++e) {
            acc[0][e] = acc[1][e] = acc[2][e] = acc[3][e] = 0.f;
            dummy[e] = 0.f;
          }
          const bool gok = (j == 1)
                               ? ring_gemv<W, 4, NPT, true>(s, args.status, bms, bmph, mt, lane, s.a, al, acc, dummy, false)
                               : ring_gemv<W, 4, NPT, false>(s, args.status, ms, mph, mt, lane, s.a, al, acc, dummy, false);
          if (!gok) ok = false;
          math_sync();     // every thread has read a, c and I
          if (!ok) break;
          // B is free again for W_2 (the TMA producer waits for this before loading it)
          if (j == 1 && mt == 0) mbar_arrive(&s.bar[BAR_RINGBFREE]);
#pragma unroll
          for (int e = 0; e < NPT; ++e) {
            const int nn = mt + e * kMathThreads;
            s.c[nn] = acc[0][e] + N.b[j][nn];
            s.Inew[nn] = acc[1][e];
            s.Inew[W + nn] = acc[2][e];
            s.Inew[2 * W + nn] = acc[3][e];
          }
        }
        if (mt == 0) trace(args, 0, cell / gridDim.x, 3 + 4 * (j - 1));
        // ---- combine: radius and slack of z_{j+1} ----
        if (!group_wait(&s.bar[BAR_RED], red_n & 1)) { ok = false; break; }
        ++red_n;
        if (mt == 0) trace(args, 0, cell / gridDim.x, 4 + 4 * (j - 1));
        const bool stored = (j >= 2) && (j < H - 1);
        const float* bj = N.b[j];
        for (int nn = mt; nn < W; nn += kMathThreads) {
          const float tc = (j >= 2) ? s.red[nn] + s.red[W + nn] + s.red[2 * W + nn] + s.red[3 * W + nn] : 0.f;
          const float i0 = s.Inew[nn], i1 = s.Inew[W + nn], i2 = s.Inew[2 * W + nn];
          const float rI = clt ? i0 * i0 + i1 * i1 + i2 * i2 : fabsf(i0) + fabsf(i1) + fabsf(i2);
          const float imp = clt ? s.imp[nn] : s.imp[nn] * (infl ? kGemvSafe : 1.0f);
          const float tot = tc + rI + imp;
          s.rprev[nn] = s.r[nn];
          s.r[nn] = clt ? sqrtf(tot) : tot;
          s.delta[nn] = infl ? (kap * s.ig[nn] + gamma_k(W + 2, kLinU) * (s.ie[nn] + fabsf(bj[nn]))) * kGemvSafe +
                                   (stored ? kUb / (1.0f - kUb) * tc * kLinSafe : 0.f)
                             : 0.f;
          s.I[nn] = i0;
          s.I[W + nn] = i1;
          s.I[2 * W + nn] = i2;
        }
        math_sync();
        if (mt == 0) trace(args, 0, cell / gridDim.x, 5 + 4 * (j - 1));
      }
      if (!ok) break;
      // ---- ReLU H, then the output layer (through layer H-1 for the G rows) ----
      float* al = s.alpha + (H % 3) * W;
      float* ga = s.gamma + (H % 3) * W;
      const float* wout = N.W[H];
      for (int nn = mt; nn < W; nn += kMathThreads) {
        Lin L = clt ? act_clt(N.act, s.c[nn], s.r[nn]) : relu_sound(s.c[nn], s.r[nn], s.delta[nn], infl);
        al[nn] = L.alpha;
        ga[nn] = L.gamma;
        s.a[nn] = L.center;
        s.Inew[nn] = L.alpha * wout[nn];          // alpha_H * w_out (x of the v GEMV)
      }
      math_sync();
      if (mt == 0) trace(args, 0, cell / gridDim.x, 40);
      const float* alm1 = s.alpha + ((H - 1) % 3) * W;
      float* v = s.imp;
      float* u = s.ig;
      float* vabs = s.ie;
      {
        // v_k = sum_n W_{H-1}[n][k] alpha_H,n w_out,n (rows n of W_{H-1} through the ring)
        float acc[1][NPT], aacc[NPT];
#pragma unroll
        for (int e = 0; e < NPT; ++e) acc[0][e] = aacc[e] = 0.f;
        if (!ring_gemv<W, 1, NPT, true>(s, args.status, bms, bmph, mt, lane, s.Inew, al, acc, aacc, true)) ok = false;
        math_sync();
        if (!ok) break;
#pragma unroll
        for (int e = 0; e < NPT; ++e) {
          const int k = mt + e * kMathThreads;
          v[k] = acc[0][e];
          vabs[k] = aacc[e];
          u[k] = alm1[k] * acc[0][e];
        }
      }
      math_sync();
      const int TO = out_tiles(H, W);
      if (TO > 0) {
        // Bs row 0 = bf16(u), rows 1-5 cleared
        __nv_bfloat16* bs = reinterpret_cast<__nv_bfloat16*>(s.Bs);
        for (int k = mt; k < W; k += kMathThreads) {
          bs[swz(16, 0, k) / 2] = __float2bfloat16_rn(u[k]);
          for (int rr = 1; rr < 6; ++rr) bs[swz(16, rr, k) / 2] = __float2bfloat16_rn(0.0f);
        }
        fence_async_shared();
        math_sync();
        if (mt == 0) mbar_arrive(&s.bar[BAR_BOUTREADY]);
      }
      float gsum[NPT];
#pragma unroll
      for (int e = 0; e < NPT; ++e) gsum[e] = 0.f;
      if (H >= 3) {
        // implicit G_{H-2} at z_{H-1}: sum_n W_{H-2}[n][m] u_n (rows n of W_{H-2} through the ring)
        float dummy[NPT], g1[1][NPT];
#pragma unroll
        for (int e = 0; e < NPT; ++e) g1[0][e] = dummy[e] = 0.f;
        if (!ring_gemv<W, 1, NPT, true>(s, args.status, bms, bmph, mt, lane, u, al, g1, dummy, false)) ok = false;
        if (!ok) { math_sync(); break; }
#pragma unroll
        for (int e = 0; e < NPT; ++e) gsum[e] = g1[0][e];
      }
      float acc = 0.f, eabs = 0.f, x0p = 0.f, cen = 0.f;
      const float* gam1 = s.gamma + ((H - 1) % 3) * W;
      const float* gam2 = s.gamma + ((H - 2) % 3) * W;
#pragma unroll
      for (int e = 0; e < NPT; ++e) {
        const int m = mt + e * kMathThreads;
        if (H >= 3) {
          const float y = gam2[m] * gsum[e];
          acc += sq ? y * y : fabsf(y);
        }
        const float y1 = gam1[m] * v[m];
        const float y2 = ga[m] * wout[m];
        acc += sq ? y1 * y1 + y2 * y2 : fabsf(y1) + fabsf(y2);
        x0p = fmaf(wout[m], s.a[m], x0p);
        if (infl) {
          eabs += s.rprev[m] * alm1[m] * vabs[m] + gam1[m] * vabs[m] + (s.r[m] * al[m] + ga[m]) * fabsf(wout[m]);
          cen = fmaf(fabsf(wout[m]), fabsf(s.a[m]), cen);
        }
      }
      if (mt < 3) {
        float y = 0.f;
        for (int k = 0; k < W; ++k) y = fmaf(s.I[mt * W + k], s.Inew[k], y);   // I rows of z_H . alpha_H w_out
        acc += sq ? y * y : fabsf(y);
      }
      float vals[4] = {acc, eabs, x0p, cen};
#pragma unroll
      for (int qv = 0; qv < 4; ++qv) {
        float x = vals[qv];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) s.scal[qv * 4 + mwarp] = x;
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
        if (TO > 0) tot += s.red[0] + s.red[W] + s.red[2 * W] + s.red[3 * W];
        const float x0 = xp + N.bout;
        float sp;
        if (mode == ISX_BOUND_SOUND) {
          sp = tot;
          if (infl)
            sp = __fadd_ru(__fmul_ru(sp, kLinSafe),
                           (args.kappa_out * ea + gamma_k(W + 2, kLinU) * (ce + fabsf(N.bout))) * 1.01f);
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

// The stored-row scratch of `grid` CTAs, unit-major per CTA (16-byte unit u of slice row r at
// [u * rows + r]): a 3-D map {8 elements, rows, units x CTAs} with box {8, 128, 8}, no swizzle.
isx_status make_scratch_map(CUtensorMap* m, const void* base, int w, int rows, int grid);

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

isx_status make_scratch_map(CUtensorMap* m, const void* base, int w, int rows, int grid) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available");
    return ISX_ERR_CUDA;
  }
  cuuint64_t dims[3] = {8, (cuuint64_t)rows, (cuuint64_t)(w / 8) * (cuuint64_t)grid};
  cuuint64_t strides[2] = {16, (cuuint64_t)rows * 16};
  cuuint32_t box[3] = {8, 128, 8};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (scratch) failed with code " + std::to_string((int)r));
    return ISX_ERR_CUDA;
  }
  return ISX_OK;
}

}  // namespace

namespace {
// The network descriptor of an INR (tensor maps of its BF16 copies, weight pointers), built once
// and kept in device memory with the INR.
isx_status build_net(isx_inr inr, TcNet* h) {
  std::memset(h, 0, sizeof(*h));
  const int w = inr->w;
  for (int l = 1; l < inr->n_layers - 1; ++l) {
    ISX_TRY(make_map(&h->wt[l], inr->Wt_bf16[l], w, w, 64, 128));
    ISX_TRY(make_map(&h->wrow[l], inr->W_bf16[l], w, w, 64, w));
    ISX_TRY(make_map(&h->wabs[l], inr->Wabs_bf16[l], w, w, 64, 128));
    ISX_TRY(make_map(&h->wsq[l], inr->Wsq_bf16[l], w, w, 64, 128));
  }
  for (int l = 0; l < inr->n_layers; ++l) {
    h->W[l] = inr->W[l];
    h->Wt[l] = inr->Wt[l];
    h->b[l] = inr->b[l];
  }
  h->bout = inr->hb[inr->n_layers - 1][0];
  h->H = inr->H;
  h->w = inr->w;
  h->act = inr->act;
  return ISX_OK;
}

// Shared-memory opt-in and the launch of the width-specialised kernel.
isx_status launch_tc(int w, const TcArgs& a, TcMaps& maps, int grid, cudaStream_t st) {
  const size_t smem = smem_bytes(w);
  if (w == 256) {
    ISX_CUDA(cudaFuncSetAttribute(k_bound_tc<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_bound_tc<256><<<grid, kThreads, smem, st>>>(a, maps);
  } else {
    ISX_CUDA(cudaFuncSetAttribute(k_bound_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_bound_tc<128><<<grid, kThreads, smem, st>>>(a, maps);
  }
  ISX_LAUNCH_CHECK("k_bound_tc");
  return ISX_OK;
}

void set_kappas(TcArgs& a, int w) {
  const float ub = kUb, ua = kUa, u = kLinU;
  const float gK = (w * ua) / (1.0f - w * ua), gK32 = (w * u) / (1.0f - w * u);
  a.kappa = (1 + ub) * (1 + ub) * (1 + ub) * (1 + gK) * (1 + u) - 1;
  a.kappa_out = (1 + ub) * (1 + gK) * (1 + gK32) * (1 + gK32) * (1 + u) * (1 + u) - 1;
}
}  // namespace

// Device copy of the INR's network descriptor (built on first use).
isx_status tc_net_of(isx_inr inr, const void** out) {
  if (!inr->tc_net) {
    TcNet h;
    ISX_TRY(build_net(inr, &h));
    void* d = nullptr;
    ISX_CUDA(cudaMalloc(&d, sizeof(TcNet)));
    cudaError_t e = cudaMemcpy(d, &h, sizeof(TcNet), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(d);
      return cuda_fail(e, "network descriptor", __FILE__, __LINE__);
    }
    inr->tc_net = d;
  }
  *out = inr->tc_net;
  return ISX_OK;
}

size_t tc_net_bytes() { return sizeof(TcNet); }

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
  const int w = inr->w, H = inr->H;
  int dev = inr->device, sms = 0;
  ISX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = (int)std::min<int64_t>(n, sms);
  const int rows = std::max(128, w * std::max(0, H - 3));   // >= one 128-row TMA box
  auto& ws = inr->ws;
  ISX_TRY(ws[WS_TC_SCRATCH].ensure((size_t)sms * rows * w * 2, "tc scratch"));
  ISX_TRY(ws[WS_TC_STATUS].ensure(64, "tc status"));
  const void* net = nullptr;
  ISX_TRY(tc_net_of(inr, &net));
  TcArgs a{};
  a.src = src;
  a.n = n;
  a.mode = (int)mode;
  a.inflate = (mode == ISX_BOUND_SOUND) ? inflate : 0;
  a.w = w;
  a.nets = static_cast<const TcNet*>(net);
  a.scratch = ws[WS_TC_SCRATCH].as<__nv_bfloat16>();
  a.rows_per_cta = rows;
  a.center = d_center;
  a.spread = d_spread;
  a.status = ws[WS_TC_STATUS].as<int>();
  set_kappas(a, w);
  TcMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  ISX_TRY(make_scratch_map(&maps.scratch, a.scratch, w, rows, sms));
  ISX_CUDA(cudaMemsetAsync(a.status, 0, sizeof(int), st));
  const bool tracing = std::getenv("ISX_TRACE") != nullptr;
  a.trace = nullptr;
  if (tracing) {
    ISX_TRY(ws[WS_AUX].ensure(3 * kTraceCells * kTraceEvents * sizeof(long long), "trace"));
    a.trace = ws[WS_AUX].as<long long>();
    ISX_CUDA(cudaMemsetAsync(a.trace, 0, 3 * kTraceCells * kTraceEvents * sizeof(long long), st));
  }
  {
    const double cells = (double)n;
    const double rows_gemm = (double)w * (H - 1) * (H - 2) / 2.0;   // G rows over layers 2..H-1
    prof::Scope ps(K_BOUND_TC, st, cells * 2.0 * w * w * (3.0 * (H - 1) + rows_gemm), 0);
    ISX_TRY(launch_tc(w, a, maps, grid, st));
  }
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
  const int rows = std::max(128, w * std::max(0, H - 3));   // >= one 128-row TMA box
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
  if (!inr->tc_net) {
    set_error("isx_bound_cells_noalloc: the INR has no network descriptor (created with the INR)");
    return ISX_ERR_UNSUPPORTED;
  }
  a.nets = static_cast<const TcNet*>(inr->tc_net);
  a.status = reinterpret_cast<int*>(base);
  a.scratch = reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<uint8_t*>(base) + kStaticStatusBytes);
  a.rows_per_cta = (int)(per_cta / (w * 2));
  a.center = d_center;
  a.spread = d_spread;
  a.trace = nullptr;
  set_kappas(a, w);
  TcMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  ISX_TRY(make_scratch_map(&maps.scratch, a.scratch, w, a.rows_per_cta, grid));
  // the status word must start at zero on every call; the slices need no clearing (every row is
  // written before it is read)
  ISX_CUDA(cudaMemsetAsync(a.status, 0, sizeof(int), st));
  {
    const double rows_gemm = (double)w * (H - 1) * (H - 2) / 2.0;
    prof::Scope ps(K_BOUND_TC, st, (double)n * 2.0 * w * w * (3.0 * (H - 1) + rows_gemm), 0);
    ISX_TRY(launch_tc(w, a, maps, grid, st));
  }
  int status = 0;
  ISX_CUDA(cudaMemcpyAsync(&status, a.status, sizeof(int), cudaMemcpyDeviceToHost, st));
  ISX_CUDA(cudaStreamSynchronize(st));
  if (status != 0) {
    set_error("tensor-core bound kernel gave up waiting (bounded wait expired)");
    return (isx_status)status;
  }
  return ISX_OK;
}
