// The row GEMM of the row-batched tensor-core bound path: G' = (G diag(alpha_cell)) W_j^T over the
// symbol rows of every cell of a chunk (Eq. 3 / Eq. 8 on the stored symbol blocks, with the
// activation's alpha (Eq. 4 / Eq. 9) applied to the rows), one tcgen05 GEMM per layer.
#include "rows.cuh"

#include <algorithm>

namespace isx {
namespace rows {
namespace {

using namespace tc;

template <int W>
struct RowsSmem {
  static constexpr int KC = W / 64;
  static constexpr int NQ = W > 256 ? W / 128 : 1;         // weight slices: W = 512 is split into 4 CTAs' quarters
  static constexpr int MW = W > 256 ? 128 : (W < 128 ? 128 : W);   // weight rows a CTA holds (W = 64: zero-padded)
  static constexpr int NH = MW / 128;                      // 128-row MMA halves of those rows
  static constexpr int NS = (W >= 256) ? 5 : 4;            // row ring: one 64-wide K chunk of a tile each
  static constexpr size_t kWB = (size_t)MW * W * 2;        // the weight rows, KC chunks of [MW rows][128 B]
  static constexpr size_t kAC = (size_t)kRT * 128;         // one row chunk: [128 rows][128 B]
  static constexpr size_t kMeta = 2 * kRT * (8 + 4);       // two tiles' destination rows and cells
  static constexpr size_t bytes() { return 1024 + kWB + NS * kAC + kMeta + (3 * NS + 5) * 8 + 16; }
};

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// G' = (G diag(alpha_cell)) W^T for all rows, computed transposed: D = W_j (G diag(alpha))^T, so that
// TMEM lane m holds neuron rows_weight_row(m) and column r the tile's row r.  Persistent,
// warp-specialised CTAs over 128-row tiles:
//  - warp 5 streams the rows of G by TMA, one 64-wide K chunk of a tile per stage of an NS-stage
//    ring, in the 128-byte-swizzled K-major layout of the MMA's B operand;
//  - warps 0-3 scale each staged chunk in place: thread t multiplies row t by its cell's alpha
//    (rows past R stay the TMA's zero fill);
//  - warp 4 loads W_j (bf16, [MW][W], K-major) once by TMA, owns TMEM and issues the MMAs (M = 128
//    per weight half, N = 128 rows, K = 16 per instruction).  W = 512 does not fit in shared memory:
//    each CTA then holds a 128-row quarter of W_j, and a tile's four quarters go to four CTAs;
//  - warps 6-13 drain the two TMEM accumulators, two warps per TMEM lane group: warps 6-9 take rows
//    0-63 of a tile, warps 10-13 rows 64-127.  Thread m owns the neurons of weight row m of each
//    half and walks its 64 rows in order: it stores each row's bf16 value (a bf16 pair for
//    W = 256) and adds f(value) to a running sum that it writes to part[cell + t] (t the 64-row
//    block of the input rows) whenever the row's cell changes (|stored bf16 value| for the radius,
//    which the rounding-error bound needs; the square of the float32 accumulator value for sigma,
//    within 2^-7 of the stored value's).
//    Every thread sees the same rows, so the segment boundaries are uniform; a segment's rows are
//    consecutive in the output too, so its destination advances by one row per row.
//    The destination row and cell of every row of the next tile are loaded while this tile drains
//    and handed over through shared memory.
// The scalers load the alpha of the next chunk (of this tile, or of the next tile) into registers
// as soon as they have handed over the current one.  Loads of tile k + 1 and the epilogue of tile k - 1 overlap
// the MMAs of tile k.  Every wait is bounded (2 s): on timeout the kernel records ISX_ERR_TIMEOUT,
// lets the work in flight finish, frees TMEM and returns.
constexpr int kGT = 448;                        // 4 scalers, MMA, producer, 8 epilogue warps
template <int W, bool SQ>
__global__ void __launch_bounds__(kGT, 1) k_rows_gemm(const __grid_constant__ RowsGemmArgs args,
                                                       const __grid_constant__ CUtensorMap wmap,
                                                       const __grid_constant__ CUtensorMap xmap) {
  using S = RowsSmem<W>;
  constexpr int KC = S::KC, NS = S::NS, MW = S::MW, NH = S::NH, NQ = S::NQ;
  constexpr uint32_t kCols = 2 * NH * 128;                 // two accumulators of NH x 128 columns
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* Wsm = base;
  uint8_t* Asm = Wsm + S::kWB;
  long long* mdst = reinterpret_cast<long long*>(Asm + NS * S::kAC);   // [2][128]
  int* mcell = reinterpret_cast<int*>(mdst + 2 * kRT);                  // [2][128]
  uint64_t* araw = reinterpret_cast<uint64_t*>(mcell + 2 * kRT);
  uint64_t* afull = araw + NS;
  uint64_t* aempty = afull + NS;
  uint64_t* tfull = aempty + NS;
  uint64_t* tempty = tfull + 2;
  uint64_t* wfull = tempty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(wfull + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int64_t ntiles = (args.R + kRT - 1) / kRT;
  // work items are (tile, weight slice); the grid is a multiple of NQ, so this CTA's slice q never
  // changes and it walks the tiles t0, t0 + TS, ...; the NQ CTAs of a tile run side by side and
  // share its row chunks through L2
  const int q = blockIdx.x % NQ;
  const int64_t t0 = blockIdx.x / NQ, TS = gridDim.x / NQ;

  if (W < 128) {
    // zero rows W .. 127 of every weight chunk (the MMA reads 128 weight rows)
    for (int c = 0; c < KC; ++c)
      for (int i = t; i < (MW - W) * 128 / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(Wsm + (size_t)c * MW * 128 + (size_t)W * 128)[i] = make_uint4(0, 0, 0, 0);
    fence_async_shared();
  }
  if (t == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&araw[i], 1);
      mbar_init(&afull[i], kRT);
      mbar_init(&aempty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 8);
    }
    mbar_init(wfull, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "n"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp < 4) {
    // ---- scale row t of every staged chunk by alpha of its cell, in place ----
    uint32_t it = 0;
    bool ok = true;
    int64_t r_next = t0 * kRT + t;
    int cell_next = (r_next < args.R) ? args.rowcell[r_next] : 0;
    float4 av[16];
    {
      const float4* al0 = reinterpret_cast<const float4*>(args.alpha + (size_t)cell_next * W);
#pragma unroll
      for (int g = 0; g < 16; ++g) av[g] = al0[g];
    }
    for (int64_t tile = t0; tile < ntiles && ok; tile += TS) {
      const int64_t r = tile * kRT + t;
      const bool valid = r < args.R;
      const int cell = cell_next;
      r_next = (tile + TS) * kRT + t;
      cell_next = (tile + TS < ntiles && r_next < args.R) ? args.rowcell[r_next] : cell;
      {
        // ask L2 for the alpha rows of the cells of this warp's 32 rows of the next tile (a run of
        // consecutive cells, so one contiguous range), a tile ahead of their use
        const int cf = __shfl_sync(0xffffffffu, cell_next, 0), cl = __shfl_sync(0xffffffffu, cell_next, 31);
        if (lane == 0 && tile + TS < ntiles && cl >= cf) {
          const uint32_t bytes = (uint32_t)min((cl - cf + 1) * W * 4, 32 * 1024);
          asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(args.alpha + (size_t)cf * W), "r"(bytes)
                       : "memory");
        }
      }
      for (int c = 0; c < KC; ++c, ++it) {
        const int sidx = it % NS;
        if (!rwait(&araw[sidx], (it / NS) & 1, abort, args.status)) { ok = false; break; }
        uint8_t* Ac = Asm + (size_t)sidx * S::kAC;
        if (valid) {
#pragma unroll
          for (int g = 0; g < 8; ++g) {
            uint4* p = reinterpret_cast<uint4*>(Ac + roff(t, 8 * g));
            const uint4 x = *p;
            const float4 a0 = av[2 * g], a1 = av[2 * g + 1];
            const __nv_bfloat162* xb = reinterpret_cast<const __nv_bfloat162*>(&x);
            const float2 x0 = __bfloat1622float2(xb[0]), x1 = __bfloat1622float2(xb[1]);
            const float2 x2 = __bfloat1622float2(xb[2]), x3 = __bfloat1622float2(xb[3]);
            const __nv_bfloat162 p0 = __floats2bfloat162_rn(x0.x * a0.x, x0.y * a0.y);
            const __nv_bfloat162 p1 = __floats2bfloat162_rn(x1.x * a0.z, x1.y * a0.w);
            const __nv_bfloat162 p2 = __floats2bfloat162_rn(x2.x * a1.x, x2.y * a1.y);
            const __nv_bfloat162 p3 = __floats2bfloat162_rn(x3.x * a1.z, x3.y * a1.w);
            *p = make_uint4(*reinterpret_cast<const uint32_t*>(&p0), *reinterpret_cast<const uint32_t*>(&p1),
                            *reinterpret_cast<const uint32_t*>(&p2), *reinterpret_cast<const uint32_t*>(&p3));
          }
        }
        fence_async_shared();
        mbar_arrive(&afull[sidx]);
        // alpha of the next chunk (of this tile, or of the next tile), in flight during the next wait
        const float4* aln = (c + 1 < KC) ? reinterpret_cast<const float4*>(args.alpha + (size_t)cell * W) + 16 * (c + 1)
                                         : reinterpret_cast<const float4*>(args.alpha + (size_t)cell_next * W);
#pragma unroll
        for (int g = 0; g < 16; ++g) av[g] = aln[g];
      }
    }
  } else if (warp == 5) {
    // ---- TMA producer of the row chunks ----
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int64_t tile = t0; tile < ntiles && ok; tile += TS) {
        for (int c = 0; c < KC; ++c, ++it) {
          const int sidx = it % NS;
          if (!rwait(&aempty[sidx], ((it / NS) & 1) ^ 1, abort, args.status)) { ok = false; break; }
          mbar_expect_tx(&araw[sidx], (uint32_t)S::kAC);
          tma_load_2d(Asm + (size_t)sidx * S::kAC, &xmap, &araw[sidx], c * 64, (int)(tile * kRT));
        }
      }
    }
  } else if (warp == 4) {
    // ---- W_j once, then the MMAs: D[half h] += W_j[h rows] x chunk^T ----
    if (lane == 0) {
      // the CTA's weight rows: all of W_j, or rows q * 128 .. q * 128 + 127 of it
      constexpr int rows_held = W < MW ? W : MW;
      mbar_expect_tx(wfull, (uint32_t)((size_t)rows_held * W * 2));
      for (int c = 0; c < KC; ++c)
        tma_load_2d(Wsm + (size_t)c * MW * 128, &wmap, wfull, c * 64, NQ > 1 ? q * 128 : 0);
      const uint32_t id = idesc(kRT);
      uint32_t it = 0, tt = 0;
      bool ok = rwait(wfull, 0, abort, args.status);
      for (int64_t tile = t0; tile < ntiles && ok; tile += TS, ++tt) {
        const uint32_t b = tt & 1;
        if (!rwait(&tempty[b], ((tt >> 1) & 1) ^ 1, abort, args.status)) break;
        tc_fence_after();
        const uint32_t dt = tmem + b * (NH * 128);
        for (int c = 0; c < KC; ++c, ++it) {
          const int sidx = it % NS;
          if (!rwait(&afull[sidx], (it / NS) & 1, abort, args.status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t x0 = su32(Asm + (size_t)sidx * S::kAC), w0 = su32(Wsm + (size_t)c * MW * 128);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
#pragma unroll
            for (int h = 0; h < NH; ++h)
              mma_bf16(dt + h * 128, sdesc(w0 + h * 128 * 128 + kk * 32), sdesc(x0 + kk * 32), id,
                       (c > 0 || kk > 0) ? 1u : 0u);
          mma_commit(&aempty[sidx]);
        }
        if (ok) mma_commit(&tfull[b]);
      }
    }
  } else {
    // ---- epilogue: TMEM -> bf16 rows of G' and the per-(cell, 64-row block) column sums of f(G') ----
    const int m = 32 * (warp & 3) + lane;                  // weight row (TMEM lane) of this thread
    const int h = (warp - 6) >> 2;                          // rows 64 h .. 64 h + 63 of every tile
    const bool own = m < W;                                 // W = 64: rows 64 .. 127 are padding
    const int n0 = (W == 256) ? 2 * m : q * 128 + m;        // first neuron of this thread
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    // metadata of this thread's row of the first tile, and the cell of its row of the second
    int64_t tile = t0;
    int c_cur = -1, c_nxt = -1;
    long long d_cur = 0;
    {
      const int64_t r = tile * kRT + m;
      if (tile < ntiles && r < args.R) {
        c_cur = args.rowcell[r];
        d_cur = args.off_out[c_cur] + (r - args.off_in[c_cur]);
      }
      const int64_t r2 = (tile + TS) * kRT + m;
      if (tile + TS < ntiles && r2 < args.R) c_nxt = args.rowcell[r2];
    }
    uint32_t tt = 0;
    for (; tile < ntiles; tile += TS, ++tt) {
      const uint32_t b = tt & 1;
      int* scell = mcell + b * kRT;
      long long* sdst = mdst + b * kRT;
      if (h == 0) {
        scell[m] = c_cur;
        sdst[m] = d_cur;
      }
      epi_bar();
      // the next tile's destination rows (its cells came one tile earlier) and the cells of the tile
      // after it: in flight while this tile drains
      if (h == 0) {
        const int64_t nt = tile + TS;
        const int64_t r1 = nt * kRT + m;
        c_cur = c_nxt;
        if (nt < ntiles && r1 < args.R && c_cur >= 0) d_cur = args.off_out[c_cur] + (r1 - args.off_in[c_cur]);
        const int64_t r2 = (nt + TS) * kRT + m;
        c_nxt = (nt + TS < ntiles && r2 < args.R) ? args.rowcell[r2] : -1;
      }
      // after an expired wait every epilogue warp keeps walking the tiles without work, so that all of
      // them still meet at the barrier above
      const bool got = rwait(&tfull[b], (tt >> 1) & 1, abort, args.status);
      if (!__all_sync(0xffffffffu, got)) continue;
      tc_fence_after();
      const int64_t left = args.R - tile * kRT;
      const int rbeg = kPT * h;                             // this warp's rows rbeg .. rows - 1
      const int rows = (int)(left < rbeg + kPT ? left : rbeg + kPT);
      const uint32_t tb = tmem + b * (NH * 128) + lane_off;
      const int64_t blk = 2 * tile + h;                     // 64-row block of the input rows
      // running sums of the current (cell, block) segment and the destination of its next row
      float s0 = 0.0f, s1 = 0.0f;
      int seg = rbeg < rows ? scell[rbeg] : 0;
      __nv_bfloat16* dp = args.xout + (size_t)(rbeg < rows ? sdst[rbeg] : 0) * W + n0;
#pragma unroll 1
      for (int c0 = rbeg; c0 < rows; c0 += 32) {
        // rows c0 .. c0 + 31: which of them start a segment (a ballot over the warp's lanes), and
        // each lane's row's cell and destination, handed to the row loop by shuffles
        const int rl = c0 + lane;
        const int cl = rl < rows ? scell[rl] : -1;
        const long long dl = rl < rows ? sdst[rl] : 0;
        const uint32_t starts = __ballot_sync(0xffffffffu, rl < rows && rl > rbeg && cl != scell[rl - 1]);
        float v0[32], v1[32];
        tmem_ld32(tb + c0, v0);
        if (NH == 2) tmem_ld32(tb + 128 + c0, v1);
        // row c0 + i: close the segment that ends before it, then store it and add it to the sums.
        // The loops below run over constant i (no early exit), so v0[i] / v1[i] stay registers.
        auto row = [&](int i, float x0, float x1) {
          if ((starts >> i) & 1u) {                        // uniform: every thread sees the same rows
            if (own) {
              float* pp = args.part + (size_t)rows_part_slot(seg, blk) * W + n0;
              if (NH == 2) *reinterpret_cast<float2*>(pp) = make_float2(s0, s1);
              else *pp = s0;
            }
            s0 = s1 = 0.0f;
            seg = __shfl_sync(0xffffffffu, cl, i);
            dp = args.xout + (size_t)__shfl_sync(0xffffffffu, dl, i) * W + n0;
          }
          if (NH == 2) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
            *reinterpret_cast<__nv_bfloat162*>(dp) = h;
            if (SQ) {
              s0 = fmaf(x0, x0, s0);
              s1 = fmaf(x1, x1, s1);
            } else {                                       // the radius sums the stored values
              const float2 f = __bfloat1622float2(h);
              s0 += fabsf(f.x);
              s1 += fabsf(f.y);
            }
          } else if (own) {
            const __nv_bfloat16 h = __float2bfloat16_rn(x0);
            *dp = h;
            s0 = SQ ? fmaf(x0, x0, s0) : s0 + fabsf(__bfloat162float(h));
          }
          dp += W;
        };
        if (rows - c0 >= 32) {
#pragma unroll
          for (int i = 0; i < 32; ++i) row(i, v0[i], NH == 2 ? v1[i] : 0.0f);
        } else {
          const int nl = rows - c0;                        // the last tile's last rows
#pragma unroll
          for (int i = 0; i < 32; ++i)
            if (i < nl) row(i, v0[i], NH == 2 ? v1[i] : 0.0f);
        }
      }
      if (own && rbeg < rows) {
        float* pp = args.part + (size_t)rows_part_slot(seg, blk) * W + n0;
        if (NH == 2) *reinterpret_cast<float2*>(pp) = make_float2(s0, s1);
        else *pp = s0;
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[b]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (*abort)
    for (int i = 0; i < 1000; ++i) __nanosleep(1000);
  if (warp == 4) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kCols) : "memory");
  }
}

template <int W, bool SQ>
isx_status launch_rows_gemm_w(isx_inr inr, const RowsGemmArgs& a, const CUtensorMap& map, cudaStream_t st) {
  CUtensorMap xmap;
  ISX_TRY(tensor_map_bf16(&xmap, a.xin, W, (uint64_t)a.R, 64, kRT));
  const size_t smem = RowsSmem<W>::bytes();
  ISX_CUDA(cudaFuncSetAttribute(k_rows_gemm<W, SQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int sms = 148;
  ISX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, inr->device));
  int per_sm = 1;
  ISX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rows_gemm<W, SQ>, kGT, smem));
  per_sm = std::max(1, std::min(per_sm, 512 / (2 * RowsSmem<W>::NH * 128)));   // TMEM columns per CTA
  constexpr int NQ = RowsSmem<W>::NQ;
  const int64_t ntiles = (a.R + kRT - 1) / kRT;
  int grid = (int)std::min<int64_t>(ntiles * NQ, (int64_t)sms * per_sm);
  grid -= grid % NQ;                                       // every CTA keeps one weight slice
  k_rows_gemm<W, SQ><<<grid, kGT, smem, st>>>(a, map, xmap);
  ISX_LAUNCH_CHECK("k_rows_gemm");
  return ISX_OK;
}

// One CTA waits, through rwait, on an mbarrier that nothing arrives on: the wait expires after
// limit_ns and records ISX_ERR_TIMEOUT, as in the GEMM kernels when a hand-off never comes.
__global__ void k_wait_check(uint64_t limit_ns, int* status) {
  __shared__ uint64_t bar;
  __shared__ int ab;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    ab = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) rwait(&bar, 0, &ab, status, limit_ns);
  __syncthreads();
}

}  // namespace

isx_status check_bounded_wait(int64_t limit_ns, int* d_status, cudaStream_t st) {
  k_wait_check<<<1, 32, 0, st>>>((uint64_t)limit_ns, d_status);
  ISX_LAUNCH_CHECK("k_wait_check");
  return ISX_OK;
}

isx_status launch_rows_gemm(isx_inr inr, const RowsGemmArgs& a, const CUtensorMap& wmap, int w, cudaStream_t st) {
  if (a.sq) {
    if (w == 512) return launch_rows_gemm_w<512, true>(inr, a, wmap, st);
    if (w == 256) return launch_rows_gemm_w<256, true>(inr, a, wmap, st);
    if (w == 128) return launch_rows_gemm_w<128, true>(inr, a, wmap, st);
    return launch_rows_gemm_w<64, true>(inr, a, wmap, st);
  }
  if (w == 512) return launch_rows_gemm_w<512, false>(inr, a, wmap, st);
  if (w == 256) return launch_rows_gemm_w<256, false>(inr, a, wmap, st);
  if (w == 128) return launch_rows_gemm_w<128, false>(inr, a, wmap, st);
  return launch_rows_gemm_w<64, false>(inr, a, wmap, st);
}

}  // namespace rows
}  // namespace isx
