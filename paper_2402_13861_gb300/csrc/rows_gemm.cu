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
  static constexpr int NS = (W == 256) ? 5 : 4;            // A ring: one 64-wide K chunk of a tile each
  static constexpr size_t kWB = (size_t)W * W * 2;         // W_j, KC chunks of [W rows][128 B]
  static constexpr size_t kAC = (size_t)kRT * 128;         // one A chunk: [128 rows][128 B]
  static constexpr size_t bytes() { return 1024 + kWB + NS * kAC + (3 * NS + 5) * 8 + 16; }
};

// G' = (G diag(alpha_cell)) W^T for all rows: persistent, warp-specialised CTAs over 128-row tiles.
//  - warp 5 streams the rows of G by TMA, one 64-wide K chunk of a tile per stage of an NS-stage
//    ring, already in the 128-byte-swizzled K-major layout of the MMA's A operand;
//  - warps 0-3 scale each staged chunk in place: thread t multiplies row t by its cell's alpha
//    (rows past R stay the TMA's zero fill);
//  - warp 4 loads W_j (bf16, [out][in] = N x K, K-major) once by TMA, owns TMEM and issues the MMAs;
//  - warps 6-9 drain the two TMEM accumulators to bf16 rows of G' (lane group = warp mod 4).
// The scalers load the alpha of the next chunk (of this tile, or of the next tile) into registers
// before they wait for the current one: alpha rows are not L2-resident at chunk scale, so their
// latency would otherwise sit on every chunk.
// Loads of tile k + 1 and the epilogue of tile k - 1 overlap the MMAs of tile k.  Every wait is
// bounded (2 s): on timeout the kernel records ISX_ERR_TIMEOUT, lets the work in flight finish,
// frees TMEM and returns.
constexpr int kGT = 320;
template <int W>
__global__ void __launch_bounds__(kGT, 1) k_rows_gemm(const __grid_constant__ RowsGemmArgs args,
                                                       const __grid_constant__ CUtensorMap wmap,
                                                       const __grid_constant__ CUtensorMap xmap) {
  using S = RowsSmem<W>;
  constexpr int KC = S::KC, NS = S::NS;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* Wsm = base;
  uint8_t* Asm = Wsm + S::kWB;
  uint64_t* araw = reinterpret_cast<uint64_t*>(Asm + NS * S::kAC);
  uint64_t* afull = araw + NS;
  uint64_t* aempty = afull + NS;
  uint64_t* tfull = aempty + NS;
  uint64_t* tempty = tfull + 2;
  uint64_t* wfull = tempty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(wfull + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int64_t ntiles = (args.R + kRT - 1) / kRT;

  if (t == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&araw[i], 1);
      mbar_init(&afull[i], kRT);
      mbar_init(&aempty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 4);
    }
    mbar_init(wfull, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "n"(2 * W)
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
    int64_t r_next = (int64_t)blockIdx.x * kRT + t;
    int cell_next = (r_next < args.R) ? args.rowcell[r_next] : 0;
    // alpha of chunk 0 of the first tile
    float4 av[16];
    {
      const float4* al0 = reinterpret_cast<const float4*>(args.alpha + (size_t)cell_next * W);
#pragma unroll
      for (int g = 0; g < 16; ++g) av[g] = al0[g];
    }
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const int64_t r = tile * kRT + t;
      const bool valid = r < args.R;
      const int cell = cell_next;
      // the next tile's row -> cell lookup is in flight while this tile is scaled
      r_next = (tile + gridDim.x) * kRT + t;
      cell_next = (tile + gridDim.x < ntiles && r_next < args.R) ? args.rowcell[r_next] : cell;
      for (int c = 0; c < KC; ++c, ++it) {
        const int sidx = it % NS;
        // alpha of the next chunk: this tile's chunk c + 1, else the next tile's chunk 0
        const float4* aln = (c + 1 < KC) ? reinterpret_cast<const float4*>(args.alpha + (size_t)cell * W) + 16 * (c + 1)
                                         : reinterpret_cast<const float4*>(args.alpha + (size_t)cell_next * W);
        float4 an[16];
#pragma unroll
        for (int g = 0; g < 16; ++g) an[g] = aln[g];
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
#pragma unroll
        for (int g = 0; g < 16; ++g) av[g] = an[g];
      }
    }
  } else if (warp == 5) {
    // ---- TMA producer of the row chunks ----
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        for (int c = 0; c < KC; ++c, ++it) {
          const int sidx = it % NS;
          if (!rwait(&aempty[sidx], ((it / NS) & 1) ^ 1, abort, args.status)) { ok = false; break; }
          mbar_expect_tx(&araw[sidx], (uint32_t)S::kAC);
          tma_load_2d(Asm + (size_t)sidx * S::kAC, &xmap, &araw[sidx], c * 64, (int)(tile * kRT));
        }
      }
    }
  } else if (warp == 4) {
    // ---- W_j once, then the MMAs ----
    if (lane == 0) {
      mbar_expect_tx(wfull, (uint32_t)S::kWB);
      for (int c = 0; c < KC; ++c) tma_load_2d(Wsm + (size_t)c * W * 128, &wmap, wfull, c * 64, 0);
      const uint32_t id = idesc(W);
      uint32_t it = 0, tt = 0;
      bool ok = rwait(wfull, 0, abort, args.status);
      for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++tt) {
        const uint32_t b = tt & 1;
        if (!rwait(&tempty[b], ((tt >> 1) & 1) ^ 1, abort, args.status)) break;
        tc_fence_after();
        const uint32_t dt = tmem + b * W;
        for (int c = 0; c < KC; ++c, ++it) {
          const int sidx = it % NS;
          if (!rwait(&afull[sidx], (it / NS) & 1, abort, args.status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = su32(Asm + (size_t)sidx * S::kAC), w0 = su32(Wsm + (size_t)c * W * 128);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            mma_bf16(dt, sdesc(a0 + kk * 32), sdesc(w0 + kk * 32), id, (c > 0 || kk > 0) ? 1u : 0u);
          mma_commit(&aempty[sidx]);
        }
        if (ok) mma_commit(&tfull[b]);
      }
    }
  } else {
    // ---- epilogue: TMEM -> bf16 rows of G' ----
    const int row = 32 * (warp & 3) + lane;
    uint32_t tt = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++tt) {
      const uint32_t b = tt & 1;
      // the destination row (a dependent chain of three loads) is resolved while the MMAs run
      const int64_t r = tile * kRT + row;
      const bool valid = r < args.R;
      __nv_bfloat16* dst = nullptr;
      if (valid) {
        const int cell = args.rowcell[r];
        dst = args.xout + (args.off_out[cell] + (r - args.off_in[cell])) * W;
      }
      const bool got = rwait(&tfull[b], (tt >> 1) & 1, abort, args.status);
      if (!__all_sync(0xffffffffu, got)) break;
      tc_fence_after();
      const uint32_t trow = tmem + b * W + ((uint32_t)(32 * (warp & 3)) << 16);
#pragma unroll 1
      for (int c0 = 0; c0 < W; c0 += 32) {
        float v[32];
        tmem_ld32(trow + c0, v);
        if (valid) {
          uint32_t pk[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
            pk[i] = *reinterpret_cast<const uint32_t*>(&h);
          }
          uint4* d4 = reinterpret_cast<uint4*>(dst + c0);
#pragma unroll
          for (int i = 0; i < 4; ++i) d4[i] = make_uint4(pk[4 * i], pk[4 * i + 1], pk[4 * i + 2], pk[4 * i + 3]);
        }
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(2 * W) : "memory");
  }
}

template <int W>
isx_status launch_rows_gemm_w(isx_inr inr, const RowsGemmArgs& a, const CUtensorMap& map, cudaStream_t st) {
  CUtensorMap xmap;
  ISX_TRY(tensor_map_bf16(&xmap, a.xin, W, (uint64_t)a.R, 64, kRT));
  const size_t smem = RowsSmem<W>::bytes();
  ISX_CUDA(cudaFuncSetAttribute(k_rows_gemm<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int sms = 148;
  ISX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, inr->device));
  int per_sm = 1;
  ISX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rows_gemm<W>, kGT, smem));
  per_sm = std::max(1, std::min(per_sm, 512 / (2 * W)));   // TMEM: 2 W columns per CTA
  const int64_t ntiles = (a.R + kRT - 1) / kRT;
  const int grid = (int)std::min<int64_t>(ntiles, (int64_t)sms * per_sm);
  k_rows_gemm<W><<<grid, kGT, smem, st>>>(a, map, xmap);
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
  if (w == 256) return launch_rows_gemm_w<256>(inr, a, wmap, st);
  if (w == 128) return launch_rows_gemm_w<128>(inr, a, wmap, st);
  return launch_rows_gemm_w<64>(inr, a, wmap, st);
}

}  // namespace rows
}  // namespace isx
