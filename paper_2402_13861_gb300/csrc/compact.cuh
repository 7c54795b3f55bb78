// Stable stream compaction building blocks shared by the single-INR level step (tree.cu) and the
// batched level step (batch.cu): the cull test of Algorithm 1, a block-wide rank, and the scan of
// per-block counts.
#pragma once

#include "internal.cuh"

namespace isx {
namespace compact {

constexpr int kThreads = 512;
constexpr int kPer = 4;                       // elements per thread
constexpr int kTile = kThreads * kPer;        // elements per block

// Cull test of Algorithm 1 for all iso-values at once: bit q kept iff lower <= c_q <= upper.
__device__ __forceinline__ uint32_t keep_bits(float center, float spread, const IsoSet& iso, int mode,
                                              float k, int inflate) {
  float lo, hi;
  if (sound_readout(mode)) {
    lo = inflate ? __fsub_rd(center, spread) : center - spread;
    hi = inflate ? __fadd_ru(center, spread) : center + spread;
  } else {
    float ks = k * spread;
    lo = center - ks;
    hi = center + ks;
  }
  uint32_t bits = 0;
  for (int q = 0; q < iso.n; ++q)
    if (lo <= iso.c[q] && iso.c[q] <= hi) bits |= 1u << q;
  // NaN bounds keep the cell (never cull on an undefined bound)
  if (!(lo <= hi)) bits = 0xffffffffu;
  return bits;
}

// Block-exclusive rank of `flag` among the block's threads (in thread order); returns the rank,
// writes the block total to *total.
__device__ __forceinline__ int block_rank(bool flag, int* warp_sums, int* total) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned bal = __ballot_sync(0xffffffffu, flag);
  int r = __popc(bal & ((1u << lane) - 1u));
  if (lane == 0) warp_sums[warp] = __popc(bal);
  __syncthreads();
  if (threadIdx.x < 32) {
    int v = threadIdx.x < (kThreads >> 5) ? warp_sums[threadIdx.x] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (threadIdx.x < (kThreads >> 5)) warp_sums[threadIdx.x] = incl - v;
    if (threadIdx.x == 31) *total = incl;
  }
  __syncthreads();
  int res = warp_sums[warp] + r;
  __syncthreads();
  return res;
}

// Exclusive scan of nb block counts into int64 offsets, run by one block of 1024 threads; the total
// times `scale` goes to *d_total.
__device__ __forceinline__ void scan_block_counts_dev(const int* counts, int64_t nb, int64_t* offsets,
                                                      int64_t* d_total, int64_t scale) {
  __shared__ int64_t carry;
  __shared__ int64_t wsum[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t base = 0; base < nb; base += 1024) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < nb ? counts[i] : 0;
    int64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      int64_t s = wsum[lane];
      int64_t si = s;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, si, o);
        if (lane >= o) si += t;
      }
      wsum[lane] = si - s;
    }
    __syncthreads();
    int64_t excl = carry + wsum[warp] + incl - v;
    if (i < nb) offsets[i] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) *d_total = carry * scale;
}

}  // namespace compact
}  // namespace isx
