// Octree level step (Algorithm 1's cull / emit / split, run for a whole level at once) and the
// stable stream compaction it is built on.
//
// Compaction is three passes over blocks of kTile elements: (1) every block counts its selected
// elements; (2) one block turns the counts into exclusive offsets; (3) every block recomputes its
// selection, ranks it with warp ballots and scatters.  Output order equals input order, so the
// results do not depend on scheduling.
#include "compact.cuh"

#include <algorithm>

namespace isx {
namespace {

using namespace compact;

__global__ void __launch_bounds__(kThreads) k_cull_count(const uint32_t* masks, int64_t n, const float* center,
                                                         const float* spread, int bounded, IsoSet iso,
                                                         int mode, float k, int inflate, uint32_t* newmask,
                                                         int* block_count) {
  int64_t base = (int64_t)blockIdx.x * kTile;
  int cnt = 0;
  for (int e = 0; e < kPer; ++e) {
    int64_t i = base + e * kThreads + threadIdx.x;
    if (i < n) {
      uint32_t m = masks[i];
      if (bounded) m &= keep_bits(center[i], spread[i], iso, mode, k, inflate);
      newmask[i] = m;
      cnt += (m != 0);
    }
  }
  __shared__ int red[kThreads / 32];
  int v = cnt;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int q = 0; q < kThreads / 32; ++q) s += red[q];
    block_count[blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(kThreads) k_flag_count(const uint8_t* flags, int64_t n, int* block_count) {
  int64_t base = (int64_t)blockIdx.x * kTile;
  int cnt = 0;
  for (int e = 0; e < kPer; ++e) {
    int64_t i = base + e * kThreads + threadIdx.x;
    if (i < n) cnt += flags[i] != 0;
  }
  __shared__ int red[kThreads / 32];
  int v = cnt;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int q = 0; q < kThreads / 32; ++q) s += red[q];
    block_count[blockIdx.x] = s;
  }
}

// Exclusive scan of nb block counts into int64 offsets (one block); total to *d_total.
__global__ void __launch_bounds__(1024) k_scan_counts(const int* counts, int64_t nb, int64_t* offsets,
                                                      int64_t* d_total, int64_t scale) {
  scan_block_counts_dev(counts, nb, offsets, d_total, scale);
}

// expand: 0 writes the survivors; 1 writes their 8 octree children; with split_axis >= 0 and expand
// set, their 2 k-d children along that axis.
__global__ void __launch_bounds__(kThreads) k_scatter_cells(const uint32_t* codes, const uint32_t* newmask,
                                                            int64_t n, const int64_t* offsets, int expand,
                                                            int split_axis, uint32_t* out_codes, uint32_t* out_masks,
                                                            AncIO anc) {
  __shared__ int warp_sums[32];
  __shared__ int total;
  int64_t base = (int64_t)blockIdx.x * kTile;
  int64_t off = offsets[blockIdx.x];
  for (int e = 0; e < kPer; ++e) {
    int64_t i = base + e * kThreads + threadIdx.x;
    uint32_t m = i < n ? newmask[i] : 0u;
    bool f = m != 0;
    int r = block_rank(f, warp_sums, &total);
    if (f) {
      int64_t o = off + r;
      uint32_t code = codes[i];
      if (expand && split_axis >= 0) {
        const uint32_t sh = 10u * (uint32_t)split_axis;
        const uint32_t ca = ((code >> sh) & 1023u) << 1, rest = code & ~(1023u << sh);
        out_codes[2 * o] = rest | (ca << sh);
        out_codes[2 * o + 1] = rest | ((ca + 1u) << sh);
        out_masks[2 * o] = m;
        out_masks[2 * o + 1] = m;
      } else if (expand) {
        uint32_t ci = (code & 1023u) << 1, cj = ((code >> 10) & 1023u) << 1, ck = ((code >> 20) & 1023u) << 1;
        for (int c = 0; c < 8; ++c) {
          uint32_t cc = (ci + (c & 1)) | ((cj + ((c >> 1) & 1)) << 10) | ((ck + ((c >> 2) & 1)) << 20);
          out_codes[8 * o + c] = cc;
          out_masks[8 * o + c] = m;
        }
        if (anc.out_c) {
          const float ac = anc.in_c[i], as = anc.in_s[i];
          const int g = anc.in_gap ? anc.in_gap[i] : 0;
          const uint8_t gc = (uint8_t)min(g + 1, 255);
          for (int c = 0; c < 8; ++c) {
            anc.out_c[8 * o + c] = ac;
            anc.out_s[8 * o + c] = as;
            anc.out_gap[8 * o + c] = gc;
          }
        }
      } else {
        out_codes[o] = code;
        out_masks[o] = m;
        if (anc.out_c) {
          anc.out_c[o] = anc.in_c[i];
          anc.out_s[o] = anc.in_s[i];
          anc.out_gap[o] = anc.in_gap ? anc.in_gap[i] : 0;
        }
      }
    }
    off += total;
  }
}

__global__ void __launch_bounds__(kThreads) k_scatter_flags(const uint8_t* flags, int64_t n, const int64_t* offsets,
                                                            uint32_t* out_idx, uint32_t* idx_map) {
  __shared__ int warp_sums[32];
  __shared__ int total;
  int64_t base = (int64_t)blockIdx.x * kTile;
  int64_t off = offsets[blockIdx.x];
  for (int e = 0; e < kPer; ++e) {
    int64_t i = base + e * kThreads + threadIdx.x;
    bool f = i < n && flags[i] != 0;
    int r = block_rank(f, warp_sums, &total);
    if (f) {
      out_idx[off + r] = (uint32_t)i;
      if (idx_map) idx_map[i] = (uint32_t)(off + r);
    }
    off += total;
  }
}

__global__ void k_iota(uint32_t* out, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (uint32_t)i;
}

__global__ void k_fill_f32(float* out, int64_t n, float v) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = v;
}

}  // namespace

isx_status scan_block_counts(isx_inr, const int* counts, int64_t nb, int64_t* offsets, int64_t* d_total,
                             cudaStream_t st) {
  {
    prof::Scope _ps(K_SCAN, st, 0, 0);
    k_scan_counts<<<1, 1024, 0, st>>>(counts, nb, offsets, d_total, 1);
  }
  ISX_LAUNCH_CHECK("k_scan_counts");
  return ISX_OK;
}

isx_status iota_u32(uint32_t* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return ISX_OK;
  {
    prof::Scope _ps(K_IOTA, st, 0, 0);
    k_iota<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n);
  }
  ISX_LAUNCH_CHECK("k_iota");
  return ISX_OK;
}

isx_status fill_f32(float* out, int64_t n, float v, cudaStream_t st) {
  if (n <= 0) return ISX_OK;
  {
    prof::Scope _ps(K_IOTA, st, 0, 0);
    k_fill_f32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n, v);
  }
  ISX_LAUNCH_CHECK("k_fill_f32");
  return ISX_OK;
}

isx_status level_step(isx_inr inr, const uint32_t* codes, const uint32_t* masks, int64_t n,
                      const float* center, const float* spread, bool bounded, const IsoSet& iso,
                      isx_bound_mode mode, float k, int inflate, bool expand, uint32_t* out_codes,
                      uint32_t* out_masks, int64_t* d_count, cudaStream_t st, const AncIO* anc, int split_axis) {
  if (n == 0) {
    ISX_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int64_t), st));
    return ISX_OK;
  }
  int64_t nb = (n + kTile - 1) / kTile;
  auto& ws = inr->ws;
  ISX_TRY(ws[WS_FLAGS].ensure((size_t)n * sizeof(uint32_t), "newmask"));
  size_t head = ((nb * sizeof(int) + 15) / 16) * 16;
  ISX_TRY(ws[WS_BLOCKSUM].ensure(head + nb * sizeof(int64_t), "block sums"));
  int* bc = ws[WS_BLOCKSUM].as<int>();
  int64_t* boff = reinterpret_cast<int64_t*>(ws[WS_BLOCKSUM].as<char>() + head);
  uint32_t* nm = ws[WS_FLAGS].as<uint32_t>();
  {
    prof::Scope _ps(K_CULL, st, 0, 0);
    k_cull_count<<<(unsigned)nb, kThreads, 0, st>>>(masks, n, center, spread, bounded ? 1 : 0, iso, (int)mode, k,
                                                    inflate, nm, bc);
  }
  ISX_LAUNCH_CHECK("k_cull_count");
  {
    prof::Scope _ps(K_SCAN, st, 0, 0);
    k_scan_counts<<<1, 1024, 0, st>>>(bc, nb, boff, d_count, expand ? (split_axis >= 0 ? 2 : 8) : 1);
  }
  ISX_LAUNCH_CHECK("k_scan_counts");
  {
    prof::Scope _ps(K_SCATTER, st, 0, 0);
    k_scatter_cells<<<(unsigned)nb, kThreads, 0, st>>>(codes, nm, n, boff, expand ? 1 : 0, split_axis, out_codes,
                                                       out_masks, anc ? *anc : AncIO());
  }
  ISX_LAUNCH_CHECK("k_scatter_cells");
  return ISX_OK;
}

isx_status compact_flags(isx_inr inr, const uint8_t* flags, int64_t n, uint32_t* out_idx, uint32_t* idx_map,
                         int64_t* d_count, cudaStream_t st) {
  if (n == 0) {
    ISX_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int64_t), st));
    return ISX_OK;
  }
  int64_t nb = (n + kTile - 1) / kTile;
  auto& ws = inr->ws;
  size_t head = ((nb * sizeof(int) + 15) / 16) * 16;
  ISX_TRY(ws[WS_BLOCKSUM].ensure(head + nb * sizeof(int64_t), "block sums"));
  int* bc = ws[WS_BLOCKSUM].as<int>();
  int64_t* boff = reinterpret_cast<int64_t*>(ws[WS_BLOCKSUM].as<char>() + head);
  {
    prof::Scope _ps(K_FLAGCOUNT, st, 0, 0);
    k_flag_count<<<(unsigned)nb, kThreads, 0, st>>>(flags, n, bc);
  }
  ISX_LAUNCH_CHECK("k_flag_count");
  {
    prof::Scope _ps(K_SCAN, st, 0, 0);
    k_scan_counts<<<1, 1024, 0, st>>>(bc, nb, boff, d_count, 1);
  }
  ISX_LAUNCH_CHECK("k_scan_counts");
  {
    prof::Scope _ps(K_SCATTER_FLAGS, st, 0, 0);
    k_scatter_flags<<<(unsigned)nb, kThreads, 0, st>>>(flags, n, boff, out_idx, idx_map);
  }
  ISX_LAUNCH_CHECK("k_scatter_flags");
  return ISX_OK;
}

}  // namespace isx
