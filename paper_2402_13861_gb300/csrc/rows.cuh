// Shared pieces of the row-batched tensor-core bound path (bound_rows.cu, rows_gemm.cu): the tile
// shape, the swizzled A-tile layout, the bounded mbarrier wait and the row GEMM's interface.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace isx {
namespace rows {

constexpr int kRT = 128;                        // rows per MMA tile
constexpr int kPT = 64;                         // rows per column-sum slot (half a tile)
constexpr uint64_t kRowsWaitNs = 2000000000ull;

struct RowsGemmArgs {
  const __nv_bfloat16* xin;                     // [R][W] rows of z_j
  const int* rowcell;                           // [R] cell of every row
  const int64_t* off_in;                        // [nc] first row of each cell in xin
  const int64_t* off_out;                       // [nc] first row of each cell in xout
  const float* alpha;                           // [nc][W]
  int64_t R;
  __nv_bfloat16* xout;                          // [R'][W] rows of z_{j+1}
  float* part;                                  // [nc + ceil(R / 64)][W]: slot cell + t holds, per neuron,
                                                // sum f(x) over the cell's rows among input rows
                                                // 64 t .. 64 t + 63
  int sq;                                       // f(x) = x^2 (1, Eq. 7) or |x| (0, Eq. 2)
  int* status;
};

__device__ __forceinline__ uint32_t roff(int row, int k) {  // byte offset of (row, k..k+7) in an A tile
  return (uint32_t)((k >> 6) * kRT * 128 + row * 128 + ((((k & 63) >> 3) ^ (row & 7)) << 4));
}

// Bounded wait for phase `parity` of mbarrier b: gives up when another role of the CTA raised
// *abort, or after limit_ns, in which case it raises *abort and records ISX_ERR_TIMEOUT in *status.
__device__ __forceinline__ bool rwait(uint64_t* b, uint32_t parity, volatile int* abort, int* status,
                                      uint64_t limit_ns = kRowsWaitNs) {
  if (tc::mbar_try(b, parity)) return true;
  const uint64_t t0 = tc::global_ns();
  for (uint32_t it = 1;; ++it) {
    if (tc::mbar_try(b, parity)) return true;
    if ((it & 3) == 0) {
      if (*abort) return false;
      if (tc::global_ns() - t0 > limit_ns) {
        *abort = 1;
        atomicExch(status, (int)ISX_ERR_TIMEOUT);
        return false;
      }
    }
  }
}

// G' = (G diag(alpha_cell)) W_j^T for the R rows of `a`, and the per-(cell, 64-row block) column
// sums of f(G') (rows_gemm.cu); w = 64, 128, 256 or 512, `wmap` the tensor map of W_j in bf16 with
// box {64, w} (box {64, 128} at w = 512: a CTA holds a 128-row quarter), its rows in the order of
// rows_weight_row (the neuron held by MMA row m).
isx_status launch_rows_gemm(isx_inr inr, const RowsGemmArgs& a, const CUtensorMap& wmap, int w, cudaStream_t st);
// Row of W_j the row GEMM keeps at position m of its weight operand.  For w = 256 the even neurons
// come first and the odd ones after them, so that the epilogue thread of MMA row m of the two
// 128-row halves holds the neuron pair (2m, 2m + 1); otherwise the identity.
__host__ __device__ __forceinline__ int rows_weight_row(int m, int w) {
  return w == 256 ? (m < 128 ? 2 * m : 2 * (m - 128) + 1) : m;
}
// Slot of the column partials of (cell, 64-row block t of the input rows) in RowsGemmArgs::part:
// cell + t.  Rows of a cell are contiguous, so cell c < c' implies t <= t' and the slots of all
// (cell, block) pairs that share rows are distinct.
__host__ __device__ __forceinline__ int64_t rows_part_slot(int64_t cell, int64_t t) { return cell + t; }
// One CTA waits on an mbarrier that nothing completes, with rwait and the given limit, raising
// ISX_ERR_TIMEOUT in *d_status (rows_gemm.cu).
isx_status check_bounded_wait(int64_t limit_ns, int* d_status, cudaStream_t st);

}  // namespace rows
}  // namespace isx
