// Internal declarations shared by the translation units of the isx library.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/isx.h"

namespace isx {

// ---- errors ------------------------------------------------------------------------------------
void set_error(const std::string& msg);
isx_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define ISX_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t _e = (call);                                                        \
    if (_e != cudaSuccess) return ::isx::cuda_fail(_e, #call, __FILE__, __LINE__);  \
  } while (0)

#define ISX_LAUNCH_CHECK(what)                                                         \
  do {                                                                                 \
    cudaError_t _e = cudaGetLastError();                                               \
    if (_e != cudaSuccess) return ::isx::cuda_fail(_e, what, __FILE__, __LINE__);      \
  } while (0)

#define ISX_TRY(expr)                        \
  do {                                       \
    isx_status _s = (expr);                  \
    if (_s != ISX_OK) return _s;             \
  } while (0)

// ---- device buffers ----------------------------------------------------------------------------
// A growable device allocation owned by an INR's workspace.
struct Buf {
  void* ptr = nullptr;
  size_t bytes = 0;
  isx_status ensure(size_t need, const char* name);
  void release();
  template <class T> T* as() const { return static_cast<T*>(ptr); }
};

// Workspace slots (one growable buffer each).
enum Slot {
  WS_CODES_A, WS_CODES_B, WS_MASK_A, WS_MASK_B, WS_CENTER, WS_SPREAD, WS_FLAGS, WS_BLOCKSUM,
  WS_COUNT, WS_C, WS_X0, WS_X1, WS_RAD, WS_ALPHA, WS_GAMMA, WS_DELTA, WS_AUX,
  WS_LATTICE_FLAG, WS_LATTICE_IDX, WS_POINTS, WS_VALUES, WS_TRI_COUNT, WS_TRI_OFFSET,
  WS_TC_SCRATCH, WS_TC_STATE, WS_TC_STATUS,
  WS_ANC_C_A, WS_ANC_C_B, WS_ANC_S_A, WS_ANC_S_B, WS_ANC_G_A, WS_ANC_G_B, WS_PROP_KEEP, WS_PROP_NEED,
  WS_PROP_IDX, WS_PROP_CODES,
  WS_R_I0, WS_R_I1, WS_R_A, WS_R_CNT0, WS_R_CNT1, WS_R_OFF0, WS_R_OFF1, WS_R_RC0, WS_R_RC1, WS_R_TOT, WS_R_AH, WS_R_ALO,
  WS_R_PART, WS_R_PNEW, WS_R_V, WS_R_D,
  WS_N_SLOTS
};

}  // namespace isx

// The opaque INR handle.
struct isx_inr_s {
  int device = 0;
  int n_layers = 0;           // linear layers = H + 1
  int H = 0;                  // hidden (activation) layers
  int w = 0;                  // hidden width
  int act = 0;                // isx_activation of the hidden layers
  // device copies, per linear layer l: W[l] row-major [out][in], Wt[l] = W[l]^T row-major [in][out]
  std::vector<float*> W, Wt, b;
  std::vector<__nv_bfloat16*> Wt_bf16;   // W[l]^T in bfloat16, for the tensor-core path
  std::vector<__nv_bfloat16*> W_bf16;    // W[l] in bfloat16 (row-major [out][in])
  std::vector<__nv_bfloat16*> Wabs_bf16; // |W[l]| in bfloat16 (row-major)
  std::vector<__nv_bfloat16*> Wsq_bf16;  // W[l]^2 in bfloat16 (row-major)
  std::vector<__nv_bfloat16*> Wlo_bf16;  // W[l] - float(W_bf16[l]) in bfloat16: low part of a two-term split
  std::vector<__nv_bfloat16*> Wperm_bf16; // W_bf16[l] with its rows in the row GEMM's order (w = 256 only)
  std::vector<__nv_bfloat16*> Wabsru_bf16; // |W[l]| rounded up to bfloat16 (row-major): the rounding-error
                                           // bound's GEMM, whose result must not fall below |W| v
  void* tc_net = nullptr;                // device network descriptor of the tensor-core bound kernel
  std::vector<float*> absW_rowsum;       // sum_k |W[l][n][k]| per output neuron
  std::vector<std::vector<float>> hW, hb;  // host copies
  isx::Buf ws[isx::WS_N_SLOTS];
  int64_t row_budget = (int64_t)1 << 24;  // symbol rows per chunk of the row-batched bound path
  float* h_pinned = nullptr;            // small pinned host buffer for count read-back
  int* h_pinned_i = nullptr;
};

namespace isx {

// ---- launch accounting (prof.cu) --------------------------------------------------------------
enum KernelId {
  K_INPUT, K_RELU, K_GEMV, K_GEMM_FP32, K_FRESH, K_REDUCE, K_OUTPUT, K_CULL, K_SCAN, K_SCATTER, K_MARK,
  K_FLAGCOUNT, K_SCATTER_FLAGS, K_EVAL_FP32, K_MC_COUNT, K_MC_EMIT, K_IOTA, K_BOUND_TC, K_TC_PREP, K_TC_OUTPUT,
  K_EVAL_TC, K_PROP_GATE, K_PROP_MERGE, K_PROP_FWD, K_PROP_GRAD, K_PROP_ADAM, K_BOUND_RAFIXED, K_ROWS_GEMM, K_ROWS_AUX,
  K_ROWS_ACT, K_ROWS_NEW, K_ROWS_SPLIT, K_ROWS_REDUCE, K_ROWS_OUT, K_COUNT
};
namespace prof {
// RAII bracket around one kernel launch: counts it, adds its algorithmic work, and (when
// profiling is enabled) records CUDA events before and after it on `st`.
class Scope {
 public:
  Scope(int kernel, cudaStream_t st, double flops = 0, double bytes = 0);
  ~Scope();
 private:
  int kernel_;
  cudaStream_t st_;
  bool active_ = false;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
};
}  // namespace prof

// ---- kernels and launchers (bound_fp32.cu) -----------------------------------------------------
// Cells given either as boxes (lo, hi) or as packed codes of one octree level.
struct CellSource {
  const float* lo = nullptr;
  const float* hi = nullptr;
  const uint32_t* codes = nullptr;
  int level = 0;                       // octree level of the codes: every axis split `level` times
  int lv[3] = {-1, -1, -1};            // k-d cells: split count per axis (lv[0] < 0: `level` for all)
};
// Split count of axis d of the codes of `s` (cells of width 2 / 2^count along d).
__host__ __device__ __forceinline__ int axis_level(const CellSource& s, int d) { return s.lv[0] < 0 ? s.level : s.lv[d]; }

// Bounds n cells in float32 with the layer-by-layer path; chunked over the workspace.
isx_status bound_fp32(isx_inr inr, const CellSource& src, int64_t n, isx_bound_mode mode,
                      int inflate, float* d_center, float* d_spread, cudaStream_t st);

// RA-Fixed bounds (input symbols kept, all others condensed per neuron), one fused float32 kernel.
isx_status bound_rafixed(isx_inr inr, const CellSource& src, int64_t n, int inflate, float* d_center,
                         float* d_spread, cudaStream_t st);
bool rafixed_supported(isx_inr inr);
// Whether the read-off of `mode` is the sound interval centre +- spread (no k).
__host__ __device__ __forceinline__ bool sound_readout(int mode) {
  return mode == ISX_BOUND_SOUND || mode == ISX_BOUND_RAFIXED;
}

// Row-batched tensor-core path: layer-synchronous over a chunk of cells, noise-symbol rows with a
// zero coefficient dropped, alpha applied on the A side so that one weight operand serves all
// cells (bound_rows.cu).  Hidden widths 64, 128 and 256; sound bounds with or without inflation.
isx_status bound_bf16_rows(isx_inr inr, const CellSource& src, int64_t n, isx_bound_mode mode, int inflate,
                           float* d_center, float* d_spread, cudaStream_t st);
bool rows_supported(isx_inr inr, isx_bound_mode mode, int inflate);

// Tensor-core (tcgen05, bfloat16) path; ISX_ERR_UNSUPPORTED for shapes it does not cover.
isx_status bound_bf16(isx_inr inr, const CellSource& src, int64_t n, isx_bound_mode mode,
                      int inflate, float* d_center, float* d_spread, cudaStream_t st);
bool bf16_supported(isx_inr inr);
// Device copy of the INR's network descriptor for the tensor-core bound kernel (built on first use).
isx_status tc_net_of(isx_inr inr, const void** out);
size_t tc_net_bytes();
// 2-D bfloat16 tensor map [outer][inner] (row stride inner * 2 bytes), 128-byte swizzle.
isx_status tensor_map_bf16(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint32_t box_inner,
                           uint32_t box_outer);
// MLP values at points on tcgen05 with two-term BF16 operands (eval_tc.cu); ISX_ERR_UNSUPPORTED for
// widths other than 128 / 256.  Points as in eval_points_fp32.
isx_status eval_points_tc(isx_inr inr, const float* xyz, const uint32_t* lattice_ids, int R, int64_t n,
                          float* out, cudaStream_t st);
bool eval_tc_supported(isx_inr inr);

// ---- octree level step (tree.cu) ---------------------------------------------------------------
struct IsoSet {
  int n = 0;
  float c[ISX_MAX_ISO];
};
// Computes the surviving iso mask of every cell and compacts survivors (stable).  If `expand`,
// writes the 8 children of every survivor (child c = 2 (i,j,k) + bits of c) with the parent's
// mask; otherwise writes the survivors themselves.  `bounded` = 0 keeps every cell with its mask.
// The number of written cells goes to *d_count (device int64).
// Ancestor bounds carried to the children (for the proposer's features): in_c / in_s / in_gap per
// input cell (in_gap == nullptr: 0, i.e. the cell itself was bounded), written with gap + 1 to
// every child; out_c == nullptr: nothing carried.
struct AncIO {
  const float* in_c = nullptr;
  const float* in_s = nullptr;
  const uint8_t* in_gap = nullptr;
  float* out_c = nullptr;
  float* out_s = nullptr;
  uint8_t* out_gap = nullptr;
};
isx_status level_step(isx_inr inr, const uint32_t* codes, const uint32_t* masks, int64_t n,
                      const float* center, const float* spread, bool bounded, const IsoSet& iso,
                      isx_bound_mode mode, float k, int inflate, bool expand, uint32_t* out_codes,
                      uint32_t* out_masks, int64_t* d_count, cudaStream_t st, const AncIO* anc = nullptr,
                      int split_axis = -1);

// Stable compaction of the indices i < n with flags[i] != 0 into out_idx; count to *d_count.
isx_status compact_flags(isx_inr inr, const uint8_t* flags, int64_t n, uint32_t* out_idx,
                         uint32_t* idx_map, int64_t* d_count, cudaStream_t st);

// Exclusive scan of nb int counts into int64 offsets (single block); total to *d_total.
isx_status scan_block_counts(isx_inr inr, const int* counts, int64_t nb, int64_t* offsets, int64_t* d_total,
                             cudaStream_t st);
// out[i] = i for i < n.
isx_status iota_u32(uint32_t* out, int64_t n, cudaStream_t st);
// out[i] = v for i < n.
isx_status fill_f32(float* out, int64_t n, float v, cudaStream_t st);

// ---- proposer (proposer.cu) ----------------------------------------------------------------------
// keep[i] = iso bits of cell i kept without a bound (logit >= z_hi), need[i] = 1 if some bit of its
// mask is undecided (z_lo < logit < z_hi); bits with logit <= z_lo are dropped.
isx_status proposer_gate(isx_proposer p, const uint32_t* codes, const uint32_t* masks, const float* anc_c,
                         const float* anc_s, const uint8_t* anc_gap, int64_t n, int level, const IsoSet& iso,
                         float z_lo, float z_hi, uint32_t* keep, uint8_t* need, cudaStream_t st);
// For the bounded cells idx[j]: keep[idx[j]] = masks[idx[j]] & cull(bound j); their bound becomes
// the ancestor bound (gap 0).
isx_status proposer_merge(const uint32_t* idx, int64_t nb, const uint32_t* masks, const float* c_sub,
                          const float* s_sub, const IsoSet& iso, isx_bound_mode mode, float k, int inflate,
                          uint32_t* keep, float* anc_c, float* anc_s, uint8_t* anc_gap, cudaStream_t st);
isx_status gather_codes(const uint32_t* codes, const uint32_t* idx, int64_t nb, uint32_t* out, cudaStream_t st);

// CUDA events bracketing the phases of one extraction (prediction, corner evaluation, marching cubes).
struct Timer {
  cudaEvent_t ev[4] = {};
  isx_status init() {
    for (auto& e : ev) ISX_CUDA(cudaEventCreate(&e));
    return ISX_OK;
  }
  ~Timer() {
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
  }
};

// Active cells -> mesh: copy to the caller, corner evaluation, marching cubes (api.cu).
isx_status mesh_from_active(isx_inr inr, const isx_extract_params* p, const uint32_t* codes, const uint32_t* masks,
                            int64_t n, isx_mesh* mesh, Timer& tm, cudaStream_t st);
// Batched level step helpers need the parameter checks of the single extraction (api.cu).
isx_status validate_extract_params(const isx_extract_params* p, const isx_mesh* m);
IsoSet iso_set_of(const isx_extract_params* p);

// ---- launch-shape autotuner (tune.cu) -------------------------------------------------------------
namespace tune {
// Variant to launch for `key` among n interchangeable ones (identical results): timed on first use
// with run(v) on stream st, cached for the process.
isx_status pick(const std::string& key, int n, const std::function<const char*(int)>& name,
                const std::function<isx_status(int)>& run, cudaStream_t st, int* out);
}  // namespace tune

// ---- mesh (mesh.cu) ----------------------------------------------------------------------------
// flags[lattice id] = 1 for the 8 corners of every listed cell of the R^3 grid.
isx_status mark_corners(const uint32_t* codes, int64_t n, int R, uint8_t* flags, cudaStream_t st);
// Marching cubes over n listed cells (codes, masks) or, with codes == nullptr, over all R^3 cells for
// every iso-value.  Corner values are values[idx_map[lattice id]] (idx_map == nullptr: by lattice id).
// Writes mesh->n_tris; emits only if it fits mesh->tri_cap (else ISX_ERR_CAPACITY).  With
// count_nonempty, mesh->n_active becomes the number of cells with at least one triangle, and those
// cells (code, mask of the isos with triangles) go to the mesh's active buffers when they fit.
isx_status marching_cubes(isx_inr inr, const uint32_t* codes, const uint32_t* masks, int64_t n, int R,
                          const uint32_t* idx_map, const float* values, const IsoSet& iso, isx_mesh* mesh,
                          bool count_nonempty, cudaStream_t st);
isx_status eval_points_fp32(isx_inr inr, const float* xyz, const uint32_t* lattice_ids, int R,
                            int64_t n, float* out, cudaStream_t st);
isx_status mc_upload_table(int device);
void mc_build_table(int8_t* ntri, int8_t* tris);

}  // namespace isx
