// The C interface (include/isx.h): INR handles, workspace, and the host-side driver of the level
// loop of Algorithm 1 followed by corner queries and marching cubes.
#include "internal.cuh"
#include "rows.cuh"

#include <cstdlib>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

namespace isx {

namespace {
thread_local std::string g_err;
}

void set_error(const std::string& msg) { g_err = msg; }

isx_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  std::snprintf(buf, sizeof(buf), "CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file,
                line);
  g_err = buf;
  if (e == cudaErrorMemoryAllocation) return ISX_ERR_NOMEM;
  return ISX_ERR_CUDA;
}

isx_status Buf::ensure(size_t need, const char* name) {
  if (need <= bytes) return ISX_OK;
  if (ptr) {
    cudaError_t e = cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
    if (e != cudaSuccess) return cuda_fail(e, name, __FILE__, __LINE__);
  }
  size_t alloc = std::max<size_t>(need + need / 8, 4096);
  alloc = (alloc + 255) & ~size_t(255);
  cudaError_t e = cudaMalloc(&ptr, alloc);
  if (e != cudaSuccess) {
    ptr = nullptr;
    (void)cudaGetLastError();
    return cuda_fail(e, name, __FILE__, __LINE__);
  }
  bytes = alloc;
  return ISX_OK;
}

void Buf::release() {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
}

namespace {

// The smallest bfloat16 >= x, for finite x >= 0.
__nv_bfloat16 bf16_round_up(float x) {
  __nv_bfloat16 b = __float2bfloat16_rn(x);
  if (__bfloat162float(b) < x) {
    uint16_t bits;
    std::memcpy(&bits, &b, 2);
    ++bits;
    std::memcpy(&b, &bits, 2);
  }
  return b;
}

isx_status check_inr(isx_inr inr) {
  if (!inr) {
    set_error("null INR handle");
    return ISX_ERR_ARG;
  }
  int dev = -1;
  ISX_CUDA(cudaGetDevice(&dev));
  if (dev != inr->device) {
    set_error("the INR was created on another device than the current one");
    return ISX_ERR_ARG;
  }
  return ISX_OK;
}

isx_status bound_dispatch(isx_inr inr, const CellSource& src, int64_t n, isx_bound_mode mode, isx_precision prec,
                          int inflate, float* center, float* spread, cudaStream_t st) {
  if (inr->act != ISX_ACT_RELU && mode != ISX_BOUND_CLT) {
    set_error("ELU and sine networks are bounded by uncertainty propagation (ISX_BOUND_CLT) only");
    return ISX_ERR_UNSUPPORTED;
  }
  if (mode == ISX_BOUND_RAFIXED) {
    if (prec != ISX_PREC_FP32) {
      set_error("RA-Fixed bounds are computed in float32 only");
      return ISX_ERR_UNSUPPORTED;
    }
    return bound_rafixed(inr, src, n, inflate, center, spread, st);
  }
  if (prec == ISX_PREC_BF16) {
    // one rule, no switch: the row-batched tensor-core path wherever it applies (hidden widths 64,
    // 128, 256), the per-cell tensor-core kernel for the shapes it alone covers
    if (rows_supported(inr, mode, inflate)) return bound_bf16_rows(inr, src, n, mode, inflate, center, spread, st);
    return bound_bf16(inr, src, n, mode, inflate, center, spread, st);
  }
  return bound_fp32(inr, src, n, mode, inflate, center, spread, st);
}


isx_status validate_params(const isx_extract_params* p, const isx_mesh* m) {
  if (!p || !m) {
    set_error("null params or mesh");
    return ISX_ERR_ARG;
  }
  if (p->max_level < 0 || p->max_level > ISX_MAX_LEVEL) {
    set_error("max_level must be in [0, 10]");
    return ISX_ERR_ARG;
  }
  if (p->n_iso < 1 || p->n_iso > ISX_MAX_ISO) {
    set_error("n_iso must be in [1, 32]");
    return ISX_ERR_ARG;
  }
  if (p->mode < ISX_BOUND_SOUND || p->mode > ISX_BOUND_RAFIXED || p->prec < ISX_PREC_FP32 || p->prec > ISX_PREC_BF16) {
    set_error("bad mode or precision");
    return ISX_ERR_ARG;
  }
  if (!(p->k >= 0.0f) && !sound_readout(p->mode)) {
    set_error("k must be >= 0");
    return ISX_ERR_ARG;
  }
  if (p->eval_prec < ISX_PREC_FP32 || p->eval_prec > ISX_PREC_BF16) {
    set_error("bad evaluation precision");
    return ISX_ERR_ARG;
  }
  if (p->mode == ISX_BOUND_RAFIXED && p->prec != ISX_PREC_FP32) {
    set_error("RA-Fixed bounds are computed in float32 only");
    return ISX_ERR_UNSUPPORTED;
  }
  if (p->kd_tree && p->proposer) {
    set_error("the k-d mode does not take a proposer");
    return ISX_ERR_UNSUPPORTED;
  }
  if (p->record && (p->kd_tree || p->proposer)) {
    set_error("the level record covers octree extraction without a proposer only");
    return ISX_ERR_UNSUPPORTED;
  }
  if (p->record && p->record->cap > 0 &&
      (!p->record->d_code || !p->record->d_mask || !p->record->d_center || !p->record->d_spread)) {
    set_error("null level-record buffer");
    return ISX_ERR_ARG;
  }
  if (p->proposer && !(p->tau_lo >= 0.0f && p->tau_lo < p->tau_hi && p->tau_hi <= 1.0f)) {
    set_error("proposer thresholds must satisfy 0 <= tau_lo < tau_hi <= 1");
    return ISX_ERR_ARG;
  }
  return ISX_OK;
}

// Lattice-point evaluation in the requested precision.
isx_status eval_dispatch(isx_inr inr, isx_precision prec, const uint32_t* ids, int R, int64_t n, float* out,
                         cudaStream_t st) {
  if (prec == ISX_PREC_BF16) return eval_points_tc(inr, nullptr, ids, R, n, out, st);
  return eval_points_fp32(inr, nullptr, ids, R, n, out, st);
}

// Logit of a probability threshold (0 -> -inf, 1 -> +inf).
float logit_of(float p) {
  if (p <= 0.0f) return -INFINITY;
  if (p >= 1.0f) return INFINITY;
  return std::log(p / (1.0f - p));
}

IsoSet iso_of(const isx_extract_params* p) {
  IsoSet s;
  s.n = p->n_iso;
  for (int q = 0; q < ISX_MAX_ISO; ++q) s.c[q] = q < p->n_iso ? p->iso[q] : 0.0f;
  return s;
}

}  // namespace
}  // namespace isx

using namespace isx;

namespace isx {
isx_status validate_extract_params(const isx_extract_params* p, const isx_mesh* m) { return validate_params(p, m); }
IsoSet iso_set_of(const isx_extract_params* p) { return iso_of(p); }

// Active cells -> mesh (Sec. IV-D): copies the active list to the caller's buffers, evaluates the
// distinct lattice corners of the active cells and runs marching cubes in them.  `codes` / `masks`
// hold n cells of level p->max_level; timer event 0 was recorded by the caller.
isx_status mesh_from_active(isx_inr inr, const isx_extract_params* p, const uint32_t* codes, const uint32_t* masks,
                            int64_t n, isx_mesh* mesh, Timer& tm, cudaStream_t st) {
  const int R = 1 << p->max_level;
  const IsoSet iso = iso_of(p);
  auto& ws = inr->ws;
  ISX_TRY(ws[WS_COUNT].ensure(64, "count"));
  int64_t* d_count = ws[WS_COUNT].as<int64_t>();
  ISX_CUDA(cudaEventRecord(tm.ev[1], st));
  mesh->n_active = n;
  if (n > mesh->active_cap) {
    set_error("active-cell capacity exceeded");
    return ISX_ERR_CAPACITY;
  }
  if (n > 0) {
    if (!mesh->d_active_code || !mesh->d_active_mask) {
      set_error("null active-cell output buffer");
      return ISX_ERR_ARG;
    }
    ISX_CUDA(cudaMemcpyAsync(mesh->d_active_code, codes, n * 4, cudaMemcpyDeviceToDevice, st));
    ISX_CUDA(cudaMemcpyAsync(mesh->d_active_mask, masks, n * 4, cudaMemcpyDeviceToDevice, st));
  }
  // distinct corners of the active cells
  int64_t nlat = (int64_t)(R + 1) * (R + 1) * (R + 1);
  ISX_TRY(ws[WS_LATTICE_FLAG].ensure((size_t)nlat, "lattice flags"));
  ISX_TRY(ws[WS_LATTICE_IDX].ensure((size_t)nlat * 4, "lattice map"));
  ISX_CUDA(cudaMemsetAsync(ws[WS_LATTICE_FLAG].ptr, 0, (size_t)nlat, st));
  ISX_TRY(mark_corners(codes, n, R, ws[WS_LATTICE_FLAG].as<uint8_t>(), st));
  int64_t npts_cap = std::min<int64_t>(nlat, 8 * std::max<int64_t>(n, 1));
  ISX_TRY(ws[WS_POINTS].ensure((size_t)npts_cap * 4, "points"));
  ISX_TRY(compact_flags(inr, ws[WS_LATTICE_FLAG].as<uint8_t>(), nlat, ws[WS_POINTS].as<uint32_t>(),
                        ws[WS_LATTICE_IDX].as<uint32_t>(), d_count, st));
  int64_t npts = 0;
  ISX_CUDA(cudaMemcpyAsync(&npts, d_count, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  ISX_CUDA(cudaStreamSynchronize(st));
  mesh->n_points = npts;
  ISX_TRY(ws[WS_VALUES].ensure((size_t)std::max<int64_t>(npts, 1) * 4, "values"));
  ISX_TRY(eval_dispatch(inr, p->eval_prec, ws[WS_POINTS].as<uint32_t>(), R, npts, ws[WS_VALUES].as<float>(), st));
  ISX_CUDA(cudaEventRecord(tm.ev[2], st));
  isx_status s = marching_cubes(inr, codes, masks, n, R, ws[WS_LATTICE_IDX].as<uint32_t>(),
                                ws[WS_VALUES].as<float>(), iso, mesh, false, st);
  ISX_CUDA(cudaEventRecord(tm.ev[3], st));
  ISX_CUDA(cudaEventSynchronize(tm.ev[3]));
  cudaEventElapsedTime(&mesh->ms_acp, tm.ev[0], tm.ev[1]);
  cudaEventElapsedTime(&mesh->ms_inr, tm.ev[1], tm.ev[2]);
  cudaEventElapsedTime(&mesh->ms_mc, tm.ev[2], tm.ev[3]);
  cudaEventElapsedTime(&mesh->ms_total, tm.ev[0], tm.ev[3]);
  return s;
}
}  // namespace isx

extern "C" {

const char* isx_last_error(void) { return g_err.c_str(); }

int isx_version(void) { return 100; }

isx_status isx_mc_table(int8_t* ntri, int8_t* tris) {
  if (!ntri || !tris) {
    set_error("null table pointer");
    return ISX_ERR_ARG;
  }
  mc_build_table(ntri, tris);
  return ISX_OK;
}

isx_status isx_create_inr(const isx_inr_desc* d, isx_inr* out) {
  if (!d || !out || !d->dims || !d->W || !d->b) {
    set_error("null descriptor field");
    return ISX_ERR_ARG;
  }
  *out = nullptr;
  int L = d->n_layers;
  if (L < 2 || L > ISX_MAX_LAYERS) {
    set_error("n_layers must be in [2, 16]");
    return ISX_ERR_ARG;
  }
  if (d->dims[0] != 3 || d->dims[L] != 1) {
    set_error("dims must start with 3 and end with 1");
    return ISX_ERR_ARG;
  }
  int w = d->dims[1];
  for (int l = 1; l < L; ++l)
    if (d->dims[l] != w) {
      set_error("hidden widths must be equal");
      return ISX_ERR_ARG;
    }
  if (w < 16 || w > 512 || w % 16 != 0) {
    set_error("hidden width must be a multiple of 16 in [16, 512]");
    return ISX_ERR_UNSUPPORTED;
  }
  if (d->activation < ISX_ACT_RELU || d->activation > ISX_ACT_SINE) {
    set_error("unknown activation");
    return ISX_ERR_ARG;
  }
  for (int l = 0; l < L; ++l)
    if (!d->W[l] || !d->b[l]) {
      set_error("null weight pointer");
      return ISX_ERR_ARG;
    }
  int dev = -1;
  ISX_CUDA(cudaGetDevice(&dev));
  isx_inr inr = new isx_inr_s();
  inr->device = dev;
  inr->n_layers = L;
  inr->H = L - 1;
  inr->w = w;
  inr->act = d->activation;
  inr->W.assign(L, nullptr);
  inr->Wt.assign(L, nullptr);
  inr->b.assign(L, nullptr);
  inr->Wt_bf16.assign(L, nullptr);
  inr->W_bf16.assign(L, nullptr);
  inr->Wabs_bf16.assign(L, nullptr);
  inr->Wsq_bf16.assign(L, nullptr);
  inr->Wlo_bf16.assign(L, nullptr);
  inr->Wperm_bf16.assign(L, nullptr);
  inr->Wabsru_bf16.assign(L, nullptr);
  inr->absW_rowsum.assign(L, nullptr);
  inr->hW.resize(L);
  inr->hb.resize(L);
  auto fail = [&](isx_status s) {
    isx_destroy_inr(inr);
    return s;
  };
  for (int l = 0; l < L; ++l) {
    int fi = d->dims[l], fo = d->dims[l + 1];
    inr->hW[l].assign(d->W[l], d->W[l] + (size_t)fi * fo);
    inr->hb[l].assign(d->b[l], d->b[l] + fo);
    std::vector<float> t((size_t)fi * fo);
    std::vector<__nv_bfloat16> tb((size_t)fi * fo), rb((size_t)fi * fo), ab((size_t)fi * fo), sb((size_t)fi * fo),
        lb((size_t)fi * fo), ub((size_t)fi * fo);
    for (int o = 0; o < fo; ++o)
      for (int i = 0; i < fi; ++i) {
        const float x = d->W[l][(size_t)o * fi + i];
        t[(size_t)i * fo + o] = x;
        tb[(size_t)i * fo + o] = __float2bfloat16_rn(x);
        rb[(size_t)o * fi + i] = __float2bfloat16_rn(x);
        lb[(size_t)o * fi + i] = __float2bfloat16_rn(x - __bfloat162float(rb[(size_t)o * fi + i]));
        ab[(size_t)o * fi + i] = __float2bfloat16_rn(std::fabs(x));
        ub[(size_t)o * fi + i] = bf16_round_up(std::fabs(x));
        sb[(size_t)o * fi + i] = __float2bfloat16_rn(x * x);
      }
    size_t bytes = (size_t)fi * fo * sizeof(float);
    cudaError_t e;
    if ((e = cudaMalloc(&inr->W[l], bytes)) != cudaSuccess) return fail(cuda_fail(e, "W", __FILE__, __LINE__));
    if ((e = cudaMalloc(&inr->Wt[l], bytes)) != cudaSuccess) return fail(cuda_fail(e, "Wt", __FILE__, __LINE__));
    if ((e = cudaMalloc(&inr->b[l], fo * sizeof(float))) != cudaSuccess)
      return fail(cuda_fail(e, "b", __FILE__, __LINE__));
    if ((e = cudaMalloc(&inr->Wt_bf16[l], (size_t)fi * fo * 2)) != cudaSuccess)
      return fail(cuda_fail(e, "Wt bf16", __FILE__, __LINE__));
    if ((e = cudaMalloc(&inr->W_bf16[l], (size_t)fi * fo * 2)) != cudaSuccess)
      return fail(cuda_fail(e, "W bf16", __FILE__, __LINE__));
    if ((e = cudaMemcpy(inr->W_bf16[l], rb.data(), (size_t)fi * fo * 2, cudaMemcpyHostToDevice)) != cudaSuccess)
      return fail(cuda_fail(e, "W bf16 copy", __FILE__, __LINE__));
    if (fi == 256 && fo == 256) {
      // the row GEMM's weight operand: row m holds neuron rows_weight_row(m)
      std::vector<__nv_bfloat16> pb((size_t)fi * fo);
      for (int m = 0; m < fo; ++m) {
        const int o = rows::rows_weight_row(m, fo);
        for (int i = 0; i < fi; ++i) pb[(size_t)m * fi + i] = rb[(size_t)o * fi + i];
      }
      if ((e = cudaMalloc(&inr->Wperm_bf16[l], (size_t)fi * fo * 2)) != cudaSuccess ||
          (e = cudaMemcpy(inr->Wperm_bf16[l], pb.data(), (size_t)fi * fo * 2, cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(cuda_fail(e, "permuted W bf16", __FILE__, __LINE__));
    }
    if ((e = cudaMalloc(&inr->Wabsru_bf16[l], (size_t)fi * fo * 2)) != cudaSuccess ||
        (e = cudaMemcpy(inr->Wabsru_bf16[l], ub.data(), (size_t)fi * fo * 2, cudaMemcpyHostToDevice)) != cudaSuccess)
      return fail(cuda_fail(e, "|W| bf16 rounded up", __FILE__, __LINE__));
    if ((e = cudaMalloc(&inr->Wlo_bf16[l], (size_t)fi * fo * 2)) != cudaSuccess ||
        (e = cudaMemcpy(inr->Wlo_bf16[l], lb.data(), (size_t)fi * fo * 2, cudaMemcpyHostToDevice)) != cudaSuccess)
      return fail(cuda_fail(e, "W low bf16", __FILE__, __LINE__));
    if ((e = cudaMalloc(&inr->Wabs_bf16[l], (size_t)fi * fo * 2)) != cudaSuccess ||
        (e = cudaMalloc(&inr->Wsq_bf16[l], (size_t)fi * fo * 2)) != cudaSuccess)
      return fail(cuda_fail(e, "|W| / W^2 bf16", __FILE__, __LINE__));
    if ((e = cudaMemcpy(inr->Wabs_bf16[l], ab.data(), (size_t)fi * fo * 2, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(inr->Wsq_bf16[l], sb.data(), (size_t)fi * fo * 2, cudaMemcpyHostToDevice)) != cudaSuccess)
      return fail(cuda_fail(e, "|W| / W^2 bf16 copy", __FILE__, __LINE__));
    if ((e = cudaMemcpy(inr->W[l], d->W[l], bytes, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(inr->Wt[l], t.data(), bytes, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(inr->b[l], d->b[l], fo * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(inr->Wt_bf16[l], tb.data(), (size_t)fi * fo * 2, cudaMemcpyHostToDevice)) != cudaSuccess)
      return fail(cuda_fail(e, "weight copy", __FILE__, __LINE__));
  }
  if (bf16_supported(inr)) {
    const void* net = nullptr;
    isx_status st = tc_net_of(inr, &net);
    if (st != ISX_OK) return fail(st);
  }
  *out = inr;
  return ISX_OK;
}

isx_status isx_destroy_inr(isx_inr inr) {
  if (!inr) return ISX_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(inr->device);
  for (auto* p : inr->W) if (p) cudaFree(p);
  for (auto* p : inr->Wt) if (p) cudaFree(p);
  for (auto* p : inr->b) if (p) cudaFree(p);
  for (auto* p : inr->Wt_bf16) if (p) cudaFree(p);
  for (auto* p : inr->W_bf16) if (p) cudaFree(p);
  for (auto* p : inr->Wabs_bf16) if (p) cudaFree(p);
  for (auto* p : inr->Wsq_bf16) if (p) cudaFree(p);
  for (auto* p : inr->Wlo_bf16) if (p) cudaFree(p);
  for (auto* p : inr->Wperm_bf16) if (p) cudaFree(p);
  for (auto* p : inr->Wabsru_bf16) if (p) cudaFree(p);
  if (inr->tc_net) cudaFree(inr->tc_net);
  for (auto* p : inr->absW_rowsum) if (p) cudaFree(p);
  for (auto& buf : inr->ws) buf.release();
  if (prev >= 0) cudaSetDevice(prev);
  delete inr;
  return ISX_OK;
}

isx_status isx_bound_cells(isx_inr inr, const float* d_lo, const float* d_hi, int64_t n, isx_bound_mode mode,
                           isx_precision prec, int inflate, float* d_center, float* d_spread, void* stream) {
  ISX_TRY(check_inr(inr));
  if (n < 0 || (n > 0 && (!d_lo || !d_hi || !d_center || !d_spread))) {
    set_error("bad size or null pointer");
    return ISX_ERR_ARG;
  }
  if (mode < ISX_BOUND_SOUND || mode > ISX_BOUND_RAFIXED || prec < ISX_PREC_FP32 || prec > ISX_PREC_BF16) {
    set_error("bad mode or precision");
    return ISX_ERR_ARG;
  }
  if (n == 0) return ISX_OK;
  CellSource src;
  src.lo = d_lo;
  src.hi = d_hi;
  return bound_dispatch(inr, src, n, mode, prec, inflate, d_center, d_spread, (cudaStream_t)stream);
}

isx_status isx_eval_points(isx_inr inr, const float* d_xyz, int64_t n, isx_precision prec, float* d_out,
                           void* stream) {
  ISX_TRY(check_inr(inr));
  if (n < 0 || (n > 0 && (!d_xyz || !d_out))) {
    set_error("bad size or null pointer");
    return ISX_ERR_ARG;
  }
  if (prec == ISX_PREC_BF16) return eval_points_tc(inr, d_xyz, nullptr, 0, n, d_out, (cudaStream_t)stream);
  if (prec != ISX_PREC_FP32) {
    set_error("bad precision");
    return ISX_ERR_ARG;
  }
  return eval_points_fp32(inr, d_xyz, nullptr, 0, n, d_out, (cudaStream_t)stream);
}

isx_status isx_extract_isosurface(isx_inr inr, const isx_extract_params* p, isx_mesh* mesh, void* stream) {
  ISX_TRY(check_inr(inr));
  ISX_TRY(validate_params(p, mesh));
  cudaStream_t st = (cudaStream_t)stream;
  if (p->prec == ISX_PREC_BF16 && !bf16_supported(inr) && !rows_supported(inr, p->mode, p->inflate)) {
    set_error("BF16 propagation is not available for this width");
    return ISX_ERR_UNSUPPORTED;
  }
  const int L = p->max_level;
  const IsoSet iso = iso_of(p);
  const int stop = (p->bound_stop_level < 0 || p->bound_stop_level >= L) ? L : p->bound_stop_level;
  for (int l = 0; l <= ISX_MAX_LEVEL; ++l) mesh->cells_bounded[l] = mesh->cells_kept[l] = mesh->cells_visited[l] = 0;
  mesh->n_active = mesh->n_tris = mesh->n_points = 0;
  // learned proposal: levels >= plevel (and <= stop) are gated; their ancestors' bounds are carried
  const bool use_prop = p->proposer != nullptr;
  const int plevel = use_prop ? std::max(1, p->proposer_level) : L + 1;
  const float z_lo = use_prop ? logit_of(p->tau_lo) : 0.0f, z_hi = use_prop ? logit_of(p->tau_hi) : 0.0f;
  Timer tm;
  ISX_TRY(tm.init());
  ISX_CUDA(cudaEventRecord(tm.ev[0], st));
  auto& ws = inr->ws;
  ISX_TRY(ws[WS_CODES_A].ensure(64, "codes"));
  ISX_TRY(ws[WS_MASK_A].ensure(64, "masks"));
  ISX_TRY(ws[WS_COUNT].ensure(64, "count"));
  uint32_t root[2] = {0u, (iso.n >= 32) ? 0xffffffffu : ((1u << iso.n) - 1u)};
  ISX_CUDA(cudaMemcpyAsync(ws[WS_CODES_A].ptr, &root[0], 4, cudaMemcpyHostToDevice, st));
  ISX_CUDA(cudaMemcpyAsync(ws[WS_MASK_A].ptr, &root[1], 4, cudaMemcpyHostToDevice, st));
  int64_t* d_count = ws[WS_COUNT].as<int64_t>();
  int64_t n = 1;
  Slot ca = WS_CODES_A, cb = WS_CODES_B, ma = WS_MASK_A, mb = WS_MASK_B;
  if (p->kd_tree) {
    // Algorithm 1 literally: depth d bisects axis d mod 3 (the widest side, x before y before z);
    // per-axis split counts at depth d are ceil(d/3), ceil((d-1)/3), floor(d/3)
    const int D = 3 * L, stop_d = 3 * stop;
    for (int depth = 0; depth <= D; ++depth) {
      const bool bounded = depth <= stop_d;
      const bool expand = depth < D;
      const int lvl = (depth + 2) / 3;                // octree level the statistics are filed under
      mesh->cells_visited[lvl] += n;
      if (bounded) mesh->cells_bounded[lvl] += n;
      if (n > 0) {
        ISX_TRY(ws[WS_CENTER].ensure((size_t)n * 4, "center"));
        ISX_TRY(ws[WS_SPREAD].ensure((size_t)n * 4, "spread"));
        if (bounded) {
          CellSource src;
          src.codes = ws[ca].as<uint32_t>();
          src.level = depth / 3;
          src.lv[0] = (depth + 2) / 3;
          src.lv[1] = (depth + 1) / 3;
          src.lv[2] = depth / 3;
          ISX_TRY(bound_dispatch(inr, src, n, p->mode, p->prec, p->inflate, ws[WS_CENTER].as<float>(),
                                 ws[WS_SPREAD].as<float>(), st));
        }
        size_t need = (size_t)(expand ? 2 : 1) * n * 4;
        ISX_TRY(ws[cb].ensure(need, "codes"));
        ISX_TRY(ws[mb].ensure(need, "masks"));
      }
      ISX_TRY(level_step(inr, ws[ca].as<uint32_t>(), ws[ma].as<uint32_t>(), n, ws[WS_CENTER].as<float>(),
                         ws[WS_SPREAD].as<float>(), bounded, iso, p->mode, p->k, p->inflate, expand,
                         ws[cb].as<uint32_t>(), ws[mb].as<uint32_t>(), d_count, st, nullptr, depth % 3));
      int64_t cnt = 0;
      ISX_CUDA(cudaMemcpyAsync(&cnt, d_count, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
      ISX_CUDA(cudaStreamSynchronize(st));
      mesh->cells_kept[lvl] += expand ? cnt / 2 : cnt;
      std::swap(ca, cb);
      std::swap(ma, mb);
      n = cnt;
    }
    return mesh_from_active(inr, p, ws[ca].as<uint32_t>(), ws[ma].as<uint32_t>(), n, mesh, tm, st);
  }
  Slot aca = WS_ANC_C_A, acb = WS_ANC_C_B, asa = WS_ANC_S_A, asb = WS_ANC_S_B, aga = WS_ANC_G_A, agb = WS_ANC_G_B;
  isx_level_record* rec = p->record;
  bool rec_short = false;
  if (rec)
    for (int l = 0; l <= ISX_MAX_LEVEL + 1; ++l) rec->level_off[l] = 0;
  for (int level = 0; level <= L; ++level) {
    const bool bounded = level <= stop;
    const bool expand = level < L;
    const bool gated = use_prop && bounded && level >= plevel;
    const bool carry = use_prop && expand && level + 1 >= plevel && level + 1 <= stop;
    mesh->cells_visited[level] = n;
    mesh->cells_bounded[level] = bounded ? n : 0;
    const uint32_t* step_masks = ws[ma].as<uint32_t>();
    bool step_bounded = bounded;
    AncIO anc;
    if (n > 0) {
      ISX_TRY(ws[WS_CENTER].ensure((size_t)n * 4, "center"));
      ISX_TRY(ws[WS_SPREAD].ensure((size_t)n * 4, "spread"));
      if (gated) {
        // proposer first; the undecided cells are compacted and bounded, and their bound decides
        ISX_TRY(ws[WS_PROP_KEEP].ensure((size_t)n * 4, "proposer keep"));
        ISX_TRY(ws[WS_PROP_NEED].ensure((size_t)n, "proposer need"));
        ISX_TRY(ws[WS_PROP_IDX].ensure((size_t)n * 4, "proposer index"));
        ISX_TRY(ws[WS_PROP_CODES].ensure((size_t)n * 4, "proposer codes"));
        uint32_t* keep = ws[WS_PROP_KEEP].as<uint32_t>();
        ISX_TRY(proposer_gate(p->proposer, ws[ca].as<uint32_t>(), ws[ma].as<uint32_t>(), ws[aca].as<float>(),
                              ws[asa].as<float>(), ws[aga].as<uint8_t>(), n, level, iso, z_lo, z_hi, keep,
                              ws[WS_PROP_NEED].as<uint8_t>(), st));
        ISX_TRY(compact_flags(inr, ws[WS_PROP_NEED].as<uint8_t>(), n, ws[WS_PROP_IDX].as<uint32_t>(), nullptr,
                              d_count, st));
        int64_t nneed = 0;
        ISX_CUDA(cudaMemcpyAsync(&nneed, d_count, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        ISX_CUDA(cudaStreamSynchronize(st));
        if (nneed > 0) {
          ISX_TRY(gather_codes(ws[ca].as<uint32_t>(), ws[WS_PROP_IDX].as<uint32_t>(), nneed,
                               ws[WS_PROP_CODES].as<uint32_t>(), st));
          CellSource src;
          src.codes = ws[WS_PROP_CODES].as<uint32_t>();
          src.level = level;
          ISX_TRY(bound_dispatch(inr, src, nneed, p->mode, p->prec, p->inflate, ws[WS_CENTER].as<float>(),
                                 ws[WS_SPREAD].as<float>(), st));
          ISX_TRY(proposer_merge(ws[WS_PROP_IDX].as<uint32_t>(), nneed, ws[ma].as<uint32_t>(),
                                 ws[WS_CENTER].as<float>(), ws[WS_SPREAD].as<float>(), iso, p->mode, p->k,
                                 p->inflate, keep, ws[aca].as<float>(), ws[asa].as<float>(), ws[aga].as<uint8_t>(),
                                 st));
        }
        mesh->cells_bounded[level] = nneed;
        step_masks = keep;
        step_bounded = false;
        anc.in_c = ws[aca].as<float>();
        anc.in_s = ws[asa].as<float>();
        anc.in_gap = ws[aga].as<uint8_t>();
      } else if (bounded) {
        CellSource src;
        src.codes = ws[ca].as<uint32_t>();
        src.level = level;
        ISX_TRY(bound_dispatch(inr, src, n, p->mode, p->prec, p->inflate, ws[WS_CENTER].as<float>(),
                               ws[WS_SPREAD].as<float>(), st));
        anc.in_c = ws[WS_CENTER].as<float>();
        anc.in_s = ws[WS_SPREAD].as<float>();
      }
      size_t need = (size_t)(expand ? 8 : 1) * n * 4;
      ISX_TRY(ws[cb].ensure(need, "codes"));
      ISX_TRY(ws[mb].ensure(need, "masks"));
      if (carry) {
        ISX_TRY(ws[acb].ensure(need, "ancestor centre"));
        ISX_TRY(ws[asb].ensure(need, "ancestor spread"));
        ISX_TRY(ws[agb].ensure(need / 4, "ancestor gap"));
        anc.out_c = ws[acb].as<float>();
        anc.out_s = ws[asb].as<float>();
        anc.out_gap = ws[agb].as<uint8_t>();
      }
    }
    if (rec) {
      // the visited cells of this level, their inherited masks and their bounds, appended
      const int64_t o = rec->level_off[level];
      rec->level_off[level + 1] = o + n;
      if (o + n > rec->cap) rec_short = true;
      if (!rec_short && n > 0) {
        ISX_CUDA(cudaMemcpyAsync(rec->d_code + o, ws[ca].ptr, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
        ISX_CUDA(cudaMemcpyAsync(rec->d_mask + o, ws[ma].ptr, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
        if (bounded) {
          ISX_CUDA(cudaMemcpyAsync(rec->d_center + o, ws[WS_CENTER].ptr, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
          ISX_CUDA(cudaMemcpyAsync(rec->d_spread + o, ws[WS_SPREAD].ptr, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
        } else {
          ISX_TRY(fill_f32(rec->d_center + o, n, NAN, st));
          ISX_TRY(fill_f32(rec->d_spread + o, n, NAN, st));
        }
      }
    }
    ISX_TRY(level_step(inr, ws[ca].as<uint32_t>(), step_masks, n, ws[WS_CENTER].as<float>(),
                       ws[WS_SPREAD].as<float>(), step_bounded, iso, p->mode, p->k, p->inflate, expand,
                       ws[cb].as<uint32_t>(), ws[mb].as<uint32_t>(), d_count, st, carry ? &anc : nullptr));
    int64_t cnt = 0;
    ISX_CUDA(cudaMemcpyAsync(&cnt, d_count, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    ISX_CUDA(cudaStreamSynchronize(st));
    mesh->cells_kept[level] = expand ? cnt / 8 : cnt;
    std::swap(ca, cb);
    std::swap(ma, mb);
    std::swap(aca, acb);
    std::swap(asa, asb);
    std::swap(aga, agb);
    n = cnt;
  }
  isx_status ms = mesh_from_active(inr, p, ws[ca].as<uint32_t>(), ws[ma].as<uint32_t>(), n, mesh, tm, st);
  if (ms == ISX_OK && rec_short) {
    set_error("level-record capacity exceeded (level_off holds the required sizes)");
    return ISX_ERR_CAPACITY;
  }
  return ms;
}

isx_status isx_extract_dense(isx_inr inr, const isx_extract_params* p, isx_mesh* mesh, void* stream) {
  ISX_TRY(check_inr(inr));
  ISX_TRY(validate_params(p, mesh));
  cudaStream_t st = (cudaStream_t)stream;
  const int L = p->max_level;
  const int R = 1 << L;
  const IsoSet iso = iso_of(p);
  for (int l = 0; l <= ISX_MAX_LEVEL; ++l) mesh->cells_bounded[l] = mesh->cells_kept[l] = mesh->cells_visited[l] = 0;
  mesh->n_active = mesh->n_tris = 0;
  Timer tm;
  ISX_TRY(tm.init());
  ISX_CUDA(cudaEventRecord(tm.ev[0], st));
  ISX_CUDA(cudaEventRecord(tm.ev[1], st));
  int64_t nlat = (int64_t)(R + 1) * (R + 1) * (R + 1);
  auto& ws = inr->ws;
  ISX_TRY(ws[WS_VALUES].ensure((size_t)nlat * 4, "values"));
  mesh->n_points = nlat;
  // lattice ids are 0..nlat-1: evaluate with an identity id list
  ISX_TRY(ws[WS_POINTS].ensure((size_t)nlat * 4, "points"));
  ISX_TRY(iota_u32(ws[WS_POINTS].as<uint32_t>(), nlat, st));
  ISX_TRY(eval_dispatch(inr, p->eval_prec, ws[WS_POINTS].as<uint32_t>(), R, nlat, ws[WS_VALUES].as<float>(), st));
  ISX_CUDA(cudaEventRecord(tm.ev[2], st));
  isx_status s = marching_cubes(inr, nullptr, nullptr, (int64_t)R * R * R, R, nullptr, ws[WS_VALUES].as<float>(),
                                iso, mesh, true, st);
  ISX_CUDA(cudaEventRecord(tm.ev[3], st));
  ISX_CUDA(cudaEventSynchronize(tm.ev[3]));
  cudaEventElapsedTime(&mesh->ms_acp, tm.ev[0], tm.ev[1]);
  cudaEventElapsedTime(&mesh->ms_inr, tm.ev[1], tm.ev[2]);
  cudaEventElapsedTime(&mesh->ms_mc, tm.ev[2], tm.ev[3]);
  cudaEventElapsedTime(&mesh->ms_total, tm.ev[0], tm.ev[3]);
  return s;
}

isx_status isx_check_bounded_wait(int64_t limit_ns, void* stream) {
  if (limit_ns < 1000 || limit_ns > 10000000000LL) {
    set_error("the wait limit must lie in [1000, 10^10] ns");
    return ISX_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int* d_status = nullptr;
  ISX_CUDA(cudaMalloc(&d_status, sizeof(int)));
  isx_status s = ISX_OK;
  int h = 0;
  cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    s = rows::check_bounded_wait(limit_ns, d_status, st);
    if (s == ISX_OK) {
      e = cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
  }
  cudaFree(d_status);
  if (e != cudaSuccess) return cuda_fail(e, "bounded-wait check", __FILE__, __LINE__);
  if (s != ISX_OK) return s;
  if (h != 0) {
    set_error("bounded device wait expired (as intended by the check)");
    return (isx_status)h;
  }
  set_error("bounded device wait did not report its expiry");
  return ISX_ERR_CUDA;
}

}  // extern "C"
