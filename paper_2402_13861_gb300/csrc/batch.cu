// Batched extraction: the octrees of many INRs walked level-synchronously (Algorithm 1 for every
// INR, one level of all of them at a time), their cells bounded together.
//
// All cells of one level of every INR form one list (packed code, entry index, iso mask), ordered by
// entry; stable compaction keeps each entry's cells contiguous.  Per level:
//   - one persistent tensor-core launch per hidden width present (k_bound_tc reads every cell's
//     network from a device table of descriptors and skips cells of the other width);
//   - k_bcull: the cull test of Algorithm 1 with the entry's iso-values and k; a surviving cell is
//     subdivided below its entry's finest level, and at that level it is an active cell;
//   - two stable compactions (scan of block counts, scatter): children to the next level's list,
//     active cells appended to the list of finished cells;
//   - k_badvance: next level's count and the finished count, on the device.
// Every count lives in device memory and every grid is sized from a capacity, so the level loop
// needs no host synchronisation: with graphs on, the first run sizes the capacities (reading the
// counts level by level), the whole loop is then captured once into a CUDA graph and later runs
// replay it; a count above its capacity raises an overflow flag and the run is repeated unbatched
// from the graph (sized anew, recaptured).  Corner evaluation and marching cubes then run per entry.
#include "compact.cuh"
#include "internal.cuh"

#include <algorithm>
#include <vector>

namespace isx {
namespace {

using namespace compact;

struct BNet {                          // one entry of the batch (device)
  IsoSet iso;
  float k;
  int L;                               // finest level
};

__global__ void k_binit(int n, const uint32_t* full, uint32_t* codes, uint16_t* nets, uint32_t* masks,
                        int64_t* counters, int ncounters, int64_t* done_total, int* overflow) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    codes[i] = 0u;
    nets[i] = (uint16_t)i;
    masks[i] = full[i];
  }
  if (i == 0) {
    counters[0] = n;
    for (int l = 1; l < ncounters; ++l) counters[l] = 0;
    *done_total = 0;
    *overflow = 0;
  }
}

// kind: 0 culled, 1 kept and subdivided, 2 kept at the entry's finest level (active)
__global__ void __launch_bounds__(kThreads) k_bcull(const int64_t* n_dev, const uint32_t* masks, const uint16_t* nets,
                                                    const float* center, const float* spread, const BNet* bn,
                                                    int level, int mode, int inflate, uint32_t* newmask,
                                                    uint8_t* kind, int* bc_expand, int* bc_done) {
  const int64_t n = *n_dev;
  const int64_t base = (int64_t)blockIdx.x * kTile;
  if (base >= n) return;               // the scans read ceil(n / kTile) block counts only
  int ce = 0, cd = 0;
  for (int e = 0; e < kPer; ++e) {
    const int64_t i = base + e * kThreads + threadIdx.x;
    if (i < n) {
      const BNet& b = bn[nets[i]];
      const uint32_t m = masks[i] & keep_bits(center[i], spread[i], b.iso, mode, b.k, inflate);
      const uint8_t kd = m ? (level < b.L ? 1 : 2) : 0;
      newmask[i] = m;
      kind[i] = kd;
      ce += kd == 1;
      cd += kd == 2;
    }
  }
  __shared__ int red[2][kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ce += __shfl_xor_sync(0xffffffffu, ce, o);
    cd += __shfl_xor_sync(0xffffffffu, cd, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = ce;
    red[1][threadIdx.x >> 5] = cd;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int se = 0, sd = 0;
    for (int q = 0; q < kThreads / 32; ++q) {
      se += red[0][q];
      sd += red[1][q];
    }
    bc_expand[blockIdx.x] = se;
    bc_done[blockIdx.x] = sd;
  }
}

__global__ void __launch_bounds__(1024) k_bscan(const int64_t* n_dev, const int* counts, int64_t* offsets,
                                                int64_t* total) {
  const int64_t nb = (*n_dev + kTile - 1) / kTile;
  scan_block_counts_dev(counts, nb, offsets, total, 1);
}

__global__ void __launch_bounds__(kThreads) k_bscatter(const int64_t* n_dev, const uint32_t* codes,
                                                       const uint16_t* nets, const uint32_t* newmask,
                                                       const uint8_t* kind, const int64_t* off_e,
                                                       const int64_t* off_d, const int64_t* done_base,
                                                       int64_t cap_next, int64_t cap_done, uint32_t* nc,
                                                       uint16_t* nn, uint32_t* nm, uint32_t* dc, uint16_t* dn,
                                                       uint32_t* dm, int* overflow) {
  __shared__ int ws_e[32], ws_d[32];
  __shared__ int tot_e, tot_d;
  const int64_t n = *n_dev;
  const int64_t base = (int64_t)blockIdx.x * kTile;
  if (base >= n) return;               // uniform over the block
  int64_t oe = off_e[blockIdx.x];
  int64_t od = off_d[blockIdx.x] + *done_base;
  for (int e = 0; e < kPer; ++e) {
    const int64_t i = base + e * kThreads + threadIdx.x;
    const uint8_t kd = i < n ? kind[i] : 0;
    const int re = block_rank(kd == 1, ws_e, &tot_e);
    const int rd = block_rank(kd == 2, ws_d, &tot_d);
    if (kd == 1) {
      const int64_t o = oe + re;
      if (8 * o + 8 <= cap_next) {
        const uint32_t code = codes[i], m = newmask[i];
        const uint16_t net = nets[i];
        const uint32_t ci = (code & 1023u) << 1, cj = ((code >> 10) & 1023u) << 1, ck = ((code >> 20) & 1023u) << 1;
        for (int c = 0; c < 8; ++c) {
          nc[8 * o + c] = (ci + (c & 1)) | ((cj + ((c >> 1) & 1)) << 10) | ((ck + ((c >> 2) & 1)) << 20);
          nn[8 * o + c] = net;
          nm[8 * o + c] = m;
        }
      } else {
        atomicExch(overflow, 1);
      }
    } else if (kd == 2) {
      const int64_t o = od + rd;
      if (o < cap_done) {
        dc[o] = codes[i];
        dn[o] = nets[i];
        dm[o] = newmask[i];
      } else {
        atomicExch(overflow, 1);
      }
    }
    oe += tot_e;
    od += tot_d;
  }
}

__global__ void k_badvance(const int64_t* tot_e, const int64_t* tot_d, int64_t* n_next, int64_t* done_total,
                           int64_t cap_next, int64_t cap_done, int* overflow) {
  int64_t ne = 8 * *tot_e;
  if (ne > cap_next) {
    ne = cap_next - cap_next % 8;
    *overflow = 1;
  }
  *n_next = ne;
  int64_t dt = *done_total + *tot_d;
  if (dt > cap_done) {
    dt = cap_done;
    *overflow = 1;
  }
  *done_total = dt;
}

// Start and length of every entry's run in the finished list (runs are contiguous).
__global__ void k_bsegments(const int64_t* done_total, const uint16_t* dn, int64_t* start, int64_t* count) {
  const int64_t n = *done_total;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const uint16_t e = dn[j];
    if (j == 0 || dn[j - 1] != e) start[e] = j;
    atomicAdd(reinterpret_cast<unsigned long long*>(&count[e]), 1ull);
  }
}

}  // namespace
}  // namespace isx

using namespace isx;

struct isx_batch_s {
  int device = 0, n = 0, Lmax = 0, use_graph = 0;
  std::vector<isx_inr> inrs;
  std::vector<isx_extract_params> params;
  isx_bound_mode mode = ISX_BOUND_CLT;
  int inflate = 0;
  int widths[2] = {0, 0};              // hidden widths present (0: none)
  int rows[2] = {0, 0};                // scratch rows per CTA for each width
  int grid = 0;
  Buf nets, bnets, full, counters, done_total, overflow, status, scratch;
  Buf codes[2], enets[2], masks[2], center, spread, newmask, kind, bc_e, bc_d, off_e, off_d, tot_e, tot_d;
  Buf dcodes, dnets, dmasks, seg_start, seg_count;
  std::vector<int64_t> cap;            // capacity of every level's list
  int64_t cap_done = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool captured = false;
  cudaStream_t cap_stream = nullptr;   // captures happen here (the legacy default stream cannot be captured)
};

namespace {

void drop_graph(isx_batch b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->captured = false;
}

// The list of one level (slot 0 or 1): grows without keeping its contents.
isx_status ensure_slot(isx_batch b, int slot, int64_t cap) {
  const size_t c = (size_t)std::max<int64_t>(cap, 1);
  ISX_TRY(b->codes[slot].ensure(c * 4, "batch codes"));
  ISX_TRY(b->enets[slot].ensure(c * 2, "batch nets"));
  ISX_TRY(b->masks[slot].ensure(c * 4, "batch masks"));
  return ISX_OK;
}

// Per-level working arrays (rewritten every level).
isx_status ensure_work(isx_batch b, int64_t cap) {
  const size_t c = (size_t)std::max<int64_t>(cap, 1);
  ISX_TRY(b->center.ensure(c * 4, "batch centre"));
  ISX_TRY(b->spread.ensure(c * 4, "batch spread"));
  ISX_TRY(b->newmask.ensure(c * 4, "batch new masks"));
  ISX_TRY(b->kind.ensure(c, "batch kinds"));
  const size_t nb = (c + kTile - 1) / kTile;
  ISX_TRY(b->bc_e.ensure(nb * 4, "batch block counts"));
  ISX_TRY(b->bc_d.ensure(nb * 4, "batch block counts"));
  ISX_TRY(b->off_e.ensure(nb * 8, "batch offsets"));
  ISX_TRY(b->off_d.ensure(nb * 8, "batch offsets"));
  return ISX_OK;
}

// Enqueues level `level` (list in slot level % 2, capacities cap_in -> cap_next).
isx_status enqueue_level(isx_batch b, int level, int64_t cap_in, int64_t cap_next, cudaStream_t st) {
  const int s = level & 1, t = s ^ 1;
  int64_t* cnt = b->counters.as<int64_t>();
  for (int g = 0; g < 2; ++g) {
    if (!b->widths[g]) continue;
    ISX_TRY(bound_bf16_batch(b->nets.ptr, b->widths[g], b->rows[g], b->codes[s].as<uint32_t>(),
                             b->enets[s].as<uint16_t>(), level, cnt + level, b->mode, b->inflate,
                             b->center.as<float>(), b->spread.as<float>(), b->scratch.as<__nv_bfloat16>(), b->grid,
                             b->status.as<int>(), st));
  }
  const unsigned nb = (unsigned)std::max<int64_t>(1, (cap_in + kTile - 1) / kTile);
  k_bcull<<<nb, kThreads, 0, st>>>(cnt + level, b->masks[s].as<uint32_t>(), b->enets[s].as<uint16_t>(),
                                   b->center.as<float>(), b->spread.as<float>(), b->bnets.as<BNet>(), level,
                                   (int)b->mode, b->inflate, b->newmask.as<uint32_t>(), b->kind.as<uint8_t>(),
                                   b->bc_e.as<int>(), b->bc_d.as<int>());
  ISX_LAUNCH_CHECK("k_bcull");
  k_bscan<<<1, 1024, 0, st>>>(cnt + level, b->bc_e.as<int>(), b->off_e.as<int64_t>(), b->tot_e.as<int64_t>());
  ISX_LAUNCH_CHECK("k_bscan");
  k_bscan<<<1, 1024, 0, st>>>(cnt + level, b->bc_d.as<int>(), b->off_d.as<int64_t>(), b->tot_d.as<int64_t>());
  ISX_LAUNCH_CHECK("k_bscan");
  k_bscatter<<<nb, kThreads, 0, st>>>(cnt + level, b->codes[s].as<uint32_t>(), b->enets[s].as<uint16_t>(),
                                      b->newmask.as<uint32_t>(), b->kind.as<uint8_t>(), b->off_e.as<int64_t>(),
                                      b->off_d.as<int64_t>(), b->done_total.as<int64_t>(), cap_next, b->cap_done,
                                      b->codes[t].as<uint32_t>(), b->enets[t].as<uint16_t>(),
                                      b->masks[t].as<uint32_t>(), b->dcodes.as<uint32_t>(), b->dnets.as<uint16_t>(),
                                      b->dmasks.as<uint32_t>(), b->overflow.as<int>());
  ISX_LAUNCH_CHECK("k_bscatter");
  k_badvance<<<1, 1, 0, st>>>(b->tot_e.as<int64_t>(), b->tot_d.as<int64_t>(), cnt + level + 1,
                              b->done_total.as<int64_t>(), cap_next, b->cap_done, b->overflow.as<int>());
  ISX_LAUNCH_CHECK("k_badvance");
  return ISX_OK;
}

isx_status enqueue_init(isx_batch b, cudaStream_t st) {
  k_binit<<<(b->n + 255) / 256, 256, 0, st>>>(b->n, b->full.as<uint32_t>(), b->codes[0].as<uint32_t>(),
                                               b->enets[0].as<uint16_t>(), b->masks[0].as<uint32_t>(),
                                               b->counters.as<int64_t>(), b->Lmax + 2, b->done_total.as<int64_t>(),
                                               b->overflow.as<int>());
  ISX_LAUNCH_CHECK("k_binit");
  ISX_CUDA(cudaMemsetAsync(b->status.ptr, 0, sizeof(int), st));
  return ISX_OK;
}

// Level loop with the host reading every level's count; records the capacities (1.25x the counts)
// for a later capture.  Any graph is dropped first (buffers may move).
isx_status run_sized(isx_batch b, cudaStream_t st) {
  drop_graph(b);
  std::vector<int64_t> counts(b->Lmax + 2, 0);
  counts[0] = b->n;
  if (b->cap_done < 4096) b->cap_done = 4096;
  ISX_TRY(b->dcodes.ensure((size_t)b->cap_done * 4, "batch finished codes"));
  ISX_TRY(b->dnets.ensure((size_t)b->cap_done * 2, "batch finished nets"));
  ISX_TRY(b->dmasks.ensure((size_t)b->cap_done * 4, "batch finished masks"));
  ISX_TRY(ensure_slot(b, 0, b->n));
  ISX_TRY(enqueue_init(b, st));
  int64_t n = b->n, done = 0;
  for (int level = 0; level <= b->Lmax && n > 0; ++level) {
    // worst case of this level: every cell kept and subdivided, or every cell finished
    const int64_t next_cap = 8 * n;
    ISX_TRY(ensure_slot(b, (level & 1) ^ 1, next_cap));
    ISX_TRY(ensure_work(b, n));
    if (done + n > b->cap_done) {
      // grow the finished list keeping its contents
      const int64_t nc = std::max<int64_t>(2 * b->cap_done, done + n);
      Buf c2, n2, m2;
      ISX_TRY(c2.ensure((size_t)nc * 4, "batch finished codes"));
      ISX_TRY(n2.ensure((size_t)nc * 2, "batch finished nets"));
      ISX_TRY(m2.ensure((size_t)nc * 4, "batch finished masks"));
      if (done > 0) {
        ISX_CUDA(cudaMemcpyAsync(c2.ptr, b->dcodes.ptr, done * 4, cudaMemcpyDeviceToDevice, st));
        ISX_CUDA(cudaMemcpyAsync(n2.ptr, b->dnets.ptr, done * 2, cudaMemcpyDeviceToDevice, st));
        ISX_CUDA(cudaMemcpyAsync(m2.ptr, b->dmasks.ptr, done * 4, cudaMemcpyDeviceToDevice, st));
        ISX_CUDA(cudaStreamSynchronize(st));
      }
      std::swap(b->dcodes, c2);
      std::swap(b->dnets, n2);
      std::swap(b->dmasks, m2);
      c2.release();
      n2.release();
      m2.release();
      b->cap_done = nc;
    }
    ISX_TRY(enqueue_level(b, level, n, next_cap, st));
    int64_t h[2];
    ISX_CUDA(cudaMemcpyAsync(&h[0], b->counters.as<int64_t>() + level + 1, 8, cudaMemcpyDeviceToHost, st));
    ISX_CUDA(cudaMemcpyAsync(&h[1], b->done_total.ptr, 8, cudaMemcpyDeviceToHost, st));
    ISX_CUDA(cudaStreamSynchronize(st));
    counts[level + 1] = h[0];
    n = h[0];
    done = h[1];
  }
  b->cap.assign(b->Lmax + 2, 0);
  for (int l = 0; l <= b->Lmax + 1; ++l) b->cap[l] = counts[l] + counts[l] / 4 + 1024;
  b->cap_done = std::max<int64_t>(b->cap_done, done + done / 4 + 1024);
  return ISX_OK;
}

isx_status capture(isx_batch b, cudaStream_t user_st) {
  drop_graph(b);
  if (!b->cap_stream) ISX_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  // buffers are (re)allocated before the capture; the user's stream must not be using them
  ISX_CUDA(cudaStreamSynchronize(user_st));
  cudaStream_t st = b->cap_stream;
  int64_t cmax = 0;
  for (int64_t c : b->cap) cmax = std::max(cmax, c);
  ISX_TRY(ensure_slot(b, 0, cmax));
  ISX_TRY(ensure_slot(b, 1, cmax));
  ISX_TRY(ensure_work(b, cmax));
  ISX_TRY(b->dcodes.ensure((size_t)b->cap_done * 4, "batch finished codes"));
  ISX_TRY(b->dnets.ensure((size_t)b->cap_done * 2, "batch finished nets"));
  ISX_TRY(b->dmasks.ensure((size_t)b->cap_done * 4, "batch finished masks"));
  ISX_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
  isx_status s = enqueue_init(b, st);
  for (int level = 0; level <= b->Lmax && s == ISX_OK; ++level)
    s = enqueue_level(b, level, b->cap[level], b->cap[level + 1], st);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &g);
  if (s != ISX_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
  b->graph = g;
  ISX_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
  b->captured = true;
  return ISX_OK;
}

}  // namespace

extern "C" {

isx_status isx_batch_create(const isx_inr* inrs, const isx_extract_params* params, int n, int use_graph,
                            isx_batch* out) {
  if (!inrs || !params || !out || n <= 0 || n > 65535) {
    set_error("batch: need 1..65535 INRs with their parameters");
    return ISX_ERR_ARG;
  }
  *out = nullptr;
  int dev = 0;
  ISX_CUDA(cudaGetDevice(&dev));
  for (int i = 0; i < n; ++i) {
    if (!inrs[i] || inrs[i]->device != dev) {
      set_error("batch: every INR must live on the current device");
      return ISX_ERR_ARG;
    }
    isx_mesh dummy{};
    ISX_TRY(validate_extract_params(&params[i], &dummy));
    if (params[i].prec != ISX_PREC_BF16 || !bf16_supported(inrs[i])) {
      set_error("batch: BF16 tensor-core bounds only (hidden widths 128 and 256)");
      return ISX_ERR_UNSUPPORTED;
    }
    if (params[i].mode != params[0].mode || params[i].inflate != params[0].inflate) {
      set_error("batch: every entry must use the same bound mode and inflation");
      return ISX_ERR_ARG;
    }
    if (params[i].proposer || params[i].kd_tree ||
        (params[i].bound_stop_level >= 0 && params[i].bound_stop_level < params[i].max_level)) {
      set_error("batch: the proposer, the k-d mode and bound_stop_level are not supported in a batch");
      return ISX_ERR_UNSUPPORTED;
    }
  }
  isx_batch b = new isx_batch_s();
  b->device = dev;
  b->n = n;
  b->use_graph = use_graph != 0;
  b->inrs.assign(inrs, inrs + n);
  b->params.assign(params, params + n);
  b->mode = params[0].mode;
  b->inflate = params[0].mode == ISX_BOUND_SOUND ? params[0].inflate : 0;
  auto fail = [&](isx_status s) {
    isx_batch_destroy(b);
    return s;
  };
  std::vector<uint8_t> nets((size_t)n * tc_net_bytes());
  std::vector<BNet> bn(n);
  std::vector<uint32_t> full(n);
  for (int i = 0; i < n; ++i) {
    const void* d = nullptr;
    isx_status s = tc_net_of(inrs[i], &d);
    if (s != ISX_OK) return fail(s);
    cudaError_t e = cudaMemcpy(nets.data() + (size_t)i * tc_net_bytes(), d, tc_net_bytes(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(cuda_fail(e, "batch descriptors", __FILE__, __LINE__));
    bn[i].iso = iso_set_of(&params[i]);
    bn[i].k = params[i].k;
    bn[i].L = params[i].max_level;
    full[i] = params[i].n_iso >= 32 ? 0xffffffffu : ((1u << params[i].n_iso) - 1u);
    b->Lmax = std::max(b->Lmax, params[i].max_level);
    const int w = inrs[i]->w, g = (w == 256) ? 1 : 0;
    b->widths[g] = w;
    b->rows[g] = std::max(b->rows[g], std::max(128, w * std::max(0, inrs[i]->H - 3)));
  }
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->grid = sms;
  isx_status s;
  if ((s = b->nets.ensure(nets.size(), "batch descriptors")) != ISX_OK ||
      (s = b->bnets.ensure(bn.size() * sizeof(BNet), "batch entries")) != ISX_OK ||
      (s = b->full.ensure(full.size() * 4, "batch masks")) != ISX_OK ||
      (s = b->counters.ensure((size_t)(b->Lmax + 2) * 8, "batch counters")) != ISX_OK ||
      (s = b->done_total.ensure(8, "batch counters")) != ISX_OK || (s = b->overflow.ensure(8, "batch flag")) != ISX_OK ||
      (s = b->status.ensure(8, "batch status")) != ISX_OK || (s = b->tot_e.ensure(8, "batch totals")) != ISX_OK ||
      (s = b->tot_d.ensure(8, "batch totals")) != ISX_OK ||
      (s = b->seg_start.ensure((size_t)n * 8, "batch segments")) != ISX_OK ||
      (s = b->seg_count.ensure((size_t)n * 8, "batch segments")) != ISX_OK)
    return fail(s);
  const int wmax = b->widths[1] ? 256 : 128;
  const int rmax = std::max(b->rows[0], b->rows[1]);
  if ((s = b->scratch.ensure((size_t)b->grid * rmax * wmax * 2, "batch scratch")) != ISX_OK) return fail(s);
  cudaError_t e;
  if ((e = cudaMemcpy(b->nets.ptr, nets.data(), nets.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(b->bnets.ptr, bn.data(), bn.size() * sizeof(BNet), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(b->full.ptr, full.data(), full.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
    return fail(cuda_fail(e, "batch tables", __FILE__, __LINE__));
  *out = b;
  return ISX_OK;
}

isx_status isx_batch_run(isx_batch b, isx_mesh* meshes, void* stream) {
  if (!b || !meshes) {
    set_error("null batch or meshes");
    return ISX_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  Timer tm;
  ISX_TRY(tm.init());
  ISX_CUDA(cudaEventRecord(tm.ev[0], st));
  // ---- the level loop of all entries ----
  bool done = false;
  // a graph is captured from the capacities of the previous (sized) run, then replayed
  if (b->use_graph && !b->captured && !b->cap.empty()) ISX_TRY(capture(b, st));
  if (b->use_graph && b->captured) {
    ISX_CUDA(cudaGraphLaunch(b->exec, st));
    int flags[2] = {0, 0};
    ISX_CUDA(cudaMemcpyAsync(&flags[0], b->overflow.ptr, 4, cudaMemcpyDeviceToHost, st));
    ISX_CUDA(cudaMemcpyAsync(&flags[1], b->status.ptr, 4, cudaMemcpyDeviceToHost, st));
    ISX_CUDA(cudaStreamSynchronize(st));
    if (flags[1] != 0) {
      set_error("batch: the tensor-core bound kernel gave up waiting (bounded wait expired)");
      return (isx_status)flags[1];
    }
    done = flags[0] == 0;              // an overflow reruns sized and recaptures
  }
  if (!done) {
    ISX_TRY(run_sized(b, st));
    int stat = 0;
    ISX_CUDA(cudaMemcpyAsync(&stat, b->status.ptr, 4, cudaMemcpyDeviceToHost, st));
    ISX_CUDA(cudaStreamSynchronize(st));
    if (stat != 0) {
      set_error("batch: the tensor-core bound kernel gave up waiting (bounded wait expired)");
      return (isx_status)stat;
    }
  }
  ISX_CUDA(cudaEventRecord(tm.ev[1], st));
  float ms_levels = 0.f;
  // ---- per entry: its finished cells, corner evaluation and marching cubes ----
  ISX_CUDA(cudaMemsetAsync(b->seg_count.ptr, 0, (size_t)b->n * 8, st));
  ISX_CUDA(cudaMemsetAsync(b->seg_start.ptr, 0, (size_t)b->n * 8, st));
  k_bsegments<<<256, 256, 0, st>>>(b->done_total.as<int64_t>(), b->dnets.as<uint16_t>(), b->seg_start.as<int64_t>(),
                                   b->seg_count.as<int64_t>());
  ISX_LAUNCH_CHECK("k_bsegments");
  std::vector<int64_t> start(b->n), count(b->n);
  ISX_CUDA(cudaMemcpyAsync(start.data(), b->seg_start.ptr, (size_t)b->n * 8, cudaMemcpyDeviceToHost, st));
  ISX_CUDA(cudaMemcpyAsync(count.data(), b->seg_count.ptr, (size_t)b->n * 8, cudaMemcpyDeviceToHost, st));
  ISX_CUDA(cudaStreamSynchronize(st));
  cudaEventElapsedTime(&ms_levels, tm.ev[0], tm.ev[1]);
  isx_status result = ISX_OK;
  for (int i = 0; i < b->n; ++i) {
    isx_mesh* m = &meshes[i];
    for (int l = 0; l <= ISX_MAX_LEVEL; ++l) m->cells_bounded[l] = m->cells_kept[l] = m->cells_visited[l] = 0;
    m->n_tris = m->n_points = 0;
    m->n_active = count[i];
    if (count[i] > m->active_cap) {
      set_error("batch: active-cell capacity exceeded");
      result = ISX_ERR_CAPACITY;
      continue;
    }
    Timer ti;
    ISX_TRY(ti.init());
    ISX_CUDA(cudaEventRecord(ti.ev[0], st));
    isx_status s = mesh_from_active(b->inrs[i], &b->params[i], b->dcodes.as<uint32_t>() + start[i],
                                    b->dmasks.as<uint32_t>() + start[i], count[i], m, ti, st);
    m->ms_acp = ms_levels;            // the level loop is shared by the whole batch
    if (s != ISX_OK) result = s;
  }
  return result;
}

isx_status isx_batch_destroy(isx_batch b) {
  if (!b) return ISX_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  drop_graph(b);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (Buf* p : {&b->nets, &b->bnets, &b->full, &b->counters, &b->done_total, &b->overflow, &b->status, &b->scratch,
                 &b->codes[0], &b->codes[1], &b->enets[0], &b->enets[1], &b->masks[0], &b->masks[1], &b->center,
                 &b->spread, &b->newmask, &b->kind, &b->bc_e, &b->bc_d, &b->off_e, &b->off_d, &b->tot_e, &b->tot_d,
                 &b->dcodes, &b->dnets, &b->dmasks, &b->seg_start, &b->seg_count})
    p->release();
  if (prev >= 0) cudaSetDevice(prev);
  delete b;
  return ISX_OK;
}

}  // extern "C"
