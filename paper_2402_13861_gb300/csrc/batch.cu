// Batched extraction: many independent extractions (Algorithm 1 for every INR, then corner evaluation
// and marching cubes) in flight on the GPU together.
//
// Every entry runs exactly the single-extraction code (isx_extract_isosurface: the row-batched
// tensor-core bound for BF16, the float32 path for FP32), so its outputs are bit-identical to a single
// call with the same arguments.  What the batch adds is concurrency: a pool of host workers, each
// owning a non-blocking CUDA stream, takes entries from a shared counter.  The level loop of an
// extraction reads a count back to the host at every level (to size the next level's lists and row
// buffers), and a small extraction is bound by those round trips and by launch latency; with several
// extractions in flight their kernels fill the GPU together.  A large extraction fills it by itself.
// Each worker owns a workspace and lends it to the INR of the entry it runs (an INR handle otherwise
// keeps its own, grown to its largest extraction), so the batch holds `workers` workspaces however
// many INRs it has; with several workers the row-batched path's chunks are made smaller (chunking does
// not change any cell's result).  Entries that share an INR handle run on one worker, in entry order.
#include "internal.cuh"

#include <algorithm>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

struct BatchWorker {
  isx::Buf ws[isx::WS_N_SLOTS];                // the worker's workspace, lent to the entry it runs
  ~BatchWorker() {
    for (auto& b : ws) b.release();
  }
};

struct isx_batch_s {
  int device = 0;
  int n = 0;
  std::vector<isx_inr> inrs;
  std::vector<isx_extract_params> params;
  std::vector<std::vector<int>> groups;        // entries per INR handle, in entry order
  std::vector<cudaStream_t> streams;           // one per worker
  std::vector<cudaEvent_t> events;             // one per worker, plus the caller's start event
  std::vector<BatchWorker> workers;
  int64_t row_budget = 0;                      // symbol rows per chunk of the row-batched path
};

using namespace isx;

extern "C" {

isx_status isx_batch_create(const isx_inr* inrs, const isx_extract_params* params, int n, int workers,
                            isx_batch* out) {
  if (!inrs || !params || !out || n <= 0 || n > 65535) {
    set_error("batch: need 1..65535 INRs with their parameters");
    return ISX_ERR_ARG;
  }
  if (workers < 0 || workers > 64) {
    set_error("batch: workers must lie in 0..64 (0: the default, 8)");
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
  }
  isx_batch b = new isx_batch_s();
  b->device = dev;
  b->n = n;
  b->inrs.assign(inrs, inrs + n);
  b->params.assign(params, params + n);
  for (int i = 0; i < n; ++i) {
    bool placed = false;
    for (auto& g : b->groups)
      if (b->inrs[g[0]] == inrs[i]) {
        g.push_back(i);
        placed = true;
        break;
      }
    if (!placed) b->groups.push_back({i});
  }
  const int nw = std::max(1, std::min(workers > 0 ? workers : 8, (int)b->groups.size()));
  b->workers = std::vector<BatchWorker>(nw);
  b->row_budget = std::max<int64_t>((int64_t)1 << 21, ((int64_t)1 << 24) / nw);
  for (int w = 0; w < nw; ++w) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    cudaError_t err = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (s) b->streams.push_back(s);
    if (e) b->events.push_back(e);
    if (err != cudaSuccess) {
      isx_batch_destroy(b);
      return cuda_fail(err, "batch streams", __FILE__, __LINE__);
    }
  }
  cudaEvent_t start = nullptr;
  cudaError_t err = cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
  if (err != cudaSuccess) {
    isx_batch_destroy(b);
    return cuda_fail(err, "batch event", __FILE__, __LINE__);
  }
  b->events.push_back(start);
  *out = b;
  return ISX_OK;
}

isx_status isx_batch_run(isx_batch b, isx_mesh* meshes, void* stream) {
  if (!b) {
    set_error("null batch");
    return ISX_ERR_ARG;
  }
  if (!meshes) {
    set_error("null mesh array");
    return ISX_ERR_ARG;
  }
  int dev = -1;
  ISX_CUDA(cudaGetDevice(&dev));
  if (dev != b->device) {
    set_error("the batch was created on another device than the current one");
    return ISX_ERR_ARG;
  }
  // the workers start after the work already queued on the caller's stream
  cudaStream_t st = (cudaStream_t)stream;
  const int nw = (int)b->streams.size();
  cudaEvent_t start = b->events[nw];
  ISX_CUDA(cudaEventRecord(start, st));
  for (int w = 0; w < nw; ++w) ISX_CUDA(cudaStreamWaitEvent(b->streams[w], start, 0));
  std::vector<isx_status> status(b->n, ISX_OK);
  std::vector<std::string> message(b->n);
  std::atomic<int> next{0};
  auto work = [&](int w) {
    cudaSetDevice(b->device);
    for (int g = next++; g < (int)b->groups.size(); g = next++)
      for (int i : b->groups[g]) {
        isx_inr inr = b->inrs[i];
        // lend the worker's workspace and chunk size to the entry's INR for the call
        std::swap(inr->ws, b->workers[w].ws);
        const int64_t rb = inr->row_budget;
        inr->row_budget = b->row_budget;
        status[i] = isx_extract_isosurface(inr, &b->params[i], &meshes[i], b->streams[w]);
        if (status[i] != ISX_OK) message[i] = isx_last_error();
        inr->row_budget = rb;
        std::swap(inr->ws, b->workers[w].ws);
      }
  };
  std::vector<std::thread> pool;
  for (int w = 1; w < nw; ++w) pool.emplace_back(work, w);
  work(0);
  for (auto& t : pool) t.join();
  // the caller's stream sees every entry's work (each extraction also synchronised its own stream)
  for (int w = 0; w < nw; ++w) {
    ISX_CUDA(cudaEventRecord(b->events[w], b->streams[w]));
    ISX_CUDA(cudaStreamWaitEvent(st, b->events[w], 0));
  }
  for (int i = 0; i < b->n; ++i)
    if (status[i] != ISX_OK) {
      set_error("batch entry " + std::to_string(i) + ": " + message[i]);
      return status[i];
    }
  return ISX_OK;
}

isx_status isx_batch_destroy(isx_batch b) {
  if (!b) return ISX_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  for (auto s : b->streams) cudaStreamSynchronize(s);
  for (auto s : b->streams) cudaStreamDestroy(s);
  for (auto e : b->events) cudaEventDestroy(e);
  delete b;                                     // frees the workers' workspaces on this device
  if (prev >= 0) cudaSetDevice(prev);
  return ISX_OK;
}

}  // extern "C"
