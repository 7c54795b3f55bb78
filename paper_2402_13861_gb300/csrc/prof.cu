// Per-kernel launch accounting: launch counts always; CUDA-event durations and algorithmic work
// (FLOPs and bytes as defined by the method, not by the implementation) when enabled.
#include "internal.cuh"

#include <mutex>

namespace isx {
namespace prof {

namespace {
struct Rec {
  int kernel;
  cudaEvent_t a, b;
  double flops, bytes;
};
std::mutex mu;
bool enabled = false;
std::vector<Rec> pending;
struct Acc {
  int64_t launches = 0;
  double ms = 0, flops = 0, bytes = 0;
};
Acc acc[K_COUNT];
const char* names[K_COUNT] = {"input_layer",   "relu",          "center_gemv",   "gemm_fp32",    "fresh_rows",
                              "reduce",        "output",        "cull_count",    "scan_counts",  "scatter_cells",
                              "mark_corners",  "flag_count",    "scatter_flags", "eval_fp32",    "mc_count",
                              "mc_emit",       "iota",          "bound_tc",      "tc_prep",      "tc_output",
                              "eval_tc",       "prop_gate",     "prop_merge",   "prop_forward",
                              "prop_grad",     "prop_adam",     "bound_rafixed", "rows_gemm",     "rows_aux",
                              "rows_act",      "rows_new",      "rows_split",    "rows_reduce",  "rows_out"};

void drain_locked() {
  for (auto& r : pending) {
    float ms = 0;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      acc[r.kernel].ms += ms;
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  pending.clear();
}
}  // namespace

Scope::Scope(int kernel, cudaStream_t st, double flops, double bytes) : kernel_(kernel), st_(st) {
  std::lock_guard<std::mutex> lk(mu);
  acc[kernel].launches += 1;
  acc[kernel].flops += flops;
  acc[kernel].bytes += bytes;
  if (!enabled) return;
  active_ = true;
  cudaEventCreate(&a_);
  cudaEventCreate(&b_);
  cudaEventRecord(a_, st_);
}

Scope::~Scope() {
  if (!active_) return;
  cudaEventRecord(b_, st_);
  std::lock_guard<std::mutex> lk(mu);
  pending.push_back({kernel_, a_, b_, 0, 0});
  if (pending.size() > 4096) drain_locked();
}

}  // namespace prof
}  // namespace isx

using namespace isx;

extern "C" {

void isx_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(prof::mu);
  prof::enabled = on != 0;
}

void isx_profile_reset(void) {
  std::lock_guard<std::mutex> lk(prof::mu);
  prof::drain_locked();
  for (auto& a : prof::acc) a = prof::Acc();
}

int isx_profile_read(isx_kernel_stats* out, int max) {
  std::lock_guard<std::mutex> lk(prof::mu);
  prof::drain_locked();
  int n = 0;
  for (int k = 0; k < K_COUNT && n < max; ++k) {
    out[n].name = prof::names[k];
    out[n].launches = prof::acc[k].launches;
    out[n].ms = prof::acc[k].ms;
    out[n].flops = prof::acc[k].flops;
    out[n].bytes = prof::acc[k].bytes;
    ++n;
  }
  return n;
}

}  // extern "C"
