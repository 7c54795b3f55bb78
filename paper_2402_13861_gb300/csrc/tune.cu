// Launch-shape autotuner.  A kernel with several interchangeable variants (tile shapes that give
// bit-identical results) asks pick() which variant to launch for a key (kernel, width, size
// bucket).  The first time a key is seen every variant is run twice on the caller's real operands
// and timed with CUDA events on the caller's stream (the second run counts); the fastest is cached
// for the process.  ISX_TUNE=0 disables tuning (variant 0 always); no tuning happens while the
// stream is being captured into a graph.  The choices are readable through isx_tune_read.
#include "internal.cuh"

#include <cstdlib>
#include <map>
#include <mutex>
#include <vector>

namespace isx {
namespace tune {
namespace {
struct Entry {
  int variant = 0;
  std::string choice;
  std::vector<float> ms;
};
std::mutex mu;
std::map<std::string, Entry> table;

bool enabled() {
  const char* e = std::getenv("ISX_TUNE");
  return !(e && e[0] == '0');
}
}  // namespace

isx_status pick(const std::string& key, int n, const std::function<const char*(int)>& name,
                const std::function<isx_status(int)>& run, cudaStream_t st, int* out) {
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = table.find(key);
    if (it != table.end()) {
      *out = it->second.variant;
      return ISX_OK;
    }
  }
  *out = 0;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  ISX_CUDA(cudaStreamIsCapturing(st, &cs));
  if (!enabled() || n <= 1 || cs != cudaStreamCaptureStatusNone) return ISX_OK;
  Entry e;
  e.ms.assign(n, 0.f);
  cudaEvent_t a = nullptr, b = nullptr;
  ISX_CUDA(cudaEventCreate(&a));
  ISX_CUDA(cudaEventCreate(&b));
  isx_status s = ISX_OK;
  for (int v = 0; v < n && s == ISX_OK; ++v) {
    s = run(v);
    if (s != ISX_OK) break;
    cudaEventRecord(a, st);
    s = run(v);
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&e.ms[v], a, b);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (s != ISX_OK) return s;
  for (int v = 1; v < n; ++v)
    if (e.ms[v] < e.ms[e.variant]) e.variant = v;
  e.choice = name(e.variant);
  *out = e.variant;
  std::lock_guard<std::mutex> lk(mu);
  table.emplace(key, e);
  return ISX_OK;
}

}  // namespace tune
}  // namespace isx

using namespace isx;

extern "C" {

int isx_tune_read(isx_tune_entry* out, int max) {
  std::lock_guard<std::mutex> lk(tune::mu);
  int i = 0;
  for (auto& kv : tune::table) {
    if (i >= max) break;
    out[i].key = kv.first.c_str();
    out[i].choice = kv.second.choice.c_str();
    out[i].variant = kv.second.variant;
    out[i].n_variants = (int)kv.second.ms.size();
    out[i].ms_best = kv.second.ms[kv.second.variant];
    out[i].ms_first = kv.second.ms[0];
    ++i;
  }
  return (int)tune::table.size();
}

void isx_tune_reset(void) {
  std::lock_guard<std::mutex> lk(tune::mu);
  tune::table.clear();
}

}  // extern "C"
