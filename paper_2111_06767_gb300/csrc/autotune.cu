// Process-wide runtime settings of the library: launch-shape autotuning (element-batch and tile
// schedules: the first time a kernel shape is seen in the process, every candidate launch
// configuration is timed with CUDA events on the caller's stream, one warm-up launch and three
// timed ones, and the fastest is kept; it replaces hand-picked launch heuristics and has no
// counterpart in the paper), the stream of this thread's allocations, and the switch for
// programmatic dependent launch.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <set>
#include <string>

#include "internal.h"

namespace dg {

namespace {
std::mutex g_tune_mu;
std::map<std::vector<int64_t>, int> g_tuned;

thread_local cudaStream_t tl_alloc_stream = nullptr;

bool tuning_enabled() {
  const char* v = std::getenv("DG_AUTOTUNE");
  return !(v && std::strcmp(v, "0") == 0);
}
}  // namespace

// DG_TUNE_LOG=1: one line on stderr per tuned shape with the candidate kept and every candidate's
// time, and one per captured whole-solve graph.
bool tune_log() {
  static const bool on = [] {
    const char* v = std::getenv("DG_TUNE_LOG");
    return v && std::strcmp(v, "1") == 0;
  }();
  return on;
}

cudaStream_t alloc_stream() { return tl_alloc_stream; }

void keep_pool_memory() {
  static std::mutex mu;
  static std::set<int> done;
  int dev = 0;
  DG_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (done.count(dev)) return;
  // memory released to the device's default pool stays there for the next domain instead of
  // being returned at every synchronisation (this process's pool only)
  cudaMemPool_t pool;
  DG_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t keep = UINT64_MAX;
  DG_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
  done.insert(dev);
}
AllocStreamScope::AllocStreamScope(cudaStream_t s) : prev(tl_alloc_stream) { tl_alloc_stream = s; }
AllocStreamScope::~AllocStreamScope() { tl_alloc_stream = prev; }

// Off by default for every launch: measured on the 8^3, N = 8 workload it slowed the FP64 solve
// from 339 to 630 ms (dependent CTAs parked on the SMs during the long FP64 GEMMs) and the mixed one
// from 5.55 to 5.78 ms. DG_PDL=1 turns it on everywhere; a PdlScope turns it on for the launches
// made inside it on this thread (the coarse levels of the V-cycle, see schwarz_smooth).
namespace {
thread_local int tl_pdl_scope = 0;
}
bool pdl_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("DG_PDL");
    return v && std::strcmp(v, "1") == 0;
  }();
  return on || tl_pdl_scope > 0;
}
PdlScope::PdlScope(bool on_) : on(on_) {
  if (on) ++tl_pdl_scope;
}
PdlScope::~PdlScope() {
  if (on) --tl_pdl_scope;
}
// Off unless DG_PDL_KRYLOV=1: on the 8^3, N = 8 workload it gained 0.4 % for one solve at a time
// (194.0 -> 194.8 solves/s) but cost concurrent solves much more (a 512-solve batched graph 600 ->
// 516 solves/s, 8 streams 370 -> 341): the next vector kernel's ~1200 CTAs wait on the SMs that
// other solves' kernels would use.
bool pdl_krylov_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("DG_PDL_KRYLOV");
    return v && std::strcmp(v, "1") == 0;
  }();
  return on;
}
int pdl_vcycle_mode() {
  static const int mode = [] {
    const char* v = std::getenv("DG_PDL_COARSE");
    return v ? std::atoi(v) : 1;
  }();
  return mode;
}

int autotune(const std::vector<int64_t>& key, const std::vector<int>& candidates,
             const std::function<void(int)>& run, cudaStream_t s) {
  DG_REQUIRE(!candidates.empty(), "autotune needs candidates");
  if (candidates.size() == 1 || !tuning_enabled()) return candidates[0];
  int dev = 0;
  DG_CUDA(cudaGetDevice(&dev));
  std::vector<int64_t> k = key;
  k.push_back(dev);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(k);
    if (it != g_tuned.end()) return it->second;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  DG_CUDA(cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone) return candidates[0];
  cudaEvent_t a = nullptr, b = nullptr;
  DG_CUDA(cudaEventCreate(&a));
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    fail(DG_ERR_CUDA, "cudaEventCreate failed");
  }
  int best = candidates[0];
  float best_ms = std::numeric_limits<float>::infinity();
  std::string timings;
  try {
    for (int c : candidates) {
      run(c);  // warm-up (first launch of a kernel pays for module loading)
      DG_CUDA(cudaEventRecord(a, s));
      for (int r = 0; r < 3; ++r) run(c);
      DG_CUDA(cudaEventRecord(b, s));
      DG_CUDA(cudaEventSynchronize(b));
      float ms = 0.0f;
      DG_CUDA(cudaEventElapsedTime(&ms, a, b));
      timings += " " + std::to_string(c) + ":" + std::to_string(ms / 3.0f * 1e3f);
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
  } catch (...) {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    throw;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (tune_log()) {
    std::string line = "dg autotune key";
    for (int64_t v : key) line += " " + std::to_string(v);
    line += ": picked " + std::to_string(best) + "; us per launch" + timings + "\n";
    std::fputs(line.c_str(), stderr);
  }
  return g_tuned.emplace(k, best).first->second;
}

}  // namespace dg
