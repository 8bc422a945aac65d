// Allocation-free inner products for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need these inner products: code
// running while a CUDA stream is being captured into a graph (allocation is not a capturable
// operation), serving or real-time loops whose device memory is fixed up front by a pool or an
// external allocator, and plugins embedded in a host that owns every allocation. They call
// dg_dot_noalloc, which computes the same deterministic two-pass reduction as dg_dot but keeps
// its per-block partial sums in a fixed file-scope device array instead of a domain workspace.
//
// The array is ordinary module memory: every GPU that loads this library holds its
// 304 x DG_NOALLOC_MAX_VECTORS doubles until the process exits. In host code its name is only a
// host-side stand-in, so its device address is looked up with cudaGetSymbolAddress once per device,
// with that device current, on that device's first call, and kept for the life of the process: a
// cudaDeviceReset after that first call would leave the kept address pointing into a destroyed
// context, so callers of this entry point must not reset the device.
#include <mutex>

#include "internal.h"

namespace {

constexpr int kMaxDevices = 64;
constexpr int kPartialBlocks = 304;  // blocks of the first reduction pass (multidot_partial_blocks)
constexpr int kPartials = kPartialBlocks * DG_NOALLOC_MAX_VECTORS;

static __device__ __align__(256) double g_noalloc_partials[kPartials];

std::mutex g_mu;
double* g_ptr[kMaxDevices] = {};

dg_status noalloc_fail(dg_status st, const std::string& msg) {
  dg::set_null_handle_error(msg);
  return st;
}

}  // namespace

extern "C" dg_status dg_dot_noalloc(int64_t n, int32_t m, const double* V, int64_t ld, const double* w, double* out,
                                    void* stream) {
  if (m < 1 || m > DG_NOALLOC_MAX_VECTORS)
    return noalloc_fail(DG_ERR_INVALID_ARG, "dg_dot_noalloc: m must be in [1, DG_NOALLOC_MAX_VECTORS = " +
                                                std::to_string(DG_NOALLOC_MAX_VECTORS) + "], got " + std::to_string(m));
  if (n < 0 || ld < n) return noalloc_fail(DG_ERR_INVALID_ARG, "dg_dot_noalloc: need 0 <= n <= ld");
  if (!V || !w || !out) return noalloc_fail(DG_ERR_INVALID_ARG, "dg_dot_noalloc: null pointer");
  if (dg::multidot_partial_blocks() != kPartialBlocks)
    return noalloc_fail(DG_ERR_INVALID_ARG, "dg_dot_noalloc: reduction shape mismatch");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return noalloc_fail(DG_ERR_CUDA, std::string("cudaGetDevice failed: ") + cudaGetErrorString(e));
  }
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(DG_ERR_INVALID_ARG, "dg_dot_noalloc: device index too large");
  double* partial = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
      // first call on this device (the current one): resolve the array's device address
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_partials);
      if (e != cudaSuccess || !p) {
        (void)cudaGetLastError();
        return noalloc_fail(DG_ERR_CUDA, std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      }
      g_ptr[dev] = static_cast<double*>(p);
    }
    partial = g_ptr[dev];
  }
  try {
    // every partial slot the final pass reads is written by the first pass of the same call,
    // so nothing has to be cleared between calls
    dg::launch_multidot(n, m, V, ld, w, partial, out, (cudaStream_t)stream);
  } catch (const dg::Error& err) {
    return noalloc_fail(err.status, err.message);
  }
  dg::set_null_handle_error("");
  return DG_OK;
}
