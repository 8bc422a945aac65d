// Debug builds (compiled with -DDG_BOUNDS_CHECK: `python paper_2111_06767_gb300/build.py --debug`,
// loaded with DG_DEBUG_BUILD=1): the indices that come from set-up tables (subdomain point maps,
// orientation maps, column maps) are checked against the size of the buffer they index before the
// access they feed. An index out of range is not used (the access is skipped, nothing traps) and
// the first offending source line is recorded in a per-module device word, which
// dg_debug_bounds_check() reads and clears. In the release build the checks compile away.
#pragma once

#include <cuda_runtime.h>

namespace dg {

#ifdef DG_BOUNDS_CHECK
static __device__ int g_oob_line;

__device__ __forceinline__ bool in_bounds(long long i, long long n, int line) {
  if (i >= 0 && i < n) return true;
  atomicCAS(&g_oob_line, 0, line);
  return false;
}
#define DG_IN_BOUNDS(i, n) ::dg::in_bounds((long long)(i), (long long)(n), __LINE__)

// Every translation unit that checks registers a reader of its own word (read and cleared).
int register_oob_reader(int (*reader)());
static int read_and_clear_oob_line() {
  int v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_oob_line, sizeof(int)) != cudaSuccess) return 0;
  cudaMemcpyToSymbol(g_oob_line, &z, sizeof(int));
  return v;
}
static const int g_oob_reader_id = register_oob_reader(&read_and_clear_oob_line);
#else
#define DG_IN_BOUNDS(i, n) true
#endif

}  // namespace dg
