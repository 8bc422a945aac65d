// Vector kernels of the FP64 flexible GMRES (Sec. III.B): axpby, precision conversion, and the
// Arnoldi orthogonalisation as blocked classical Gram-Schmidt (one multi-dot and one combined
// update per pass). Every reduction is a fixed-shape two-pass tree (per-block partials, then one
// block per output summing them in order), so results are bitwise reproducible run to run.
#include "internal.h"

namespace dg {

namespace {
constexpr int kDotBlocks = 304;  // 2 x 152 SMs
constexpr int kThreads = 256;

inline int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, 152 * 8)); }
}  // namespace

int multidot_partial_blocks() { return kDotBlocks; }

// y = a x + b y; with b == 0 the old y is not read (it may be uninitialised memory whose bits
// decode as NaN, and 0 * NaN would poison the result)
template <typename T>
__global__ void axpby_kernel(int64_t n, T a, const T* __restrict__ x, T b, T* __restrict__ y) {
  if (b == T(0)) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
      y[i] = a * x[i];
    return;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

template <typename T>
void launch_axpby(int64_t n, T a, const T* x, T b, T* y, cudaStream_t s) {
  if (n == 0) return;
  axpby_kernel<T><<<grid_for(n), kThreads, 0, s>>>(n, a, x, b, y);
  DG_LAUNCHED(1);
}
template void launch_axpby<double>(int64_t, double, const double*, double, double*, cudaStream_t);
template void launch_axpby<float>(int64_t, float, const float*, float, float*, cudaStream_t);

template <typename T>
__global__ void fill_kernel(int64_t n, T v, T* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) y[i] = v;
}

template <typename T>
void launch_fill(int64_t n, T v, T* y, cudaStream_t s) {
  if (n == 0) return;
  fill_kernel<T><<<grid_for(n), kThreads, 0, s>>>(n, v, y);
  DG_LAUNCHED(1);
}
template void launch_fill<double>(int64_t, double, double*, cudaStream_t);

__global__ void d2f_kernel(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
__global__ void f2d_kernel(int64_t n, const float* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}
__global__ void addf2d_kernel(int64_t n, const float* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += (double)x[i];
}
__global__ void mul_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a[i] * b[i];
}

void launch_convert_d2f(int64_t n, const double* x, float* y, cudaStream_t s) {
  if (n == 0) return;
  d2f_kernel<<<grid_for(n), kThreads, 0, s>>>(n, x, y);
  DG_LAUNCHED(1);
}
void launch_convert_f2d(int64_t n, const float* x, double* y, cudaStream_t s) {
  if (n == 0) return;
  f2d_kernel<<<grid_for(n), kThreads, 0, s>>>(n, x, y);
  DG_LAUNCHED(1);
}
void launch_add_f2d(int64_t n, const float* x, double* y, cudaStream_t s) {
  if (n == 0) return;
  addf2d_kernel<<<grid_for(n), kThreads, 0, s>>>(n, x, y);
  DG_LAUNCHED(1);
}
void launch_scale_mul(int64_t n, const double* a, const double* b, double* y, cudaStream_t s) {
  if (n == 0) return;
  mul_kernel<<<grid_for(n), kThreads, 0, s>>>(n, a, b, y);
  DG_LAUNCHED(1);
}

// partial[k * kDotBlocks + bx] = sum over this block's chunk of V_k . w
__global__ void multidot_partial_kernel(int64_t n, const double* __restrict__ V, int64_t ld, const double* __restrict__ w,
                                        double* __restrict__ partial) {
  __shared__ double red[kThreads / 32];
  const int k = blockIdx.y;
  const double* v = V + (int64_t)k * ld;
  const int64_t chunk = (n + kDotBlocks - 1) / kDotBlocks;
  const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  double acc = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += v[i] * w[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += red[q];
    partial[(int64_t)k * kDotBlocks + blockIdx.x] = t;
  }
}

__global__ void multidot_final_kernel(const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double red[kThreads / 32];
  const int k = blockIdx.x;
  double acc = 0.0;
  for (int q = threadIdx.x; q < kDotBlocks; q += blockDim.x) acc += partial[(int64_t)k * kDotBlocks + q];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += red[q];
    out[k] = t;
  }
}

void launch_multidot(int64_t n, int m, const double* V, int64_t ld, const double* w, double* partial, double* out,
                     cudaStream_t s) {
  if (m == 0) return;
  multidot_partial_kernel<<<dim3(kDotBlocks, m), kThreads, 0, s>>>(n, V, ld, w, partial);
  multidot_final_kernel<<<m, kThreads, 0, s>>>(partial, out);
  DG_LAUNCHED(2);
}

__global__ void sub_comb_kernel(int64_t n, int m, const double* __restrict__ V, int64_t ld, const double* __restrict__ h,
                                double* __restrict__ w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = w[i];
    for (int k = 0; k < m; ++k) acc -= h[k] * V[(int64_t)k * ld + i];
    w[i] = acc;
  }
}
__global__ void add_comb_kernel(int64_t n, int m, const double* __restrict__ Z, int64_t ld, const double* __restrict__ y,
                                double* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = x[i];
    for (int k = 0; k < m; ++k) acc += y[k] * Z[(int64_t)k * ld + i];
    x[i] = acc;
  }
}

void launch_subtract_combination(int64_t n, int m, const double* V, int64_t ld, const double* h, double* w,
                                 cudaStream_t s) {
  if (n == 0 || m == 0) return;
  sub_comb_kernel<<<grid_for(n), kThreads, 0, s>>>(n, m, V, ld, h, w);
  DG_LAUNCHED(1);
}
void launch_add_combination(int64_t n, int m, const double* Z, int64_t ld, const double* y, double* x, cudaStream_t s) {
  if (n == 0 || m == 0) return;
  add_comb_kernel<<<grid_for(n), kThreads, 0, s>>>(n, m, Z, ld, y, x);
  DG_LAUNCHED(1);
}

}  // namespace dg
