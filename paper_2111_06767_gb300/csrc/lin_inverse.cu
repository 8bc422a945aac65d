// Per-subdomain explicit inverses of the linearized subdomain matrices A_S + D_S (Sec. III.E's
// explicit-inverse solver applied to the full linearized operator of a nonlinear problem rather
// than to its Laplacian approximation). The Poisson part A_S is shared by all subdomains of a
// boundary-contact class; the diagonal D_S = R_S M S'(u) R_S^T differs per subdomain and per
// linearization, so every linearization assembles E matrices, inverts them in place with the
// batched Gauss-Jordan kernels, and every smoothing step applies them with one batched
// matrix-vector product. Both are HBM streams over E n_S^2 values: the product reads each inverse
// once per smoothing step.
#include <cuda_fp16.h>

#include <algorithm>

#include "internal.h"

namespace dg {

// M_c = A_{class(c)} + diag(d_S[:, c]) for every subdomain column c (compact n_S x n_S). One CTA
// per column, a warp per row, lanes along the row.
template <typename T>
__global__ void __launch_bounds__(256) lin_assemble_kernel(const T* __restrict__ A, const int* __restrict__ class_of_col,
                                                           const T* __restrict__ dS, int nS, int ld,
                                                           T* __restrict__ M) {
  const int c = blockIdx.x;
  const size_t n2 = (size_t)nS * nS;
  const T* a = A + (size_t)class_of_col[c] * n2;
  T* m = M + (size_t)c * n2;
  const T* d = dS + (size_t)c * ld;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int r = warp; r < nS; r += 8) {
    const T dr = d[r];
    const size_t o = (size_t)r * nS;
    for (int j = lane; j < nS; j += 32) m[o + j] = a[o + j] + (j == r ? dr : T(0));
  }
}

template <typename T>
void launch_lin_assemble(const T* A, const int* class_of_col, const T* dS, int nS, int ld, int E, T* M,
                         cudaStream_t s) {
  if (E == 0) return;
  lin_assemble_kernel<T><<<E, 256, 0, s>>>(A, class_of_col, dS, nS, ld, M);
  DG_LAUNCHED(1);
}

template <typename T, int V>
struct VecOf;
template <>
struct VecOf<float, 4> { using type = float4; };
template <>
struct VecOf<double, 2> { using type = double2; };
template <typename T>
struct VecOf<T, 1> { using type = T; };

template <typename T>
__device__ __forceinline__ T dot_vec(const T& a, const T& b) { return a * b; }
__device__ __forceinline__ float dot_vec(const float4& a, const float4& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}
__device__ __forceinline__ double dot_vec(const double2& a, const double2& b) { return a.x * b.x + a.y * b.y; }

// du_S[:, c] = Minv_c r_S[:, c] for rows [r0, r1) of every column: grid (E, row splits), a warp
// per group of R rows with the lanes along the rows (V values per load; rows of V-aligned length),
// one warp reduction per row. The inverses are streamed once with no reuse: loads bypass L1.
template <typename T, int V, int R>
__global__ void __launch_bounds__(256) lin_gemv_kernel(const T* __restrict__ Minv, const T* __restrict__ rS, int nS,
                                                       int ld, int rows_per_split, T* __restrict__ duS) {
  using VT = typename VecOf<T, V>::type;
  const int c = blockIdx.x;
  const int r0 = blockIdx.y * rows_per_split, r1 = min(nS, r0 + rows_per_split);
  const T* m = Minv + (size_t)c * nS * nS;
  const VT* x = reinterpret_cast<const VT*>(rS + (size_t)c * ld);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nv = nS / V;
  for (int rb = r0 + warp * R; rb < r1; rb += 8 * R) {
    T acc[R];
#pragma unroll
    for (int q = 0; q < R; ++q) acc[q] = T(0);
    for (int j = lane; j < nv; j += 32) {
      const VT xv = x[j];
#pragma unroll
      for (int q = 0; q < R; ++q)
        if (rb + q < r1) acc[q] += dot_vec(__ldcs(reinterpret_cast<const VT*>(m + (size_t)(rb + q) * nS) + j), xv);
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    }
    if (lane < R && rb + lane < r1) {
      T v = acc[0];
#pragma unroll
      for (int q = 1; q < R; ++q)
        if (lane == q) v = acc[q];
      duS[(size_t)c * ld + rb + lane] = v;
    }
  }
}

template <typename T>
void launch_lin_gemv(const T* Minv, const T* rS, int nS, int ld, int E, T* duS, cudaStream_t s) {
  if (E == 0) return;
  int dev = 0, n_sm = 0;
  DG_CUDA(cudaGetDevice(&dev));
  DG_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  // enough CTAs to fill the GPU (8 per SM) when the subdomains are few, with >= 64 rows each
  const int want = std::max(1, (8 * n_sm + E - 1) / E);
  const int splits = std::max(1, std::min(want, nS / 64));
  const int rps = (nS + splits - 1) / splits;
  const dim3 grid(E, splits);
  constexpr int VV = 16 / sizeof(T);
  const bool vec = nS % VV == 0 && ld % VV == 0 && (reinterpret_cast<uintptr_t>(Minv) % 16) == 0 &&
                   (reinterpret_cast<uintptr_t>(rS) % 16) == 0;
  if (vec) lin_gemv_kernel<T, VV, 4><<<grid, 256, 0, s>>>(Minv, rS, nS, ld, rps, duS);
  else lin_gemv_kernel<T, 1, 4><<<grid, 256, 0, s>>>(Minv, rS, nS, ld, rps, duS);
  DG_LAUNCHED(1);
}

// FP16 copies of per-subdomain inverses for the MIXED curved smoother: every matrix is divided by
// its largest magnitude (kept in scale[c]) and rounded to FP16, whose 11-bit significand matches the
// TF32 inputs of the tensor-core GEMM used for the shared class inverses; products accumulate in
// FP32 and are rescaled.
__global__ void __launch_bounds__(256) to_half_kernel(const float* __restrict__ src, int64_t n2,
                                                      uint16_t* __restrict__ dst, float* __restrict__ scale) {
  __shared__ float red[8];
  const int c = blockIdx.x;
  const float* a = src + (size_t)c * n2;
  float m = 0.f;
  for (int64_t t = threadIdx.x; t < n2; t += blockDim.x) m = fmaxf(m, fabsf(a[t]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  m = 0.f;
  for (int q = 0; q < 8; ++q) m = fmaxf(m, red[q]);
  const float inv = m > 0.f ? 1.f / m : 0.f;
  __half* d = reinterpret_cast<__half*>(dst) + (size_t)c * n2;
  for (int64_t t = threadIdx.x; t < n2; t += blockDim.x) d[t] = __float2half_rn(a[t] * inv);
  if (threadIdx.x == 0) scale[c] = m;
}

void launch_to_half_scaled(const float* src, int nS, int E, uint16_t* dst, float* scale, cudaStream_t s) {
  if (E == 0) return;
  to_half_kernel<<<E, 256, 0, s>>>(src, (int64_t)nS * nS, dst, scale);
  DG_LAUNCHED(1);
}

// du_S[:, c] = scale[c] (Minv16_c r_S[:, c]): as lin_gemv_kernel with FP16 matrix entries (eight
// per 16-byte load when the rows allow it) and FP32 vectors and sums.
template <int V, int R>
__global__ void __launch_bounds__(256) lin_gemv_half_kernel(const uint16_t* __restrict__ Minv,
                                                            const float* __restrict__ scale,
                                                            const float* __restrict__ rS, int nS, int ld,
                                                            int rows_per_split, float* __restrict__ duS) {
  const int c = blockIdx.x;
  const int r0 = blockIdx.y * rows_per_split, r1 = min(nS, r0 + rows_per_split);
  const __half* m = reinterpret_cast<const __half*>(Minv) + (size_t)c * nS * nS;
  const float* x = rS + (size_t)c * ld;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nv = nS / V;
  for (int rb = r0 + warp * R; rb < r1; rb += 8 * R) {
    float acc[R];
#pragma unroll
    for (int q = 0; q < R; ++q) acc[q] = 0.f;
    for (int j = lane; j < nv; j += 32) {
      if constexpr (V == 8) {
        const float4 x0 = reinterpret_cast<const float4*>(x)[2 * j], x1 = reinterpret_cast<const float4*>(x)[2 * j + 1];
#pragma unroll
        for (int q = 0; q < R; ++q) {
          if (rb + q >= r1) continue;
          const uint4 raw = __ldcs(reinterpret_cast<const uint4*>(m + (size_t)(rb + q) * nS) + j);
          const __half2* h = reinterpret_cast<const __half2*>(&raw);
          const float2 f0 = __half22float2(h[0]), f1 = __half22float2(h[1]);
          const float2 f2 = __half22float2(h[2]), f3 = __half22float2(h[3]);
          acc[q] += f0.x * x0.x + f0.y * x0.y + f1.x * x0.z + f1.y * x0.w + f2.x * x1.x + f2.y * x1.y +
                    f3.x * x1.z + f3.y * x1.w;
        }
      } else {
        const float xv = x[j];
#pragma unroll
        for (int q = 0; q < R; ++q)
          if (rb + q < r1) acc[q] += __half2float(m[(size_t)(rb + q) * nS + j]) * xv;
      }
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    }
    if (lane < R && rb + lane < r1) {
      float v = acc[0];
#pragma unroll
      for (int q = 1; q < R; ++q)
        if (lane == q) v = acc[q];
      duS[(size_t)c * ld + rb + lane] = scale[c] * v;
    }
  }
}

void launch_lin_gemv_half(const uint16_t* Minv, const float* scale, const float* rS, int nS, int ld, int E,
                          float* duS, cudaStream_t s) {
  if (E == 0) return;
  int dev = 0, n_sm = 0;
  DG_CUDA(cudaGetDevice(&dev));
  DG_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  const int want = std::max(1, (8 * n_sm + E - 1) / E);
  const int splits = std::max(1, std::min(want, nS / 64));
  const int rps = (nS + splits - 1) / splits;
  const dim3 grid(E, splits);
  const bool vec = nS % 8 == 0 && ld % 8 == 0 && (reinterpret_cast<uintptr_t>(Minv) % 16) == 0 &&
                   (reinterpret_cast<uintptr_t>(rS) % 32) == 0;
  if (vec) lin_gemv_half_kernel<8, 4><<<grid, 256, 0, s>>>(Minv, scale, rS, nS, ld, rps, duS);
  else lin_gemv_half_kernel<1, 4><<<grid, 256, 0, s>>>(Minv, scale, rS, nS, ld, rps, duS);
  DG_LAUNCHED(1);
}

template void launch_lin_assemble<double>(const double*, const int*, const double*, int, int, int, double*,
                                          cudaStream_t);
template void launch_lin_assemble<float>(const float*, const int*, const float*, int, int, int, float*, cudaStream_t);
template void launch_lin_gemv<double>(const double*, const double*, int, int, int, double*, cudaStream_t);
template void launch_lin_gemv<float>(const float*, const float*, int, int, int, float*, cudaStream_t);

}  // namespace dg
