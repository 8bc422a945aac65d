// Whole-line vector moves for element-major data: a line is N consecutive values of one element
// (u[e][k][j][0..N-1] and the like), moved in 16-, 8- or scalar-byte pieces as N sizeof(T) allows.
#pragma once

#include <cuda_runtime.h>

namespace dg {

// Vector width for moving one line of N values of type T: 16 bytes where N sizeof(T) allows it,
// else 8, else scalar. Element blocks are N^3 values and lines N values, so every line of a
// 16-byte aligned buffer starts on that width.
template <typename T, int W>
struct VT;
template <>
struct VT<float, 16> { using type = float4; };
template <>
struct VT<float, 8> { using type = float2; };
template <>
struct VT<float, 4> { using type = float; };
template <>
struct VT<double, 16> { using type = double2; };
template <>
struct VT<double, 8> { using type = double; };
template <>
struct VT<int, 16> { using type = int4; };
template <>
struct VT<int, 8> { using type = int2; };
template <>
struct VT<int, 4> { using type = int; };

template <int N, typename T>
struct LineVec {
  static constexpr int bytes = N * (int)sizeof(T);
  static constexpr int w = bytes % 16 == 0 ? 16 : (bytes % 8 == 0 ? 8 : (int)sizeof(T));
  static constexpr int per = w / (int)sizeof(T);
  static constexpr int n = N / per;
  using V = typename VT<T, w>::type;
};

// L2ONLY: load through L2 only (ld.global.cg), for data that other CTAs of the same kernel wrote
// after a grid-wide barrier; otherwise the read-only path (data constant during the kernel).
template <int N, typename T, bool L2ONLY = false>
__device__ __forceinline__ void gld_line(const T* __restrict__ p, T (&v)[N]) {
  using L = LineVec<N, T>;
#pragma unroll
  for (int q = 0; q < L::n; ++q) {
    const typename L::V* vp = reinterpret_cast<const typename L::V*>(p) + q;
    const typename L::V x = L2ONLY ? __ldcg(vp) : __ldg(vp);
    const T* xs = reinterpret_cast<const T*>(&x);
#pragma unroll
    for (int r = 0; r < L::per; ++r) v[q * L::per + r] = xs[r];
  }
}

template <int N, typename T>
__device__ __forceinline__ void gst_line(T* __restrict__ p, const T (&v)[N]) {
  using L = LineVec<N, T>;
#pragma unroll
  for (int q = 0; q < L::n; ++q) {
    typename L::V x;
    T* xs = reinterpret_cast<T*>(&x);
#pragma unroll
    for (int r = 0; r < L::per; ++r) xs[r] = v[q * L::per + r];
    reinterpret_cast<typename L::V*>(p)[q] = x;
  }
}

template <int N, typename T>
__device__ __forceinline__ void sld_line(const T* p, T (&v)[N]) {
  using L = LineVec<N, T>;
#pragma unroll
  for (int q = 0; q < L::n; ++q) {
    const typename L::V x = reinterpret_cast<const typename L::V*>(p)[q];
    const T* xs = reinterpret_cast<const T*>(&x);
#pragma unroll
    for (int r = 0; r < L::per; ++r) v[q * L::per + r] = xs[r];
  }
}

template <int N, typename T>
__device__ __forceinline__ void sst_line(T* p, const T (&v)[N]) {
  using L = LineVec<N, T>;
#pragma unroll
  for (int q = 0; q < L::n; ++q) {
    typename L::V x;
    T* xs = reinterpret_cast<T*>(&x);
#pragma unroll
    for (int r = 0; r < L::per; ++r) xs[r] = v[q * L::per + r];
    reinterpret_cast<typename L::V*>(p)[q] = x;
  }
}

}  // namespace dg
