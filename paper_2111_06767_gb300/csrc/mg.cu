// Multigrid intermesh operators (Sec. III.C.2).
//
// Prolongation (Eq. prol): Lagrange interpolation from the parent's LGL points to each child's
// points at parent-logical coordinates (xi - 1)/2 (lower half), (xi + 1)/2 (upper half) or xi
// (the child spans the parent in that dimension). Restriction R = P^T (no mass matrices, since
// it acts on DG residuals that already carry them). Both are sum-factorised: three 1-D passes of
// N^4 work per element, one CTA per element (at most 512 threads), data staged in shared memory. The restriction
// gathers its (up to 8) children in a fixed order: deterministic, no atomics; up to N = 8 (one
// point per thread) it reads all children's values before the first pass.
#include "internal.h"
#include "pdl.cuh"

namespace dg {

struct XferGeom {
  int nf[3], nc[3];
};

// per dimension: which half a fine coordinate is in (0 lower, 1 upper, 2 full) and its parent
__device__ __forceinline__ void parent_of(int cf, int nf, int nc, int& pc, int& half) {
  if (nf == nc) { pc = cf; half = 2; }
  else { pc = cf >> 1; half = cf & 1; }
}

template <int N, typename T>
__device__ __forceinline__ T interp(const T* sI, int half, int t, int j) {
  // sI: [2][N*N] lower/upper interpolation matrices; half 2 = identity
  return half == 2 ? (t == j ? T(1) : T(0)) : sI[half * N * N + t * N + j];
}

template <int N>
struct XferShape {
  static constexpr int n3 = N * N * N;
  static constexpr int threads = n3 > 512 ? 512 : n3;
};

template <int N, typename T>
__global__ void __launch_bounds__(XferShape<N>::threads) prolongate_kernel(XferGeom x, const T* __restrict__ Ilo,
                                                                           const T* __restrict__ Ihi,
                                                                           const T* __restrict__ uc,
                                                                           T* __restrict__ uf) {
  constexpr int N2 = N * N, N3 = N2 * N, NT = XferShape<N>::threads;
  __shared__ T sI[2 * N2];
  __shared__ T s0[N3], s1[N3];
  const int ef = blockIdx.x;
  const int tid = threadIdx.x;
  for (int t = tid; t < N2; t += NT) { sI[t] = Ilo[t]; sI[N2 + t] = Ihi[t]; }
  const int cx = ef % x.nf[0], cy = (ef / x.nf[0]) % x.nf[1], cz = ef / (x.nf[0] * x.nf[1]);
  int px, py, pz, hx, hy, hz;
  parent_of(cx, x.nf[0], x.nc[0], px, hx);
  parent_of(cy, x.nf[1], x.nc[1], py, hy);
  parent_of(cz, x.nf[2], x.nc[2], pz, hz);
  const int ec = px + x.nc[0] * (py + x.nc[1] * pz);
  pdl_launch_dependents();
  pdl_wait();
  for (int t = tid; t < N3; t += NT) s0[t] = uc[(int64_t)ec * N3 + t];
  __syncthreads();
  for (int t = tid; t < N3; t += NT) {  // along x: s1[c][b][i] = sum_a Ix[i][a] uc[c][b][a]
    const int i = t % N, j = (t / N) % N, k = t / N2;
    T a = 0;
#pragma unroll
    for (int l = 0; l < N; ++l) a += interp<N, T>(sI, hx, i, l) * s0[(k * N + j) * N + l];
    s1[t] = a;
  }
  __syncthreads();
  for (int t = tid; t < N3; t += NT) {  // along y
    const int i = t % N, j = (t / N) % N, k = t / N2;
    T a = 0;
#pragma unroll
    for (int l = 0; l < N; ++l) a += interp<N, T>(sI, hy, j, l) * s1[(k * N + l) * N + i];
    s0[t] = a;
  }
  __syncthreads();
  for (int t = tid; t < N3; t += NT) {  // along z
    const int i = t % N, j = (t / N) % N, k = t / N2;
    T a = 0;
#pragma unroll
    for (int l = 0; l < N; ++l) a += interp<N, T>(sI, hz, k, l) * s0[(l * N + j) * N + i];
    uf[(int64_t)ef * N3 + t] += a;
  }
}

template <int N, typename T>
__global__ void __launch_bounds__(XferShape<N>::threads) restrict_kernel(XferGeom x, const T* __restrict__ Ilo,
                                                                         const T* __restrict__ Ihi,
                                                                         const T* __restrict__ rf,
                                                                         T* __restrict__ bc) {
  constexpr int N2 = N * N, N3 = N2 * N, NT = XferShape<N>::threads;
  __shared__ T sI[2 * N2];
  __shared__ T s0[N3], s1[N3], sacc[N3];
  const int ec = blockIdx.x;
  const int tid = threadIdx.x;
  for (int t = tid; t < N2; t += NT) { sI[t] = Ilo[t]; sI[N2 + t] = Ihi[t]; }
  for (int t = tid; t < N3; t += NT) sacc[t] = T(0);
  const int px = ec % x.nc[0], py = (ec / x.nc[0]) % x.nc[1], pz = ec / (x.nc[0] * x.nc[1]);
  const int rx = x.nf[0] == x.nc[0] ? 1 : 2, ry = x.nf[1] == x.nc[1] ? 1 : 2, rz = x.nf[2] == x.nc[2] ? 1 : 2;
  const int nch = rx * ry * rz;
  // child c (x fastest) of the parent: its element index and the half it occupies per dimension
  auto child = [&](int c, int& ef, int& hx, int& hy, int& hz) {
    const int dx = c % rx, dy = (c / rx) % ry, dz = c / (rx * ry);
    const int cx = rx == 2 ? 2 * px + dx : px, cy = ry == 2 ? 2 * py + dy : py, cz = rz == 2 ? 2 * pz + dz : pz;
    hx = rx == 2 ? dx : 2;
    hy = ry == 2 ? dy : 2;
    hz = rz == 2 ? dz : 2;
    ef = cx + x.nf[0] * (cy + x.nf[1] * cz);
  };
  pdl_launch_dependents();
  pdl_wait();
  // one point per thread (N <= 8): every child's value is read up front, so the children cost one
  // round trip to memory instead of one each
  constexpr bool kPre = N3 <= NT;
  T pre[8];
  if constexpr (kPre) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      int ef, hx, hy, hz;
      child(c < nch ? c : 0, ef, hx, hy, hz);
      pre[c] = c < nch && tid < N3 ? rf[(int64_t)ef * N3 + tid] : T(0);
    }
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (c >= nch) break;
    int ef, hx, hy, hz;
    child(c, ef, hx, hy, hz);
    __syncthreads();
    if constexpr (kPre) {
      if (tid < N3) s0[tid] = pre[c];
    } else {
      for (int t = tid; t < N3; t += NT) s0[t] = rf[(int64_t)ef * N3 + t];
    }
    __syncthreads();
    for (int t = tid; t < N3; t += NT) {  // s1[k][j][a] = sum_i Ix[i][a] r[k][j][i]
      const int i = t % N, j = (t / N) % N, k = t / N2;
      T a = 0;
#pragma unroll
      for (int l = 0; l < N; ++l) a += interp<N, T>(sI, hx, l, i) * s0[(k * N + j) * N + l];
      s1[t] = a;
    }
    __syncthreads();
    for (int t = tid; t < N3; t += NT) {  // s0[k][b][a] = sum_j Iy[j][b] s1[k][j][a]
      const int i = t % N, j = (t / N) % N, k = t / N2;
      T a = 0;
#pragma unroll
      for (int l = 0; l < N; ++l) a += interp<N, T>(sI, hy, l, j) * s1[(k * N + l) * N + i];
      s0[t] = a;
    }
    __syncthreads();
    for (int t = tid; t < N3; t += NT) {  // sum_k Iz[k][c] s0[k][b][a]
      const int i = t % N, j = (t / N) % N, k = t / N2;
      T a = 0;
#pragma unroll
      for (int l = 0; l < N; ++l) a += interp<N, T>(sI, hz, l, k) * s0[(l * N + j) * N + i];
      sacc[t] += a;
    }
  }
  __syncthreads();
  for (int t = tid; t < N3; t += NT) bc[(int64_t)ec * N3 + t] = sacc[t];
}

template <typename T>
void launch_prolongate_add(int N, const int nf[3], const int nc[3], const T* Ilo, const T* Ihi, const T* uc, T* uf,
                           cudaStream_t s) {
  XferGeom x{{nf[0], nf[1], nf[2]}, {nc[0], nc[1], nc[2]}};
  const int E = nf[0] * nf[1] * nf[2];
  switch (N) {
#define DG_CASE(NN) \
  case NN: launch_pdl(prolongate_kernel<NN, T>, dim3(E), dim3(XferShape<NN>::threads), 0, s, x, Ilo, Ihi, uc, uf); break;
    DG_CASE(2) DG_CASE(3) DG_CASE(4) DG_CASE(5) DG_CASE(6) DG_CASE(7) DG_CASE(8) DG_CASE(9) DG_CASE(10)
#undef DG_CASE
    default: fail(DG_ERR_INVALID_ARG, "unsupported N");
  }
  DG_LAUNCHED(1);
}

template <typename T>
void launch_restrict(int N, const int nf[3], const int nc[3], const T* Ilo, const T* Ihi, const T* rf, T* bc,
                     cudaStream_t s) {
  XferGeom x{{nf[0], nf[1], nf[2]}, {nc[0], nc[1], nc[2]}};
  const int E = nc[0] * nc[1] * nc[2];
  switch (N) {
#define DG_CASE(NN) \
  case NN: launch_pdl(restrict_kernel<NN, T>, dim3(E), dim3(XferShape<NN>::threads), 0, s, x, Ilo, Ihi, rf, bc); break;
    DG_CASE(2) DG_CASE(3) DG_CASE(4) DG_CASE(5) DG_CASE(6) DG_CASE(7) DG_CASE(8) DG_CASE(9) DG_CASE(10)
#undef DG_CASE
    default: fail(DG_ERR_INVALID_ARG, "unsupported N");
  }
  DG_LAUNCHED(1);
}

template void launch_prolongate_add<double>(int, const int*, const int*, const double*, const double*, const double*,
                                            double*, cudaStream_t);
template void launch_prolongate_add<float>(int, const int*, const int*, const float*, const float*, const float*,
                                           float*, cudaStream_t);
template void launch_restrict<double>(int, const int*, const int*, const double*, const double*, const double*,
                                      double*, cudaStream_t);
template void launch_restrict<float>(int, const int*, const int*, const float*, const float*, const float*, float*,
                                     cudaStream_t);

}  // namespace dg
