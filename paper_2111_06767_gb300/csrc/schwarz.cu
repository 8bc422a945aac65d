// Additive Schwarz kernels (Sec. III.D) and the explicit-inverse subdomain solver (Sec. III.E).
//
//  * build:   A_S = R_S A R_S^T column by column: column q is the DG operator applied to the unit
//             vector of subdomain point q on the patch (central element + face neighbours), with
//             zero data outside S (Eq. schwarz_subd_problem). One CTA (<= 512 threads) per column.
//  * invert:  in-place Gauss-Jordan without pivoting (A_S is a principal submatrix of the SPD
//             operator, hence SPD), batched over subdomain classes. Setup only.
//  * gather:  r_S = R_S r into class-ordered columns of n_S values (zero at padding).
//  * gemm:    du_S = A_S^-1 r_S for all subdomains of a class at once: one [n_S x n_S] x [n_S x m]
//             product per class (the dense contraction of the smoother).
//  * scatter: u += sum_S R_S^T (w_S du_S) (Eq. schwarz_weighting) as a gather per destination
//             point over its own subdomain and at most 6 face neighbours' subdomains:
//             deterministic, atomic-free.
//
// Subdomain point order (in the subdomain's canonical orientation, see setup.cu): the central
// element's N^3 points (element order), then for faces f = 2 d + side the neighbour's N_overlap
// layers counted from the shared face, each layer in (a2, a1) order of the tangential indices.
// Missing neighbours keep their slots as padding (identity rows and columns in A_S, zero data),
// so every subdomain has n_S = N^3 + 6 N_ov N^2.
#include <limits>

#include "internal.h"
#include "pdl.cuh"
#include "schwarz_dev.cuh"

namespace dg {

// ------------------------------------------------------------------ A_S columns

// Patch description per class: for slot s in 0..6 (0 = centre, 1 + f = neighbour across face f)
// info[s*6 + f'] = face type of that slot's face f': >= 0 slot inside the patch, -1 Dirichlet box
// face, -2 internal face with zero data outside the patch, -3 Neumann box face; info[42 + s] = slot
// exists.
constexpr int kPatchInts = 49;

template <int N>
struct ColumnShape {
  static constexpr int n3 = N * N * N;
  static constexpr int threads = n3 > 512 ? 512 : n3;
};

template <int N, typename T>
__global__ void __launch_bounds__(ColumnShape<N>::threads) subdomain_column_kernel(
    const OpGeom<T> g, const T* __restrict__ Dg, const T* __restrict__ wg,
    const int* __restrict__ patch_info, int ov, int nS, T* __restrict__ A_out) {
  constexpr int N2 = N * N, N3 = N * N * N, NT = ColumnShape<N>::threads;
  __shared__ T sD[N2];
  __shared__ T sw[N];
  __shared__ T su[N3];
  __shared__ T sv[3][N3];
  __shared__ T sfb[6][N2];
  __shared__ int sinfo[kPatchInts];

  const int q = blockIdx.x;  // column
  const int cls = blockIdx.y;
  const int tid = threadIdx.x;
  T* A = A_out + (size_t)cls * nS * nS + (size_t)q * nS;  // column q, contiguous
  for (int t = tid; t < N2; t += NT) sD[t] = Dg[t];
  for (int t = tid; t < N; t += NT) sw[t] = wg[t];
  for (int t = tid; t < kPatchInts; t += NT) sinfo[t] = patch_info[cls * kPatchInts + t];
  __syncthreads();

  // slot and point of the unit entry
  int P, pP;
  if (q < N3) {
    P = 0;
    pP = q;
  } else {
    const int r = q - N3;
    const int f = r / (ov * N2);
    const int rr = r - f * ov * N2;
    const int depth = rr / N2, a2 = (rr / N) % N, a1 = rr % N;
    const int d = f >> 1, side = f & 1;
    P = 1 + f;
    pP = node_of<N>(d, side ? depth : N - 1 - depth, a1, a2);
  }
  if (!sinfo[42 + P]) {  // padding column: identity
    for (int r = tid; r < nS; r += NT) A[r] = (r == q) ? 1.0 : 0.0;
    return;
  }
  for (int r = tid; r < nS; r += NT) A[r] = 0.0;
  __syncthreads();

  for (int X = 0; X < 7; ++X) {
    if (!sinfo[42 + X]) continue;
    for (int p = tid; p < N3; p += NT) su[p] = (X == P && p == pP) ? 1.0 : 0.0;
    __syncthreads();
    for (int p = tid; p < N3; p += NT) {
      const int i = p % N, j = (p / N) % N, k = p / N2;
      T gx = 0, gy = 0, gz = 0;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        gx += sD[i * N + l] * su[(k * N + j) * N + l];
        gy += sD[j * N + l] * su[(k * N + l) * N + i];
        gz += sD[k * N + l] * su[(l * N + j) * N + i];
      }
      sv[0][p] = g.dxi[0] * gx;
      sv[1][p] = g.dxi[1] * gy;
      sv[2][p] = g.dxi[2] * gz;
    }
    __syncthreads();
    for (int item = tid; item < 6 * N2; item += NT) {
      const int f = item / N2, ab = item - f * N2;
      const int a1 = ab % N, a2 = ab / N;
      const int d = f >> 1, side = f & 1;
      const T s = side ? 1.0 : -1.0;
      const T dxi = d == 0 ? g.dxi[0] : (d == 1 ? g.dxi[1] : g.dxi[2]);
      const T lift = d == 0 ? g.lift[0] : (d == 1 ? g.lift[1] : g.lift[2]);
      const T sigma = d == 0 ? g.sigma[0] : (d == 1 ? g.sigma[1] : g.sigma[2]);
      const T Jf = d == 0 ? g.Jf[0] : (d == 1 ? g.Jf[1] : g.Jf[2]);
      const int pf = node_of<N>(d, side ? N - 1 : 0, a1, a2);
      const T u_int = su[pf];
      const T g_int = sv[d][pf];
      const int t = sinfo[X * 6 + f];
      T u_ext, g_ext;
      if (t == -1) {
        u_ext = -u_int;
        g_ext = g_int;
      } else if (t == -2) {
        u_ext = 0.0;
        g_ext = 0.0;
      } else if (t == -3) {  // homogeneous Neumann face of the box
        u_ext = u_int;
        g_ext = -g_int;
      } else {
        // neighbour data is the unit vector restricted to slot t
        const int opp = side ? 0 : N - 1;
        u_ext = (t == P && node_of<N>(d, opp, a1, a2) == pP) ? 1.0 : 0.0;
        T acc = 0.0;
        if (t == P) {
          for (int l = 0; l < N; ++l)
            if (node_of<N>(d, l, a1, a2) == pP) acc += sD[opp * N + l];
        }
        g_ext = dxi * acc;
      }
      const T jump = u_ext - u_int;
      sv[d][pf] = g_int + s * jump * lift;
      const T Bf = Jf * sw[a1] * sw[a2];
      sfb[f][ab] = Bf * (0.5 * s * (g_ext - g_int) + (sigma - lift) * jump);
    }
    __syncthreads();
    for (int p = tid; p < N3; p += NT) {
      const int i = p % N, j = (p / N) % N, k = p / N2;
      T dx = 0, dy = 0, dz = 0;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        dx += sD[i * N + l] * sv[0][(k * N + j) * N + l];
        dy += sD[j * N + l] * sv[1][(k * N + l) * N + i];
        dz += sD[k * N + l] * sv[2][(l * N + j) * N + i];
      }
      const T M = g.J * sw[i] * sw[j] * sw[k];
      T res = -M * (g.dxi[0] * dx + g.dxi[1] * dy + g.dxi[2] * dz);
      if (i == 0) res -= sfb[0][k * N + j];
      if (i == N - 1) res -= sfb[1][k * N + j];
      if (j == 0) res -= sfb[2][k * N + i];
      if (j == N - 1) res -= sfb[3][k * N + i];
      if (k == 0) res -= sfb[4][j * N + i];
      if (k == N - 1) res -= sfb[5][j * N + i];
      const int row = subdomain_row<N>(X, p, ov);
      if (row >= 0) A[row] = res;
    }
    __syncthreads();
  }
}

template <typename T>
void launch_build_subdomain_matrices(int N, int overlap, const OpGeom<T>& g, const T* D, const T* w,
                                     const int* d_patch_info, int n_classes, int nS, T* A_out, cudaStream_t s) {
  dim3 grid(nS, n_classes);
  switch (N) {
#define DG_CASE(NN) \
  case NN: subdomain_column_kernel<NN, T><<<grid, ColumnShape<NN>::threads, 0, s>>>(g, D, w, d_patch_info, overlap, nS, A_out); break;
    DG_CASE(2) DG_CASE(3) DG_CASE(4) DG_CASE(5) DG_CASE(6) DG_CASE(7) DG_CASE(8) DG_CASE(9) DG_CASE(10)
#undef DG_CASE
    default: fail(DG_ERR_INVALID_ARG, "unsupported N");
  }
  DG_LAUNCHED(1);
}
template void launch_build_subdomain_matrices<double>(int, int, const OpGeom<double>&, const double*, const double*,
                                                      const int*, int, int, double*, cudaStream_t);
template void launch_build_subdomain_matrices<float>(int, int, const OpGeom<float>&, const float*, const float*,
                                                     const int*, int, int, float*, cudaStream_t);

// ------------------------------------------------------------------ Gauss-Jordan inversion

// One Gauss-Jordan step on pivot k, reading `in` and writing `out` (ping-pong, so no element is
// overwritten while another thread still needs it):
//   out[k][j] = in[k][j] / in[k][k] (j != k),   out[k][k] = 1 / in[k][k],
//   out[i][j] = in[i][j] - in[i][k] out[k][j] (i != k, j != k),   out[i][k] = -in[i][k] / in[k][k].
// ------------------------------------------------------------------ blocked Gauss-Jordan inversion
//
// In-place inversion of n_classes SPD matrices (n x n, row-major) without pivoting: A_S is a
// principal submatrix of the SPD operator and well conditioned (tens to hundreds for N = 4..8),
// so no pivoting is needed and the FP32 variant loses only ~2 digits. Pivots are processed in
// blocks P of GJB: with X = A[P,P]^-1,
//   A[P,P] <- X,  A[P,Q] <- X A[P,Q],  A[Q,Q] <- A[Q,Q] - A[Q,P] (X A[P,Q]),  A[Q,P] <- -A[Q,P] X
// for Q the complement of P; after the last block A holds A^-1. Every step is a small dense
// product, so the n^3 work runs from shared memory in n / GJB passes instead of n memory-bound
// rank-1 sweeps.

template <typename T>
struct GjbShape {
  static constexpr int B = sizeof(T) == 4 ? 64 : 32;  // pivot block (64 FP32 / 32 FP64 keeps tiles in 48 KB)
};

// X = A[P,P]^-1 in shared memory (one CTA per class).
template <typename T>
__global__ void __launch_bounds__(256) gjb_diag_kernel(T* __restrict__ A, int n, int k0, int bs) {
  constexpr int B = GjbShape<T>::B;
  __shared__ T x[B][B + 1];
  T* a = A + (size_t)blockIdx.x * n * n;
  for (int t = threadIdx.x; t < bs * bs; t += blockDim.x) x[t / bs][t % bs] = a[(size_t)(k0 + t / bs) * n + k0 + t % bs];
  __syncthreads();
  for (int k = 0; k < bs; ++k) {
    const T inv_piv = T(1) / x[k][k];
    // new row k and column k from the old values, then the rank-1 update of the rest
    T rowk = T(0), colk = T(0);
    const int t = threadIdx.x;
    if (t < bs) rowk = (t == k ? T(1) : x[k][t]) * inv_piv;
    T upd[(B * B + 255) / 256];
    int m = 0;
    for (int q = t; q < bs * bs; q += blockDim.x, ++m) {
      const int i = q / bs, j = q % bs;
      upd[m] = (i == k || j == k) ? T(0) : x[i][j] - x[i][k] * x[k][j] * inv_piv;
    }
    if (t < bs) colk = (t == k ? inv_piv : -x[t][k] * inv_piv);
    __syncthreads();
    m = 0;
    for (int q = t; q < bs * bs; q += blockDim.x, ++m) {
      const int i = q / bs, j = q % bs;
      if (i != k && j != k) x[i][j] = upd[m];
    }
    if (t < bs) {
      x[k][t] = rowk;
      if (t != k) x[t][k] = colk;
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < bs * bs; t += blockDim.x) a[(size_t)(k0 + t / bs) * n + k0 + t % bs] = x[t / bs][t % bs];
}

// A[P, j] <- X A[P, j] for 64 columns j outside P (grid: column tiles x classes).
template <typename T>
__global__ void __launch_bounds__(256) gjb_row_kernel(T* __restrict__ A, int n, int k0, int bs) {
  constexpr int B = GjbShape<T>::B;
  __shared__ T x[B][B + 1];
  __shared__ T r[B][64 + 1];
  T* a = A + (size_t)blockIdx.y * n * n;
  const int j0 = blockIdx.x * 64;
  if (j0 >= k0 && j0 + 64 <= k0 + bs) return;  // only pivot columns
  for (int t = threadIdx.x; t < bs * bs; t += blockDim.x) x[t / bs][t % bs] = a[(size_t)(k0 + t / bs) * n + k0 + t % bs];
  for (int t = threadIdx.x; t < bs * 64; t += blockDim.x) {
    const int i = t / 64, j = j0 + t % 64;
    r[i][t % 64] = j < n ? a[(size_t)(k0 + i) * n + j] : T(0);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < bs * 64; t += blockDim.x) {
    const int i = t / 64, jj = t % 64, j = j0 + jj;
    if (j >= n || (j >= k0 && j < k0 + bs)) continue;
    T acc = T(0);
    for (int q = 0; q < bs; ++q) acc += x[i][q] * r[q][jj];
    a[(size_t)(k0 + i) * n + j] = acc;
  }
}

// A[i, j] -= A[i, P] A[P, j] on a 64 x 64 tile with i, j outside P (A[P, j] already X A[P, j]).
template <typename T>
__global__ void __launch_bounds__(256) gjb_update_kernel(T* __restrict__ A, int n, int k0, int bs) {
  constexpr int B = GjbShape<T>::B;
  __shared__ T lt[64][B + 1];
  __shared__ T up[B][64 + 1];
  T* a = A + (size_t)blockIdx.z * n * n;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  if ((i0 >= k0 && i0 + 64 <= k0 + bs) || (j0 >= k0 && j0 + 64 <= k0 + bs)) return;  // only pivot rows or columns
  for (int t = threadIdx.x; t < 64 * bs; t += blockDim.x) {
    const int i = t / bs, q = t % bs;
    lt[i][q] = i0 + i < n ? a[(size_t)(i0 + i) * n + k0 + q] : T(0);
  }
  for (int t = threadIdx.x; t < bs * 64; t += blockDim.x) {
    const int q = t / 64, j = t % 64;
    up[q][j] = j0 + j < n ? a[(size_t)(k0 + q) * n + j0 + j] : T(0);
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 4 x 4 outputs per thread
  T acc[4][4] = {};
  for (int q = 0; q < bs; ++q) {
    T l[4], u[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      l[r] = lt[ty + 16 * r][q];
      u[r] = up[q][tx + 16 * r];
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] += l[r] * u[c];
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = i0 + ty + 16 * r, j = j0 + tx + 16 * c;
      if (i < n && j < n && (i < k0 || i >= k0 + bs) && (j < k0 || j >= k0 + bs)) a[(size_t)i * n + j] -= acc[r][c];
    }
}

// A[i, P] <- -A[i, P] X for 64 rows i outside P.
template <typename T>
__global__ void __launch_bounds__(256) gjb_col_kernel(T* __restrict__ A, int n, int k0, int bs) {
  constexpr int B = GjbShape<T>::B;
  __shared__ T x[B][B + 1];
  __shared__ T c[64][B + 1];
  T* a = A + (size_t)blockIdx.y * n * n;
  const int i0 = blockIdx.x * 64;
  if (i0 >= k0 && i0 + 64 <= k0 + bs) return;  // only pivot rows
  for (int t = threadIdx.x; t < bs * bs; t += blockDim.x) x[t / bs][t % bs] = a[(size_t)(k0 + t / bs) * n + k0 + t % bs];
  for (int t = threadIdx.x; t < 64 * bs; t += blockDim.x) {
    const int i = t / bs, q = t % bs;
    c[i][q] = i0 + i < n ? a[(size_t)(i0 + i) * n + k0 + q] : T(0);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 64 * bs; t += blockDim.x) {
    const int i = t / bs, q = t % bs;
    if (i0 + i >= n || (i0 + i >= k0 && i0 + i < k0 + bs)) continue;
    T acc = T(0);
    for (int p = 0; p < bs; ++p) acc += c[i][p] * x[p][q];
    a[(size_t)(i0 + i) * n + k0 + q] = -acc;
  }
}

template <typename T>
void launch_invert_spd_batched(T* A, int n, int n_classes, cudaStream_t s) {
  if (n_classes == 0 || n == 0) return;
  constexpr int B = GjbShape<T>::B;
  const int nt = (n + 63) / 64;
  int launches = 0;
  for (int k0 = 0; k0 < n; k0 += B) {
    const int bs = std::min(B, n - k0);
    gjb_diag_kernel<T><<<n_classes, 256, 0, s>>>(A, n, k0, bs);
    gjb_row_kernel<T><<<dim3(nt, n_classes), 256, 0, s>>>(A, n, k0, bs);
    gjb_update_kernel<T><<<dim3(nt, nt, n_classes), 256, 0, s>>>(A, n, k0, bs);
    gjb_col_kernel<T><<<dim3(nt, n_classes), 256, 0, s>>>(A, n, k0, bs);
    launches += 4;
  }
  DG_LAUNCHED(launches);
  DG_CUDA(cudaStreamSynchronize(s));
}
template void launch_invert_spd_batched<double>(double*, int, int, cudaStream_t);
template void launch_invert_spd_batched<float>(float*, int, int, cudaStream_t);

// Copy compact [n_classes][n][n] inverses into [n_classes][ld][ld] storage of type T with zero
// padding (ld = n rounded up to 32 so rows are 128-byte aligned for TMA and vector loads).
template <typename S, typename T>
__global__ void pad_convert_kernel(const S* __restrict__ src, int n, int ld, int64_t total, T* __restrict__ dst) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cls = t / ((int64_t)ld * ld);
    const int64_t rem = t - cls * ld * ld;
    const int r = (int)(rem / ld), c = (int)(rem - (int64_t)r * ld);
    dst[t] = (r < n && c < n) ? (T)src[cls * n * n + (int64_t)r * n + c] : T(0);
  }
}

template <typename S, typename T>
void launch_pad_convert(const S* src, int n, int ld, int n_classes, T* dst, cudaStream_t s) {
  const int64_t total = (int64_t)n_classes * ld * ld;
  if (total == 0) return;
  pad_convert_kernel<S, T><<<(int)std::min<int64_t>((total + 255) / 256, 152 * 32), 256, 0, s>>>(src, n, ld, total,
                                                                                                dst);
  DG_LAUNCHED(1);
}
template void launch_pad_convert<double, double>(const double*, int, int, int, double*, cudaStream_t);
template void launch_pad_convert<double, float>(const double*, int, int, int, float*, cudaStream_t);
template void launch_pad_convert<float, float>(const float*, int, int, int, float*, cudaStream_t);


// ------------------------------------------------------------------ gather / scatter


// ------------------------------------------------------------------ table-driven gather / scatter
//
// The point maps depend only on (N, N_overlap) and the subdomain's orientation (48 reflections x
// axis permutations), so they are tabulated once per domain: map[o][q] = (actual slot << 16) |
// actual point for canonical subdomain row q, and its inverse inv[o][slot][p] = canonical row of
// point p of the given actual slot (or -1 outside the subdomain). One CTA per subdomain column
// (gather) or per element (scatter) resolves its neighbours once in shared memory; each point then
// costs one table load instead of a chain of integer divisions.

template <typename T>
__global__ void gather_tab_kernel(SubdomainGeom g, const T* __restrict__ r, const int* __restrict__ elem_of_col,
                                  const int* __restrict__ orient, const int* __restrict__ map, T* __restrict__ rS) {
  pdl_launch_dependents();
  gather_column<T, true>(g, r, elem_of_col, orient, map, rS, blockIdx.x);
}

template <typename T, typename TU>
__global__ void scatter_tab_kernel(SubdomainGeom g, const T* __restrict__ duS, const int* __restrict__ col_of_elem,
                                   const int* __restrict__ orient, const int* __restrict__ inv,
                                   const T* __restrict__ shares, TU* __restrict__ u) {
  pdl_launch_dependents();
  scatter_element<T, TU, true>(g, duS, col_of_elem, orient, inv, shares, u, blockIdx.x);
}

template <typename T>
void launch_gather_tab(const SubdomainGeom& g, const T* r, const int* elem_of_col, const int* orient, const int* map,
                       T* rS, cudaStream_t s) {
  if (g.E == 0) return;
  launch_pdl(gather_tab_kernel<T>, dim3(g.E), dim3(256), 0, s, g, r, elem_of_col, orient, map, rS);
  DG_LAUNCHED(1);
}

template <typename T, typename TU>
void launch_scatter_tab(const SubdomainGeom& g, const T* duS, const int* col_of_elem, const int* orient,
                        const int* inv, const T* shares, TU* u, cudaStream_t s) {
  if (g.E == 0) return;
  const int N3 = g.N * g.N * g.N;
  launch_pdl(scatter_tab_kernel<T, TU>, dim3(g.E), dim3(N3 > 512 ? 512 : (N3 < 32 ? 32 : N3)), 0, s, g, duS,
             col_of_elem, orient, inv, shares, u);
  DG_LAUNCHED(1);
}

template void launch_gather_tab<double>(const SubdomainGeom&, const double*, const int*, const int*, const int*,
                                        double*, cudaStream_t);
template void launch_gather_tab<float>(const SubdomainGeom&, const float*, const int*, const int*, const int*, float*,
                                       cudaStream_t);
template void launch_scatter_tab<double, double>(const SubdomainGeom&, const double*, const int*, const int*,
                                                 const int*, const double*, double*, cudaStream_t);
template void launch_scatter_tab<float, float>(const SubdomainGeom&, const float*, const int*, const int*, const int*,
                                               const float*, float*, cudaStream_t);

// ------------------------------------------------------------------ class GEMM (SIMT)

// Y[:, c0:c0+m] = Inv_c (nS x nS, row-major) * X[:, c0:c0+m] (columns of nS contiguous values).
// 64-row output tiles of 64, 32 or 16 columns (a class's columns are covered with little padding),
// K chunks of 16 staged in shared memory, 4 x (width / 16) outputs per thread. Only the K chunks
// that meet a slot of the subdomain present in the class are read (a missing neighbour's slot has
// zero coupling in the inverse), and tiles whose rows all lie in missing slots only write zeros.
// SPLIT > 1: the K chunks of a tile are split over the SPLIT CTAs of a thread-block cluster (on
// GB300 a single CTA of this FP64 product occupies an SM's FP64 pipe for a long time, so coarse
// levels with few tiles would leave most SMs idle); each CTA keeps its partial tile in shared
// memory and, after a cluster barrier, sums 1/SPLIT of the tile's rows over all partials through
// distributed shared memory in rank order, so the result does not depend on timing.
template <typename T, int SPLIT, int NR>
__device__ __forceinline__ void class_gemm_tile(const T* __restrict__ A, const T* __restrict__ X, T* __restrict__ Y,
                                                int ld, int row0, int col0, int ncol, const int* __restrict__ kl,
                                                int nk, int rank, unsigned char* raw, T alpha) {
  constexpr int BM = 64, BN = 16 * NR, BK = 16;
  T(*sA)[BM + 1] = reinterpret_cast<T(*)[BM + 1]>(raw);
  T(*sB)[BM + 1] = reinterpret_cast<T(*)[BM + 1]>(raw + BK * (BM + 1) * sizeof(T));
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int kc0 = rank * nk / SPLIT, kc1 = (rank + 1) * nk / SPLIT;
  T acc[4][NR] = {};
  // each thread stages 4 values of A and NR of X per K chunk; the next chunk's values are loaded
  // into registers while the current chunk is multiplied
  constexpr int PA = BM * BK / 256, PB = BN * BK / 256;
  T pa[PA], pb[PB];
  auto fetch = [&](int kc) {
    const int k0 = kl[kc] * BK;
#pragma unroll
    for (int q = 0; q < PA; ++q) {
      const int t = threadIdx.x + 256 * q;
      const int r = t / BK, kk = t % BK;
      const int gr = row0 + r, gk = k0 + kk;
      pa[q] = (gr < ld && gk < ld) ? A[(size_t)gr * ld + gk] : T(0);
    }
#pragma unroll
    for (int q = 0; q < PB; ++q) {
      const int t = threadIdx.x + 256 * q;
      const int c = t / BK, kk = t % BK;
      const int gk = k0 + kk;
      pb[q] = (c < ncol && gk < ld) ? X[(size_t)(col0 + c) * ld + gk] : T(0);
    }
  };
  if (kc0 < kc1) fetch(kc0);
  for (int kc = kc0; kc < kc1; ++kc) {
#pragma unroll
    for (int q = 0; q < PA; ++q) {
      const int t = threadIdx.x + 256 * q;
      sA[t % BK][t / BK] = pa[q];
    }
#pragma unroll
    for (int q = 0; q < PB; ++q) {
      const int t = threadIdx.x + 256 * q;
      sB[t % BK][t / BK] = pb[q];
    }
    __syncthreads();
    if (kc + 1 < kc1) fetch(kc + 1);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[NR];
#pragma unroll
      for (int q = 0; q < 4; ++q) a[q] = sA[kk][ty + 16 * q];
#pragma unroll
      for (int r = 0; r < NR; ++r) b[r] = sB[kk][tx + 16 * r];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[q][r] += a[q] * b[r];
    }
    __syncthreads();
  }
  if constexpr (SPLIT == 1) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gr = row0 + ty + 16 * q;
      if (gr >= ld) continue;
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const int c = tx + 16 * r;
        if (c < ncol) Y[(size_t)(col0 + c) * ld + gr] = alpha * acc[q][r];
      }
    }
  } else {
    // partial tile [row][col] in this CTA's shared memory (the staging is free: the K loop ended
    // with a barrier, or never ran)
    T(*part)[64 + 1] = reinterpret_cast<T(*)[64 + 1]>(raw);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int r = 0; r < NR; ++r) part[ty + 16 * q][tx + 16 * r] = acc[q][r];
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    // this CTA sums rows [rank BM / SPLIT, (rank + 1) BM / SPLIT) over the partials in rank order
    constexpr int RPC = BM / SPLIT;
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(&part[0][0]);
    for (int t = threadIdx.x; t < RPC * BN; t += 256) {
      const int rr = rank * RPC + t / BN, c = t % BN;
      const uint32_t off = base + (uint32_t)((rr * (64 + 1) + c) * sizeof(T));
      T sum = T(0);
#pragma unroll
      for (int p = 0; p < SPLIT; ++p) {
        uint32_t remote;
        asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(off), "r"(p));
        T v;
        if constexpr (sizeof(T) == 8) asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(remote));
        else asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(remote));
        sum += v;
      }
      const int gr = row0 + rr;
      if (gr < ld && c < ncol) Y[(size_t)(col0 + c) * ld + gr] = alpha * sum;
    }
    // no CTA leaves while a peer still reads its partial tile
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
  }
}

// tiles: (class | width code << 24 | zero-tile flag << 30, row0, col0, columns of the class from
// col0); kchunks: per class [count, chunk indices...] (ld / 16 + 1 ints per class).
template <typename T, int SPLIT>
__global__ void __launch_bounds__(256) class_gemm_kernel(const T* __restrict__ inv, const T* __restrict__ X,
                                                         T* __restrict__ Y, int ld, const int4* __restrict__ tiles,
                                                         const int* __restrict__ kchunks, T alpha) {
  // the K chunks' staging, then (SPLIT > 1) the partial tile in the same memory
  constexpr size_t kStage = 2 * 16 * (64 + 1) * sizeof(T), kPart = SPLIT > 1 ? 64 * (64 + 1) * sizeof(T) : 0;
  __shared__ __align__(16) unsigned char raw[kStage > kPart ? kStage : kPart];
  const int4 tile = tiles[blockIdx.x / SPLIT];
  const int cls = tile.x & 0xFFFF, wcode = (tile.x >> 24) & 3;
  const bool zero = (tile.x >> 30) & 1;
  const int ncol = min(tile.w, 64 >> wcode);
  const T* A = inv + (size_t)cls * ld * ld;
  const int* kl = kchunks + (size_t)cls * (ld / 16 + 1);
  int rank = 0;
  if constexpr (SPLIT > 1) asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  pdl_launch_dependents();
  pdl_wait();
  const int nk = zero ? 0 : kl[0];
  if (wcode == 0) class_gemm_tile<T, SPLIT, 4>(A, X, Y, ld, tile.y, tile.z, ncol, kl + 1, nk, rank, raw, alpha);
  else if (wcode == 1) class_gemm_tile<T, SPLIT, 2>(A, X, Y, ld, tile.y, tile.z, ncol, kl + 1, nk, rank, raw, alpha);
  else class_gemm_tile<T, SPLIT, 1>(A, X, Y, ld, tile.y, tile.z, ncol, kl + 1, nk, rank, raw, alpha);
}

// K split of the CUDA-core class GEMM: 1, 2, 4 or 8 CTAs per tile (0: the smallest that gives at
// least two CTAs per SM, keeping >= 8 K chunks per CTA).
template <typename T>
void launch_class_gemm_tiles(const T* inv, const T* X, T* Y, int ld, const int4* d_tiles, int n_tiles,
                             const int* d_kchunks, T alpha, cudaStream_t s, int split) {
  if (n_tiles == 0) return;
  DG_REQUIRE(ld % 16 == 0, "class GEMM stride must be a multiple of 16");
  const int nk = ld / 16;
  if (split == 0) {
    split = 1;
    while (split < 8 && n_tiles * split < 2 * 152 && nk / (split * 2) >= 8) split *= 2;
  }
  DG_REQUIRE(split == 1 || split == 2 || split == 4 || split == 8, "class GEMM split must be 1, 2, 4 or 8");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_tiles * split);
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  int na = 0;
  if (pdl_enabled()) {
    at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  if (split > 1) {
    at[na].id = cudaLaunchAttributeClusterDimension;
    at[na].val.clusterDim.x = split;
    at[na].val.clusterDim.y = 1;
    at[na].val.clusterDim.z = 1;
    ++na;
  }
  cfg.attrs = at;
  cfg.numAttrs = na;
  if (split == 1)
    DG_CUDA(cudaLaunchKernelEx(&cfg, class_gemm_kernel<T, 1>, inv, X, Y, ld, d_tiles, d_kchunks, alpha));
  else if (split == 2)
    DG_CUDA(cudaLaunchKernelEx(&cfg, class_gemm_kernel<T, 2>, inv, X, Y, ld, d_tiles, d_kchunks, alpha));
  else if (split == 4)
    DG_CUDA(cudaLaunchKernelEx(&cfg, class_gemm_kernel<T, 4>, inv, X, Y, ld, d_tiles, d_kchunks, alpha));
  else DG_CUDA(cudaLaunchKernelEx(&cfg, class_gemm_kernel<T, 8>, inv, X, Y, ld, d_tiles, d_kchunks, alpha));
  DG_LAUNCHED(1);
}

// ------------------------------------------------------------------ subdomain GMRES (linearized problems)
//
// Sec. III.E: each subdomain problem (A_S + D_S) du_S = r_S of a linearized operator (D_S the
// diagonal linearization term) is solved by GMRES from du_S = 0 for a fixed number of iterations,
// right-preconditioned by the explicit inverse of the Poisson subdomain matrix A_S (the
// Laplacian approximation). With z = A_S^-1 v, (A_S + D_S) z = v + D_S z, so every iteration is
// one class GEMM plus per-subdomain vector work. One warp per subdomain column (8 per CTA): the
// reductions are warp shuffles in a fixed order, with no CTA barrier, and every subdomain of a
// level is resident at once.

constexpr int kSubWarps = 8;  // subdomain columns (warps) per CTA

// Sum over the warp's lanes in a fixed order, returned to every lane.
template <typename T>
__device__ __forceinline__ T warp_total(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}

// 16-byte vector moves of a column's values (the register forms of the kernels below)
template <typename T>
struct SubVec;
template <>
struct SubVec<float> {
  using V = float4;
  static constexpr int E = 4;
  static __device__ __forceinline__ void ld(const float* p, float (&r)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
  }
  static __device__ __forceinline__ void st(float* p, const float (&r)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(r[0], r[1], r[2], r[3]);
  }
};
template <>
struct SubVec<double> {
  static constexpr int E = 2;
  static __device__ __forceinline__ void ld(const double* p, double (&r)[2]) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    r[0] = v.x; r[1] = v.y;
  }
  static __device__ __forceinline__ void st(double* p, const double (&r)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(r[0], r[1]);
  }
};

// V_0 = r_S / ||r_S|| per column; beta[col] = ||r_S||
template <typename T>
__global__ void __launch_bounds__(32 * kSubWarps)
    sub_normalize_kernel(int E, int nS, const T* __restrict__ rS, T* __restrict__ V0, T* __restrict__ beta) {
  const int col = blockIdx.x * kSubWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (col >= E) return;  // whole warps
  const T* r = rS + (size_t)col * nS;
  T acc = 0;
  for (int i = lane; i < nS; i += 32) acc += r[i] * r[i];
  const T nrm = sqrt(warp_total(acc));
  const T inv = nrm > T(0) ? T(1) / nrm : T(0);
  for (int i = lane; i < nS; i += 32) V0[(size_t)col * nS + i] = r[i] * inv;
  if (lane == 0) beta[col] = nrm;
}

// Arnoldi step j: w = V_j + D Z_j, modified Gram-Schmidt against V_0..V_j, V_{j+1} = w / ||w||.
// H is [col][m+1][m]; V and Z are blocks of E*nS values per basis index. w is built in place in
// V_{j+1}; every lane reads back only the entries it wrote.
template <typename T>
__global__ void __launch_bounds__(32 * kSubWarps)
    sub_arnoldi_kernel(int E, int nS, int64_t stride, int j, int m, const T* __restrict__ D, T* V,
                       const T* __restrict__ Z, T* __restrict__ H) {
  const int col = blockIdx.x * kSubWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (col >= E) return;  // whole warps
  const size_t off = (size_t)col * nS;
  const T* vj = V + (size_t)j * stride + off;
  const T* zj = Z + (size_t)j * stride + off;
  T* w = V + (size_t)(j + 1) * stride + off;
  T acc0 = 0;
  for (int i = lane; i < nS; i += 32) {
    const T x = vj[i] + D[off + i] * zj[i];
    w[i] = x;
    acc0 += x * x;
  }
  const T w0 = sqrt(warp_total(acc0));  // ||w|| before orthogonalisation
  T* h = H + (size_t)col * (m + 1) * m;
  for (int i = 0; i <= j; ++i) {
    const T* vi = V + (size_t)i * stride + off;
    T acc = 0;
    for (int t = lane; t < nS; t += 32) acc += w[t] * vi[t];
    const T hij = warp_total(acc);
    for (int t = lane; t < nS; t += 32) w[t] -= hij * vi[t];
    if (lane == 0) h[i * m + j] = hij;
  }
  T acc = 0;
  for (int t = lane; t < nS; t += 32) acc += w[t] * w[t];
  T hn = sqrt(warp_total(acc));
  // what is left after orthogonalisation at the level of the cancellation error is rounding noise,
  // not a new direction: treat it as a (happy) breakdown so that the least-squares step ignores it
  if (hn <= T(64) * std::numeric_limits<T>::epsilon() * w0) hn = T(0);
  if (lane == 0) h[(j + 1) * m + j] = hn;
  const T inv = hn > T(0) ? T(1) / hn : T(0);
  for (int t = lane; t < nS; t += 32) w[t] *= inv;
}

// y = argmin || beta e1 - H y || (Givens, by lane 0 of the column's warp), then du_S = sum_j y_j Z_j.
template <typename T, int G = 0>
__global__ void __launch_bounds__(32 * kSubWarps)
    sub_lsq_combine_kernel(int E, int nS, int64_t stride, int m, const T* __restrict__ beta,
                           const T* __restrict__ H, const T* __restrict__ Z, T* __restrict__ duS) {
  __shared__ T ys[kSubWarps][16];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int col = blockIdx.x * kSubWarps + wid;
  if (col >= E) return;  // whole warps
  T* y = ys[wid];
  if (lane == 0) {
    T R[17][16], g[17];
    const T* h = H + (size_t)col * (m + 1) * m;
    for (int i = 0; i <= m; ++i) {
      g[i] = 0;
      for (int c = 0; c < m; ++c) R[i][c] = h[i * m + c];
    }
    g[0] = beta[col];
    int k = m;  // stop at a (happy) breakdown: zero subdiagonal
    for (int c = 0; c < m; ++c) {
      const T a = R[c][c], b = R[c + 1][c];
      const T den = sqrt(a * a + b * b);
      if (den == T(0)) { k = c; break; }
      const T cs = a / den, sn = b / den;
      for (int cc = c; cc < m; ++cc) {
        const T x0 = R[c][cc], x1 = R[c + 1][cc];
        R[c][cc] = cs * x0 + sn * x1;
        R[c + 1][cc] = -sn * x0 + cs * x1;
      }
      const T g0 = g[c];
      g[c] = cs * g0;
      g[c + 1] = -sn * g0;
      if (b == T(0)) { k = c + 1; break; }
    }
    for (int c = 0; c < m; ++c) y[c] = 0;
    for (int i = k - 1; i >= 0; --i) {
      T acc = g[i];
      for (int c = i + 1; c < k; ++c) acc -= R[i][c] * y[c];
      y[i] = acc / R[i][i];
    }
  }
  __syncwarp();
  const size_t off = (size_t)col * nS;
  if constexpr (G == 0) {
    for (int t = lane; t < nS; t += 32) {
      T acc = 0;
      for (int c = 0; c < m; ++c) acc += y[c] * Z[(size_t)c * stride + off + t];
      duS[off + t] = acc;
    }
  } else {
    // 16-byte vectors per lane, as the register forms of the other two kernels
    using SV = SubVec<T>;
    constexpr int EV = SV::E;
    T acc[G][EV] = {};
    for (int c = 0; c < m; ++c) {
      const T yc = y[c];
      const T* zc = Z + (size_t)c * stride + off;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int i = (g * 32 + lane) * EV;
        if (i >= nS) continue;
        T z[EV];
        SV::ld(zc + i, z);
#pragma unroll
        for (int e = 0; e < EV; ++e) acc[g][e] += yc * z[e];
      }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int i = (g * 32 + lane) * EV;
      if (i < nS) SV::st(duS + off + i, acc[g]);
    }
  }
}

// Register-resident forms of the two per-subdomain kernels above: a warp keeps its column's w
// (and the current V_i) in registers as G 16-byte vectors per lane (lane l holds elements
// 16/sizeof(T) x (32 g + l) + 0..), so every vector of the column is read or written once per call
// with 16-byte coalesced accesses instead of once per Gram-Schmidt pass. Same operations in the
// same order per element as the kernels above; only the partial sums of each inner product are
// grouped differently across the lanes.
template <typename T, int G>
__global__ void __launch_bounds__(32 * kSubWarps)
    sub_normalize_reg_kernel(int E, int ld, const T* __restrict__ rS, T* __restrict__ V0, T* __restrict__ beta) {
  using SV = SubVec<T>;
  constexpr int EV = SV::E;
  const int col = blockIdx.x * kSubWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (col >= E) return;  // whole warps
  const size_t off = (size_t)col * ld;
  T r[G][EV];
  T acc = 0;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int i = (g * 32 + lane) * EV;
    if (i < ld) SV::ld(rS + off + i, r[g]);
    else
#pragma unroll
      for (int e = 0; e < EV; ++e) r[g][e] = 0;
#pragma unroll
    for (int e = 0; e < EV; ++e) acc += r[g][e] * r[g][e];
  }
  const T nrm = sqrt(warp_total(acc));
  const T inv = nrm > T(0) ? T(1) / nrm : T(0);
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int i = (g * 32 + lane) * EV;
    if (i >= ld) continue;
#pragma unroll
    for (int e = 0; e < EV; ++e) r[g][e] *= inv;
    SV::st(V0 + off + i, r[g]);
  }
  if (lane == 0) beta[col] = nrm;
}

template <typename T, int G>
__global__ void __launch_bounds__(32 * kSubWarps)
    sub_arnoldi_reg_kernel(int E, int ld, int64_t stride, int j, int m, const T* __restrict__ D, T* V,
                           const T* __restrict__ Z, T* __restrict__ H) {
  using SV = SubVec<T>;
  constexpr int EV = SV::E;
  const int col = blockIdx.x * kSubWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (col >= E) return;  // whole warps
  const size_t off = (size_t)col * ld;
  const T* vj = V + (size_t)j * stride + off;
  const T* zj = Z + (size_t)j * stride + off;
  T w[G][EV];
  T acc0 = 0;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int i = (g * 32 + lane) * EV;
    if (i < ld) {
      T a[EV], d[EV], z[EV];
      SV::ld(vj + i, a);
      SV::ld(D + off + i, d);
      SV::ld(zj + i, z);
#pragma unroll
      for (int e = 0; e < EV; ++e) w[g][e] = a[e] + d[e] * z[e];
    } else {
#pragma unroll
      for (int e = 0; e < EV; ++e) w[g][e] = 0;
    }
#pragma unroll
    for (int e = 0; e < EV; ++e) acc0 += w[g][e] * w[g][e];
  }
  const T w0 = sqrt(warp_total(acc0));  // ||w|| before orthogonalisation
  T* h = H + (size_t)col * (m + 1) * m;
  for (int ii = 0; ii <= j; ++ii) {
    const T* vi = V + (size_t)ii * stride + off;
    T v[G][EV];
    T acc = 0;
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int i = (g * 32 + lane) * EV;
      if (i < ld) SV::ld(vi + i, v[g]);
      else
#pragma unroll
        for (int e = 0; e < EV; ++e) v[g][e] = 0;
#pragma unroll
      for (int e = 0; e < EV; ++e) acc += w[g][e] * v[g][e];
    }
    const T hij = warp_total(acc);
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
      for (int e = 0; e < EV; ++e) w[g][e] -= hij * v[g][e];
    if (lane == 0) h[ii * m + j] = hij;
  }
  T acc = 0;
#pragma unroll
  for (int g = 0; g < G; ++g)
#pragma unroll
    for (int e = 0; e < EV; ++e) acc += w[g][e] * w[g][e];
  T hn = sqrt(warp_total(acc));
  // rounding noise after orthogonalisation is a (happy) breakdown, as in sub_arnoldi_kernel
  if (hn <= T(64) * std::numeric_limits<T>::epsilon() * w0) hn = T(0);
  if (lane == 0) h[(j + 1) * m + j] = hn;
  const T inv = hn > T(0) ? T(1) / hn : T(0);
  T* wout = V + (size_t)(j + 1) * stride + off;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int i = (g * 32 + lane) * EV;
    if (i >= ld) continue;
#pragma unroll
    for (int e = 0; e < EV; ++e) w[g][e] *= inv;
    SV::st(wout + i, w[g]);
  }
}

// 16-byte vectors per lane a column of ld values needs, rounded up to an instantiated count (0: the
// column is too long for the register forms)
template <typename T>
int sub_reg_groups(int ld) {
  if (ld % (16 / (int)sizeof(T)) != 0) return 0;
  const int g = (ld + 32 * (16 / (int)sizeof(T)) - 1) / (32 * (16 / (int)sizeof(T)));
  for (int c : {1, 2, 3, 4, 6, 8, 10, 12, 14, 16})
    if (g <= c) return c;
  return 0;
}

template <typename T>
void launch_sub_normalize(int E, int nS, const T* rS, T* V0, T* beta, cudaStream_t s) {
  if (E == 0) return;
  const dim3 grid((E + kSubWarps - 1) / kSubWarps), block(32 * kSubWarps);
  switch (sub_reg_groups<T>(nS)) {
#define DG_SUB_NORM(GG) \
  case GG: sub_normalize_reg_kernel<T, GG><<<grid, block, 0, s>>>(E, nS, rS, V0, beta); break;
    DG_SUB_NORM(1) DG_SUB_NORM(2) DG_SUB_NORM(3) DG_SUB_NORM(4) DG_SUB_NORM(6) DG_SUB_NORM(8) DG_SUB_NORM(10)
    DG_SUB_NORM(12) DG_SUB_NORM(14) DG_SUB_NORM(16)
#undef DG_SUB_NORM
    default: sub_normalize_kernel<T><<<grid, block, 0, s>>>(E, nS, rS, V0, beta);
  }
  DG_LAUNCHED(1);
}
template <typename T>
void launch_sub_arnoldi(int E, int nS, int j, int m, const T* D, T* V, const T* Z, T* H, cudaStream_t s) {
  if (E == 0) return;
  const dim3 grid((E + kSubWarps - 1) / kSubWarps), block(32 * kSubWarps);
  const int64_t stride = (int64_t)E * nS;
  switch (sub_reg_groups<T>(nS)) {
#define DG_SUB_ARN(GG) \
  case GG: sub_arnoldi_reg_kernel<T, GG><<<grid, block, 0, s>>>(E, nS, stride, j, m, D, V, Z, H); break;
    DG_SUB_ARN(1) DG_SUB_ARN(2) DG_SUB_ARN(3) DG_SUB_ARN(4) DG_SUB_ARN(6) DG_SUB_ARN(8) DG_SUB_ARN(10)
    DG_SUB_ARN(12) DG_SUB_ARN(14) DG_SUB_ARN(16)
#undef DG_SUB_ARN
    default: sub_arnoldi_kernel<T><<<grid, block, 0, s>>>(E, nS, stride, j, m, D, V, Z, H);
  }
  DG_LAUNCHED(1);
}
template <typename T>
void launch_sub_lsq_combine(int E, int nS, int m, const T* beta, const T* H, const T* Z, T* duS, cudaStream_t s) {
  if (E == 0) return;
  const dim3 grid((E + kSubWarps - 1) / kSubWarps), block(32 * kSubWarps);
  const int64_t stride = (int64_t)E * nS;
  switch (sub_reg_groups<T>(nS)) {
#define DG_SUB_LSQ(GG) \
  case GG: sub_lsq_combine_kernel<T, GG><<<grid, block, 0, s>>>(E, nS, stride, m, beta, H, Z, duS); break;
    DG_SUB_LSQ(1) DG_SUB_LSQ(2) DG_SUB_LSQ(3) DG_SUB_LSQ(4) DG_SUB_LSQ(6) DG_SUB_LSQ(8) DG_SUB_LSQ(10)
    DG_SUB_LSQ(12) DG_SUB_LSQ(14) DG_SUB_LSQ(16)
#undef DG_SUB_LSQ
    default: sub_lsq_combine_kernel<T><<<grid, block, 0, s>>>(E, nS, stride, m, beta, H, Z, duS);
  }
  DG_LAUNCHED(1);
}
template void launch_sub_normalize<double>(int, int, const double*, double*, double*, cudaStream_t);
template void launch_sub_normalize<float>(int, int, const float*, float*, float*, cudaStream_t);
template void launch_sub_arnoldi<double>(int, int, int, int, const double*, double*, const double*, double*,
                                         cudaStream_t);
template void launch_sub_arnoldi<float>(int, int, int, int, const float*, float*, const float*, float*, cudaStream_t);
template void launch_sub_lsq_combine<double>(int, int, int, const double*, const double*, const double*, double*,
                                             cudaStream_t);
template void launch_sub_lsq_combine<float>(int, int, int, const float*, const float*, const float*, float*,
                                            cudaStream_t);


template void launch_class_gemm_tiles<double>(const double*, const double*, double*, int, const int4*, int,
                                               const int*, double, cudaStream_t, int);
template void launch_class_gemm_tiles<float>(const float*, const float*, float*, int, const int4*, int, const int*,
                                              float, cudaStream_t, int);

}  // namespace dg
