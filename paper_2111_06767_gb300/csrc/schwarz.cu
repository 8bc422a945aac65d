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
// Subdomain point order: the central element's N^3 points (element order), then for faces
// f = 2 d + side the neighbour's N_overlap layers counted from the shared face, each layer in
// (a2, a1) order of the tangential indices. Missing neighbours keep their slots as padding
// (identity rows and columns in A_S, zero data), so every subdomain has n_S = N^3 + 6 N_ov N^2.
#include "internal.h"

namespace dg {

// ------------------------------------------------------------------ A_S columns

// Patch description per class: for slot s in 0..6 (0 = centre, 1 + f = neighbour across face f)
// info[s*6 + f'] = face type of that slot's face f': >= 0 slot inside the patch, -1 external
// boundary, -2 internal face with zero data outside the patch; info[42 + s] = slot exists.
constexpr int kPatchInts = 49;

template <int N>
__device__ __forceinline__ int node_of(int d, int idx_d, int a1, int a2) {
  int c0, c1, c2;
  if (d == 0) { c0 = idx_d; c1 = a1; c2 = a2; }
  else if (d == 1) { c0 = a1; c1 = idx_d; c2 = a2; }
  else { c0 = a1; c1 = a2; c2 = idx_d; }
  return (c2 * N + c1) * N + c0;
}

// Subdomain row of point p of slot s, or -1 if outside S.
template <int N>
__device__ __forceinline__ int subdomain_row(int s, int p, int ov) {
  if (s == 0) return p;
  const int f = s - 1, d = f >> 1, side = f & 1;
  const int c[3] = {p % N, (p / N) % N, p / (N * N)};
  const int depth = side ? c[d] : N - 1 - c[d];
  if (depth >= ov) return -1;
  const int a1 = d == 0 ? c[1] : c[0];
  const int a2 = d == 2 ? c[1] : c[2];
  return N * N * N + f * ov * N * N + (depth * N + a2) * N + a1;
}

template <int N>
struct ColumnShape {
  static constexpr int n3 = N * N * N;
  static constexpr int threads = n3 > 512 ? 512 : n3;
};

template <int N>
__global__ void __launch_bounds__(ColumnShape<N>::threads) subdomain_column_kernel(
    const OpGeom<double> g, const double* __restrict__ Dg, const double* __restrict__ wg,
    const int* __restrict__ patch_info, int ov, int nS, double* __restrict__ A_out) {
  constexpr int N2 = N * N, N3 = N * N * N, NT = ColumnShape<N>::threads;
  __shared__ double sD[N2];
  __shared__ double sw[N];
  __shared__ double su[N3];
  __shared__ double sv[3][N3];
  __shared__ double sfb[6][N2];
  __shared__ int sinfo[kPatchInts];

  const int q = blockIdx.x;  // column
  const int cls = blockIdx.y;
  const int tid = threadIdx.x;
  double* A = A_out + (size_t)cls * nS * nS + (size_t)q * nS;  // column q, contiguous
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
      double gx = 0, gy = 0, gz = 0;
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
      const double s = side ? 1.0 : -1.0;
      const double dxi = d == 0 ? g.dxi[0] : (d == 1 ? g.dxi[1] : g.dxi[2]);
      const double lift = d == 0 ? g.lift[0] : (d == 1 ? g.lift[1] : g.lift[2]);
      const double sigma = d == 0 ? g.sigma[0] : (d == 1 ? g.sigma[1] : g.sigma[2]);
      const double Jf = d == 0 ? g.Jf[0] : (d == 1 ? g.Jf[1] : g.Jf[2]);
      const int pf = node_of<N>(d, side ? N - 1 : 0, a1, a2);
      const double u_int = su[pf];
      const double g_int = sv[d][pf];
      const int t = sinfo[X * 6 + f];
      double u_ext, g_ext;
      if (t == -1) {
        u_ext = -u_int;
        g_ext = g_int;
      } else if (t == -2) {
        u_ext = 0.0;
        g_ext = 0.0;
      } else {
        // neighbour data is the unit vector restricted to slot t
        const int opp = side ? 0 : N - 1;
        u_ext = (t == P && node_of<N>(d, opp, a1, a2) == pP) ? 1.0 : 0.0;
        double acc = 0.0;
        if (t == P) {
          for (int l = 0; l < N; ++l)
            if (node_of<N>(d, l, a1, a2) == pP) acc += sD[opp * N + l];
        }
        g_ext = dxi * acc;
      }
      const double jump = u_ext - u_int;
      sv[d][pf] = g_int + s * jump * lift;
      const double Bf = Jf * sw[a1] * sw[a2];
      sfb[f][ab] = Bf * (0.5 * s * (g_ext - g_int) + (sigma - lift) * jump);
    }
    __syncthreads();
    for (int p = tid; p < N3; p += NT) {
      const int i = p % N, j = (p / N) % N, k = p / N2;
      double dx = 0, dy = 0, dz = 0;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        dx += sD[i * N + l] * sv[0][(k * N + j) * N + l];
        dy += sD[j * N + l] * sv[1][(k * N + l) * N + i];
        dz += sD[k * N + l] * sv[2][(l * N + j) * N + i];
      }
      const double M = g.J * sw[i] * sw[j] * sw[k];
      double res = -M * (g.dxi[0] * dx + g.dxi[1] * dy + g.dxi[2] * dz);
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

void launch_build_subdomain_matrices(int N, int overlap, const OpGeom<double>& g, const double* D, const double* w,
                                     const int* d_patch_info, int n_classes, int nS, double* A_out, cudaStream_t s) {
  dim3 grid(nS, n_classes);
  switch (N) {
#define DG_CASE(NN) \
  case NN: subdomain_column_kernel<NN><<<grid, ColumnShape<NN>::threads, 0, s>>>(g, D, w, d_patch_info, overlap, nS, A_out); break;
    DG_CASE(2) DG_CASE(3) DG_CASE(4) DG_CASE(5) DG_CASE(6) DG_CASE(7) DG_CASE(8) DG_CASE(9) DG_CASE(10)
#undef DG_CASE
    default: fail(DG_ERR_INVALID_ARG, "unsupported N");
  }
  DG_LAUNCHED(1);
}

// ------------------------------------------------------------------ Gauss-Jordan inversion

// Copy pivot row k and column k of every matrix into buffers.
__global__ void gj_copy_kernel(const double* __restrict__ A, int n, int k, double* __restrict__ row,
                               double* __restrict__ col) {
  const int c = blockIdx.y;
  const double* M = A + (size_t)c * n * n;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    row[(size_t)c * n + t] = M[(size_t)k * n + t];
    col[(size_t)c * n + t] = M[(size_t)t * n + k];
  }
}

// A[i][j] <- in-place Gauss-Jordan step k, from the saved pivot row and column.
__global__ void gj_update_kernel(double* __restrict__ A, int n, int k, const double* __restrict__ row,
                                 const double* __restrict__ col) {
  const int c = blockIdx.z;
  double* M = A + (size_t)c * n * n;
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || j >= n) return;
  const double piv = col[(size_t)c * n + k];
  const double rk = (j == k ? 1.0 : row[(size_t)c * n + j]) / piv;  // scaled pivot row
  if (i == k) {
    M[(size_t)k * n + j] = rk;
  } else {
    const double f = col[(size_t)c * n + i];
    M[(size_t)i * n + j] = (j == k ? 0.0 : M[(size_t)i * n + j]) - f * rk;
  }
}

void launch_invert_spd_batched(double* A, int n, int n_classes, cudaStream_t s) {
  if (n_classes == 0) return;
  DevBuf<double> row((size_t)n * n_classes), col((size_t)n * n_classes);
  dim3 cb(256), cg((n + 255) / 256, n_classes);
  dim3 ub(32, 8), ug((n + 31) / 32, (n + 7) / 8, n_classes);
  for (int k = 0; k < n; ++k) {
    gj_copy_kernel<<<cg, cb, 0, s>>>(A, n, k, row.get(), col.get());
    gj_update_kernel<<<ug, ub, 0, s>>>(A, n, k, row.get(), col.get());
  }
  DG_LAUNCHED(2 * n);
  DG_CUDA(cudaStreamSynchronize(s));  // row/col are freed on return
}

// ------------------------------------------------------------------ gather / scatter

// Subdomain rows and neighbours are computed from element coordinates, so the only tables are the
// element <-> subdomain-column maps and the per-point weight shares of the 64 neighbour patterns.

__device__ __forceinline__ int nbr_elem(const SubdomainGeom& g, int e, int f) {
  const int c0 = e % g.n[0], c1 = (e / g.n[0]) % g.n[1], c2 = e / (g.n[0] * g.n[1]);
  int c[3] = {c0, c1, c2};
  const int d = f >> 1;
  c[d] += (f & 1) ? 1 : -1;
  if (c[d] < 0 || c[d] >= g.n[d]) return -1;
  return c[0] + g.n[0] * (c[1] + g.n[1] * c[2]);
}

// r_S[col * nS + q] = r at subdomain point q of the subdomain in column col (0 outside the domain)
template <typename T>
__global__ void gather_kernel(SubdomainGeom g, const T* __restrict__ r, const int* __restrict__ elem_of_col,
                              T* __restrict__ rS) {
  const int N = g.N, N2 = N * N, N3 = N2 * N, ov = g.ov, nS = g.nS;
  const int64_t total = (int64_t)g.E * nS;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(t / nS);
    const int q = (int)(t - (int64_t)col * nS);
    const int e = elem_of_col[col];
    T v = 0;
    if (q < N3) {
      v = r[(int64_t)e * N3 + q];
    } else {
      const int rr = q - N3;
      const int f = rr / (ov * N2);
      const int k = rr - f * ov * N2;
      const int depth = k / N2, a2 = (k / N) % N, a1 = k % N;
      const int nb = nbr_elem(g, e, f);
      if (nb >= 0) {
        const int d = f >> 1, side = f & 1;
        const int idx = side ? depth : N - 1 - depth;
        int c0, c1, c2;
        if (d == 0) { c0 = idx; c1 = a1; c2 = a2; }
        else if (d == 1) { c0 = a1; c1 = idx; c2 = a2; }
        else { c0 = a1; c1 = a2; c2 = idx; }
        v = r[(int64_t)nb * N3 + (c2 * N + c1) * N + c0];
      }
    }
    rS[t] = v;
  }
}

template <typename T>
void launch_gather(const SubdomainGeom& g, const T* r, const int* elem_of_col, T* rS, cudaStream_t s) {
  const int64_t total = (int64_t)g.E * g.nS;
  if (total == 0) return;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  gather_kernel<T><<<blocks, 256, 0, s>>>(g, r, elem_of_col, rS);
  DG_LAUNCHED(1);
}

// u += sum over the subdomains containing each point of w_S du_S (Eq. schwarz_weighting)
template <typename T, typename TU>
__global__ void scatter_kernel(SubdomainGeom g, const T* __restrict__ duS, const int* __restrict__ col_of_elem,
                               const T* __restrict__ shares, TU* __restrict__ u) {
  const int N = g.N, N2 = N * N, N3 = N2 * N, ov = g.ov, nS = g.nS;
  const int64_t ndof = (int64_t)g.E * N3;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ndof; t += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(t / N3);
    const int p = (int)(t - (int64_t)q * N3);
    const int c[3] = {p % N, (p / N) % N, p / N2};
    int nb[6], pattern = 0;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      nb[f] = nbr_elem(g, q, f);
      pattern |= (nb[f] >= 0) << f;
    }
    const T* sh = shares + ((int64_t)pattern * N3 + p) * 7;
    T acc = sh[0] * duS[(int64_t)col_of_elem[q] * nS + p];
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      if (nb[f] < 0) continue;
      const int d = f >> 1, side = f & 1;
      // the neighbour sees this element across its face on the other side (slot 1 + back)
      const int back = 2 * d + (1 - side);
      const int depth = (1 - side) ? c[d] : N - 1 - c[d];
      if (depth >= ov) continue;
      const int a1 = d == 0 ? c[1] : c[0];
      const int a2 = d == 2 ? c[1] : c[2];
      const int row = N3 + back * ov * N2 + (depth * N + a2) * N + a1;
      acc += sh[1 + f] * duS[(int64_t)col_of_elem[nb[f]] * nS + row];
    }
    u[t] += (TU)acc;
  }
}

template <typename T, typename TU>
void launch_scatter_add(const SubdomainGeom& g, const T* duS, const int* col_of_elem, const T* shares, TU* u,
                        cudaStream_t s) {
  const int64_t ndof = (int64_t)g.E * g.N * g.N * g.N;
  if (ndof == 0) return;
  const int blocks = (int)std::min<int64_t>((ndof + 255) / 256, 152 * 16);
  scatter_kernel<T, TU><<<blocks, 256, 0, s>>>(g, duS, col_of_elem, shares, u);
  DG_LAUNCHED(1);
}

// ------------------------------------------------------------------ class GEMM (SIMT)

// Y[:, c0:c0+m] = Inv_c (nS x nS, row-major) * X[:, c0:c0+m] (columns of nS contiguous values).
// 64 x 64 output tiles, K chunks of 16 staged in shared memory, 4 x 4 outputs per thread.
template <typename T>
__global__ void __launch_bounds__(256) class_gemm_kernel(const T* __restrict__ inv, const T* __restrict__ X,
                                                         T* __restrict__ Y, int nS, const int4* __restrict__ tiles) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ T sA[BK][BM + 1];
  __shared__ T sB[BK][BN + 1];
  const int4 tile = tiles[blockIdx.x];  // (class, row0, col0, ncols in this class from col0)
  const int cls = tile.x, row0 = tile.y, col0 = tile.z, ncol = min(tile.w, BN);
  const T* A = inv + (size_t)cls * nS * nS;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4] = {};
  for (int k0 = 0; k0 < nS; k0 += BK) {
    for (int t = threadIdx.x; t < BM * BK; t += 256) {
      const int r = t / BK, kk = t % BK;
      const int gr = row0 + r, gk = k0 + kk;
      sA[kk][r] = (gr < nS && gk < nS) ? A[(size_t)gr * nS + gk] : T(0);
    }
    for (int t = threadIdx.x; t < BN * BK; t += 256) {
      const int c = t / BK, kk = t % BK;
      const int gk = k0 + kk;
      sB[kk][c] = (c < ncol && gk < nS) ? X[(size_t)(col0 + c) * nS + gk] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = sA[kk][ty + 16 * q]; b[q] = sB[kk][tx + 16 * q]; }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[q][r] += a[q] * b[r];
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int gr = row0 + ty + 16 * q;
    if (gr >= nS) continue;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int c = tx + 16 * r;
      if (c < ncol) Y[(size_t)(col0 + c) * nS + gr] = acc[q][r];
    }
  }
}

template <typename T>
void launch_class_gemm_tiles(const T* inv, const T* X, T* Y, int nS, const int4* d_tiles, int n_tiles, cudaStream_t s) {
  if (n_tiles == 0) return;
  class_gemm_kernel<T><<<n_tiles, 256, 0, s>>>(inv, X, Y, nS, d_tiles);
  DG_LAUNCHED(1);
}

template void launch_gather<double>(const SubdomainGeom&, const double*, const int*, double*, cudaStream_t);
template void launch_gather<float>(const SubdomainGeom&, const float*, const int*, float*, cudaStream_t);
template void launch_scatter_add<double, double>(const SubdomainGeom&, const double*, const int*, const double*,
                                                 double*, cudaStream_t);
template void launch_scatter_add<float, float>(const SubdomainGeom&, const float*, const int*, const float*, float*,
                                               cudaStream_t);
template void launch_class_gemm_tiles<double>(const double*, const double*, double*, int, const int4*, int,
                                              cudaStream_t);
template void launch_class_gemm_tiles<float>(const float*, const float*, float*, int, const int4*, int, cudaStream_t);

}  // namespace dg
