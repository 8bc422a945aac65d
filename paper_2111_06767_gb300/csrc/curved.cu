// DG operator of -div(K grad u) on curved (mapped) hexahedral elements (Sec. II with the metric
// terms of Eqs. massmat, stiffmat and liftop, flat background metric, fluxes F_v = u, F_u = K v with
// a positive scalar coefficient K per node; K = 1 is the Poisson operator) and the pieces it needs
// around it: the nodal metric, the penalty at every face node, the mass diagonal, the coarse-level
// node coordinates, and the explicit Schwarz subdomain matrices, one per subdomain.
//
// Each element's map is given isoparametrically by the physical coordinates of its LGL nodes.
// With Jac^i_j = dx^i/dxi^j = Dhat_j x^i at the nodes, J = det Jac and G = Jac^-1
// (G^j_i = dxi^j/dx^i), LGL collocation gives M = w_p J_p, (MD_i)_pq = w_p J_p G^j_i(p) Dhat_j,pq and
// the face mass w_a w_b J^f with J^f = J |G^d| (Nanson's relation), so per element
//   v_i  = G^j_i Dhat_j u + (|G^d| / w_0) n_i (u_E - u) / 2                  on face nodes
//   A u  = -w_p J G^j_i Dhat_j (K v^i)
//          - w_a w_b J |G^d| [ (K n.g - F_E)/2 - sigma (K u - K_E u_E) - K n.v ]
// with the unit outward normal n = s G^d / |G^d|, the local gradient g = G^j Dhat_j u, the exterior
// value u_E, coefficient K_E and own outward normal flux F_E = K_E n_E.g_E (Eq. numflux), and the
// ghost states of Eq. bc on box faces (K_E = K; Dirichlet: u_E = -u, F_E = -K n.g; Neumann:
// u_E = u, F_E = K n.g). sigma = C N^2 / min(h, h_E) with h = 2 / |G^d| the element size normal to
// the face at the node (the element width for affine elements).
//
// GB300 mapping: one CTA per element, one thread per node (N^3 threads), the element's values, the
// lifted auxiliary field and the exterior face data staged in shared memory. The exterior normal
// fluxes come from a trace pass (every element writes n.g on its six faces) before the operator
// pass; the metric is read once per node (J and the nine G entries, coalesced).
#include <algorithm>
#include <vector>

#include "domain.h"
#include "schwarz_dev.cuh"

namespace dg {

namespace {

enum : int { kNbr = 0, kDirichlet = 1, kNeumann = 2, kZero = 3 };

template <int N, typename T>
struct CurvedSmem {
  T D[N * N];
  T w[N];
  T u[N * N * N];
  T v[3][N * N * N];
  T uE[6][N * N];  // exterior value at each face node (kNbr faces)
  T fE[6][N * N];  // exterior's own outward normal flux K_E n_E.g_E (kNbr faces)
  int type[6];
  int eE[6];       // exterior element (kNbr faces): its coefficient is read at the matching node
};

__device__ __forceinline__ int elem_nbr(int nx, int ny, int nz, int e, int f) {
  int c[3] = {e % nx, (e / nx) % ny, e / (nx * ny)};
  const int n[3] = {nx, ny, nz};
  const int d = f >> 1;
  c[d] += (f & 1) ? 1 : -1;
  if (c[d] < 0 || c[d] >= n[d]) return -1;
  return c[0] + nx * (c[1] + ny * c[2]);
}

template <int N, typename T>
__device__ __forceinline__ void load_metric(const T* __restrict__ geo, int64_t ndof, int64_t gp, T& J, T G[3][3]) {
  J = geo[gp];
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int i = 0; i < 3; ++i) G[j][i] = geo[(1 + 3 * j + i) * ndof + gp];
}

// Logical derivatives of smem field a at node (i, j, k).
template <int N, typename T>
__device__ __forceinline__ void logical_grad(const T* D, const T* a, int i, int j, int k, T du[3]) {
  T gx = 0, gy = 0, gz = 0;
#pragma unroll
  for (int l = 0; l < N; ++l) {
    gx += D[i * N + l] * a[(k * N + j) * N + l];
    gy += D[j * N + l] * a[(k * N + l) * N + i];
    gz += D[k * N + l] * a[(l * N + j) * N + i];
  }
  du[0] = gx;
  du[1] = gy;
  du[2] = gz;
}

__device__ __forceinline__ void face_coords(int d, int i, int j, int k, int& a1, int& a2) {
  a1 = d == 0 ? j : i;
  a2 = d == 2 ? j : k;
}

// The element operator at node p = threadIdx.x (every thread of the CTA calls it; S.u, S.uE,
// S.fE and S.type filled and synchronised). Returns (A u)_p, massive form.
template <int N, typename T>
__device__ T curved_element(CurvedSmem<N, T>& S, const T* __restrict__ geo, int64_t ndof, int64_t gbase,
                            const T* __restrict__ sigma_e) {
  constexpr int N2 = N * N;
  const int p = threadIdx.x;
  const int i = p % N, j = (p / N) % N, k = p / N2;
  const int idx[3] = {i, j, k};
  T J, G[3][3];
  load_metric<N, T>(geo, ndof, gbase + p, J, G);
  const T Kp = geo[10 * ndof + gbase + p];
  T du[3];
  logical_grad<N, T>(S.D, S.u, i, j, k, du);
  T g[3], v[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    g[c] = G[0][c] * du[0] + G[1][c] * du[1] + G[2][c] * du[2];
    v[c] = g[c];
  }
  const T up = S.u[p];
  // the faces through the node, at most one per dimension: their unit outward normals and |G^d|
  // (one square root and one division per face)
  int fside[3];
  T nn[3][3], nrm[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    fside[d] = idx[d] == 0 ? 0 : (idx[d] == N - 1 ? 1 : -1);
    nrm[d] = T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) nn[d][c] = T(0);
    if (fside[d] >= 0) {
      nrm[d] = sqrt(G[d][0] * G[d][0] + G[d][1] * G[d][1] + G[d][2] * G[d][2]);
      const T sc = (fside[d] ? T(1) : T(-1)) / nrm[d];
#pragma unroll
      for (int c = 0; c < 3; ++c) nn[d][c] = sc * G[d][c];
    }
  }
  const T half_w0inv = T(0.5) / S.w[0];
  // lifting of the auxiliary flux on every face through the node
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (fside[d] < 0) continue;
    const int f = 2 * d + fside[d];
    int a1, a2;
    face_coords(d, i, j, k, a1, a2);
    const int ab = a2 * N + a1;
    const int t = S.type[f];
    const T uE = t == kNbr ? S.uE[f][ab] : (t == kDirichlet ? -up : (t == kNeumann ? up : T(0)));
    const T lift = (uE - up) * nrm[d] * half_w0inv;
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] += nn[d][c] * lift;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) S.v[c][p] = Kp * v[c];
  __syncthreads();
  // divergence of the flux K v: sum_i sum_j G^j_i Dhat_j (K v^i)
  T div = 0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T dv[3];
    logical_grad<N, T>(S.D, S.v[c], i, j, k, dv);
    div += G[0][c] * dv[0] + G[1][c] * dv[1] + G[2][c] * dv[2];
  }
  const T wp = S.w[i] * S.w[j] * S.w[k];
  T Au = -wp * J * div;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (fside[d] < 0) continue;
    const int side = fside[d], f = 2 * d + side;
    int a1, a2;
    face_coords(d, i, j, k, a1, a2);
    const int ab = a2 * N + a1;
    T ng = 0, nv = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ng += nn[d][c] * g[c];
      nv += nn[d][c] * v[c];
    }
    ng *= Kp;  // n.F_u of the local gradient
    nv *= Kp;
    const int t = S.type[f];
    const T uE = t == kNbr ? S.uE[f][ab] : (t == kDirichlet ? -up : (t == kNeumann ? up : T(0)));
    const T fE = t == kNbr ? S.fE[f][ab] : (t == kDirichlet ? -ng : (t == kNeumann ? ng : T(0)));
    const T KE = t == kNbr ? geo[10 * ndof + (int64_t)S.eE[f] * (N * N2) + node_of<N>(d, side ? 0 : N - 1, a1, a2)]
                           : Kp;
    const T prim = T(0.5) * (ng - fE) - sigma_e[f * N2 + ab] * (Kp * up - KE * uE);
    Au -= S.w[a1] * S.w[a2] * J * nrm[d] * (prim - nv);
  }
  return Au;
}

template <int N, typename T>
__device__ __forceinline__ void load_tables(CurvedSmem<N, T>& S, const T* __restrict__ D, const T* __restrict__ w) {
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) S.D[t] = D[t];
  for (int t = threadIdx.x; t < N; t += blockDim.x) S.w[t] = w[t];
}

// Outward normal flux n.g of every face node of every element (the exterior data of its neighbours).
template <int N, typename T>
__global__ void __launch_bounds__(N * N * N) curved_trace_kernel(CurvedArgs<T> a) {
  constexpr int N2 = N * N, N3 = N * N * N;
  __shared__ T sD[N2];
  __shared__ T su[N3];
  const int e = blockIdx.x, p = threadIdx.x;
  const int i = p % N, j = (p / N) % N, k = p / N2;
  for (int t = p; t < N2; t += N3) sD[t] = a.D[t];
  su[p] = a.u[(int64_t)e * N3 + p];
  __syncthreads();
  T J, G[3][3];
  load_metric<N, T>(a.geo, a.ndof, (int64_t)e * N3 + p, J, G);
  const T Kp = a.geo[10 * a.ndof + (int64_t)e * N3 + p];
  T du[3];
  logical_grad<N, T>(sD, su, i, j, k, du);
  const int idx[3] = {i, j, k};
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1, side = f & 1;
    if (idx[d] != (side ? N - 1 : 0)) continue;
    int a1, a2;
    face_coords(d, i, j, k, a1, a2);
    const T sc = (side ? T(1) : T(-1)) / sqrt(G[d][0] * G[d][0] + G[d][1] * G[d][1] + G[d][2] * G[d][2]);
    T ng = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) ng += G[d][c] * (G[0][c] * du[0] + G[1][c] * du[1] + G[2][c] * du[2]);
    a.trace[((int64_t)e * 6 + f) * N2 + a2 * N + a1] = Kp * sc * ng;
  }
}

// out = A u, or b - A u with b.
template <int N, typename T>
__global__ void __launch_bounds__(N * N * N) curved_apply_kernel(CurvedArgs<T> a) {
  constexpr int N2 = N * N, N3 = N * N * N;
  __shared__ CurvedSmem<N, T> S;
  const int e = blockIdx.x, p = threadIdx.x;
  load_tables<N, T>(S, a.D, a.w);
  S.u[p] = a.u[(int64_t)e * N3 + p];
  if (p < 6) {
    const int nb = elem_nbr(a.n[0], a.n[1], a.n[2], e, p);
    S.type[p] = nb >= 0 ? kNbr : (((a.neumann >> p) & 1) ? kNeumann : kDirichlet);
    S.eE[p] = nb;
  }
  for (int t = p; t < 6 * N2; t += N3) {
    const int f = t / N2, ab = t - f * N2, d = f >> 1, side = f & 1;
    const int nb = elem_nbr(a.n[0], a.n[1], a.n[2], e, f);
    if (nb >= 0) {
      S.uE[f][ab] = a.u[(int64_t)nb * N3 + node_of<N>(d, side ? 0 : N - 1, ab % N, ab / N)];
      S.fE[f][ab] = a.trace[((int64_t)nb * 6 + (f ^ 1)) * N2 + ab];
    }
  }
  __syncthreads();
  const T Au = curved_element<N, T>(S, a.geo, a.ndof, (int64_t)e * N3, a.sigma + (int64_t)e * 6 * N2);
  const int64_t gp = (int64_t)e * N3 + p;
  a.out[gp] = a.b ? a.b[gp] - Au : Au;
}

// Column q of subdomain e's matrix A_S (row-major [nS][nS] at A_out + (e - e0) nS^2): the curved
// operator on the patch (centre e and its face neighbours, zero data outside the subdomain's
// elements) applied to the unit vector of subdomain point q, restricted to the subdomain's points.
// Columns of points in a missing neighbour slot are identity columns.
template <int N, typename T>
__global__ void __launch_bounds__(N * N * N) curved_column_kernel(CurvedArgs<T> a, int ov, int nS, int e0,
                                                                  T* __restrict__ A_out) {
  constexpr int N2 = N * N, N3 = N * N * N;
  __shared__ CurvedSmem<N, T> S;
  __shared__ T sTP[6][N2];  // outward normal fluxes of the unit vector's own slot
  __shared__ int selem[7];
  const int q = blockIdx.x, e = e0 + blockIdx.y, p = threadIdx.x;
  const int i = p % N, j = (p / N) % N, k = p / N2;
  T* A = A_out + (size_t)blockIdx.y * nS * nS;
  int P, pP;
  if (q < N3) {
    P = 0;
    pP = q;
  } else {
    const int r = q - N3, f = r / (ov * N2), rr = r - f * ov * N2;
    const int depth = rr / N2, a2 = (rr / N) % N, a1 = rr % N;
    P = 1 + f;
    pP = node_of<N>(f >> 1, (f & 1) ? depth : N - 1 - depth, a1, a2);
  }
  if (p < 7) selem[p] = p == 0 ? e : elem_nbr(a.n[0], a.n[1], a.n[2], e, p - 1);
  load_tables<N, T>(S, a.D, a.w);
  for (int r = p; r < nS; r += N3) A[(size_t)r * nS + q] = T(0);
  __syncthreads();
  if (selem[P] < 0) {
    if (p == 0) A[(size_t)q * nS + q] = T(1);
    return;
  }
  // the unit vector's normal fluxes on the faces of its own slot
  {
    S.u[p] = p == pP ? T(1) : T(0);
    __syncthreads();
    T J, G[3][3];
    load_metric<N, T>(a.geo, a.ndof, (int64_t)selem[P] * N3 + p, J, G);
    const T Kp = a.geo[10 * a.ndof + (int64_t)selem[P] * N3 + p];
    T du[3];
    logical_grad<N, T>(S.D, S.u, i, j, k, du);
    const int idx[3] = {i, j, k};
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const int d = f >> 1, side = f & 1;
      if (idx[d] != (side ? N - 1 : 0)) continue;
      int a1, a2;
      face_coords(d, i, j, k, a1, a2);
      const T sc = (side ? T(1) : T(-1)) / sqrt(G[d][0] * G[d][0] + G[d][1] * G[d][1] + G[d][2] * G[d][2]);
      T ng = 0;
#pragma unroll
      for (int c = 0; c < 3; ++c) ng += G[d][c] * (G[0][c] * du[0] + G[1][c] * du[1] + G[2][c] * du[2]);
      sTP[f][a2 * N + a1] = Kp * sc * ng;
    }
    __syncthreads();
  }
  // slots whose rows the unit vector reaches: its own slot and the slots across its faces
  for (int X = 0; X < 7; ++X) {
    const bool adjacent = P == 0 ? true : X == 0;
    if (!(X == P || adjacent) || selem[X] < 0) continue;
    S.u[p] = (X == P && p == pP) ? T(1) : T(0);
    if (p < 6) {
      const int f = p;
      int t;
      if (X == 0) {
        t = selem[1 + f] >= 0 ? kNbr : (((a.neumann >> f) & 1) ? kNeumann : kDirichlet);
      } else if (f == ((X - 1) ^ 1)) {
        t = kNbr;  // faces the centre
      } else {
        t = elem_nbr(a.n[0], a.n[1], a.n[2], selem[X], f) >= 0 ? kZero
                                                                : (((a.neumann >> f) & 1) ? kNeumann : kDirichlet);
      }
      S.type[f] = t;
      S.eE[f] = t == kNbr ? selem[X == 0 ? 1 + f : 0] : -1;
    }
    for (int t = p; t < 6 * N2; t += N3) {
      const int f = t / N2, ab = t - f * N2, d = f >> 1, side = f & 1;
      const int Y = X == 0 ? 1 + f : 0;  // the slot across face f (when it is in the patch)
      const bool hit = Y == P;
      S.uE[f][ab] = (hit && pP == node_of<N>(d, side ? 0 : N - 1, ab % N, ab / N)) ? T(1) : T(0);
      S.fE[f][ab] = hit ? sTP[f ^ 1][ab] : T(0);
    }
    __syncthreads();
    const T Au = curved_element<N, T>(S, a.geo, a.ndof, (int64_t)selem[X] * N3, a.sigma + (int64_t)selem[X] * 6 * N2);
    const int row = subdomain_row<N>(X, p, ov);
    if (row >= 0) A[(size_t)row * nS + q] = Au;
    __syncthreads();
  }
}

// J and G = Jac^-1 at every node from the nodal coordinates (FP64), and the coefficient K: [11][ndof].
template <int N>
__global__ void __launch_bounds__(N * N * N) curved_metric_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                                                  const double* __restrict__ z, const double* __restrict__ K,
                                                                  const double* __restrict__ D, int64_t ndof,
                                                                  double* __restrict__ geo64, float* __restrict__ geo32,
                                                                  int* __restrict__ bad) {
  constexpr int N2 = N * N, N3 = N * N * N;
  __shared__ double sD[N2];
  __shared__ double sx[3][N3];
  const int e = blockIdx.x, p = threadIdx.x;
  const int i = p % N, j = (p / N) % N, k = p / N2;
  const int64_t gp = (int64_t)e * N3 + p;
  for (int t = p; t < N2; t += N3) sD[t] = D[t];
  sx[0][p] = x[gp];
  sx[1][p] = y[gp];
  sx[2][p] = z[gp];
  __syncthreads();
  double jac[3][3];  // jac[c][m] = dx^c / dxi^m
#pragma unroll
  for (int c = 0; c < 3; ++c) logical_grad<N, double>(sD, sx[c], i, j, k, jac[c]);
  const double c00 = jac[1][1] * jac[2][2] - jac[1][2] * jac[2][1];
  const double c01 = jac[1][2] * jac[2][0] - jac[1][0] * jac[2][2];
  const double c02 = jac[1][0] * jac[2][1] - jac[1][1] * jac[2][0];
  const double det = jac[0][0] * c00 + jac[0][1] * c01 + jac[0][2] * c02;
  if (!(det > 0.0)) atomicExch(bad, 1);  // a folded or left-handed element
  const double inv = 1.0 / det;
  // G[m][c] = (Jac^-1)[m][c], the cofactor transpose over det
  double G[3][3];
  G[0][0] = c00 * inv;
  G[1][0] = c01 * inv;
  G[2][0] = c02 * inv;
  G[0][1] = (jac[0][2] * jac[2][1] - jac[0][1] * jac[2][2]) * inv;
  G[1][1] = (jac[0][0] * jac[2][2] - jac[0][2] * jac[2][0]) * inv;
  G[2][1] = (jac[0][1] * jac[2][0] - jac[0][0] * jac[2][1]) * inv;
  G[0][2] = (jac[0][1] * jac[1][2] - jac[0][2] * jac[1][1]) * inv;
  G[1][2] = (jac[0][2] * jac[1][0] - jac[0][0] * jac[1][2]) * inv;
  G[2][2] = (jac[0][0] * jac[1][1] - jac[0][1] * jac[1][0]) * inv;
  if (!(K[gp] > 0.0)) atomicExch(bad, 2);  // the coefficient must be positive
  geo64[gp] = det;
  geo32[gp] = (float)det;
  geo64[10 * ndof + gp] = K[gp];
  geo32[10 * ndof + gp] = (float)K[gp];
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      geo64[(1 + 3 * m + c) * ndof + gp] = G[m][c];
      geo32[(1 + 3 * m + c) * ndof + gp] = (float)G[m][c];
    }
}

// sigma = C N^2 / min(h, h_E) at every face node, h = 2 / |G^d| (the interior's at box faces).
template <int N>
__global__ void curved_sigma_kernel(int nx, int ny, int nz, double penalty, const double* __restrict__ geo,
                                    int64_t ndof, double* __restrict__ sig64, float* __restrict__ sig32) {
  constexpr int N2 = N * N, N3 = N * N * N;
  const int64_t E = (int64_t)nx * ny * nz;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < E * 6 * N2; t += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(t / (6 * N2));
    const int f = (int)((t / N2) % 6), ab = (int)(t % N2), d = f >> 1, side = f & 1;
    auto size_at = [&](int el, int sd) {
      const int64_t gp = (int64_t)el * N3 + node_of<N>(d, sd ? N - 1 : 0, ab % N, ab / N);
      const double g0 = geo[(1 + 3 * d) * ndof + gp], g1 = geo[(2 + 3 * d) * ndof + gp], g2 = geo[(3 + 3 * d) * ndof + gp];
      return 2.0 / sqrt(g0 * g0 + g1 * g1 + g2 * g2);
    };
    const double h = size_at(e, side);
    const int nb = elem_nbr(nx, ny, nz, e, f);
    const double hE = nb >= 0 ? size_at(nb, 1 - side) : h;
    const double sg = penalty * N * N / fmin(h, hE);
    sig64[t] = sg;
    sig32[t] = (float)sg;
  }
}

// Coarse-level node coordinates on the fine elements' interpolated map: per coarsened dimension
// the coarse node xi_c lies in the lower child (xi_c <= 0, child coordinate 2 xi_c + 1) or the
// upper one (2 xi_c - 1); C[h][c][q] are the fine Lagrange weights there (identity for dimensions
// that are not coarsened).
template <int N>
__global__ void curved_coarsen_kernel(int cx, int cy, int cz, int fx, int fy, int fz, const double* __restrict__ C,
                                      const double* __restrict__ fin, int64_t fndof, double* __restrict__ out,
                                      int64_t cndof) {
  constexpr int N2 = N * N, N3 = N * N * N;
  const int64_t total = cndof;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(t / N3), p = (int)(t % N3);
    const int node[3] = {p % N, (p / N) % N, p / N2};
    const int ce[3] = {e % cx, (e / cx) % cy, e / (cx * cy)};
    const int cn[3] = {cx, cy, cz}, fn[3] = {fx, fy, fz};
    int child[3];
    const double* W[3];
    for (int d = 0; d < 3; ++d) {
      if (fn[d] == cn[d]) {
        child[d] = ce[d];
        W[d] = C + 2 * N2 + node[d] * N;  // identity rows
      } else {
        const int h = C[3 * N2 + node[d]] > 0.5 ? 1 : 0;  // the node's half
        child[d] = 2 * ce[d] + h;
        W[d] = C + h * N2 + node[d] * N;
      }
    }
    const int64_t fe = child[0] + (int64_t)fx * (child[1] + (int64_t)fy * child[2]);
    for (int c = 0; c < 4; ++c) {  // x, y, z and the coefficient
      const double* src = fin + c * fndof + fe * N3;
      double acc = 0.0;
      for (int kk = 0; kk < N; ++kk)
        for (int jj = 0; jj < N; ++jj) {
          const double wkj = W[2][kk] * W[1][jj];
          for (int ii = 0; ii < N; ++ii) acc += wkj * W[0][ii] * src[(kk * N + jj) * N + ii];
        }
      out[c * cndof + t] = acc;
    }
  }
}

__global__ void curved_mass_kernel(int N, const double* __restrict__ w, const double* __restrict__ geo, int64_t ndof,
                                   double* __restrict__ mass) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ndof; t += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(t % ((int64_t)N * N * N));
    mass[t] = w[p % N] * w[(p / N) % N] * w[p / (N * N)] * geo[t];
  }
}

int grid_for(int64_t n, int threads) { return (int)std::min<int64_t>((n + threads - 1) / threads, 152 * 64); }

}  // namespace

#define DG_CURVED_SWITCH(NN_CASE)                                                                        \
  switch (N) {                                                                                           \
    NN_CASE(2) NN_CASE(3) NN_CASE(4) NN_CASE(5) NN_CASE(6) NN_CASE(7) NN_CASE(8) NN_CASE(9) NN_CASE(10) \
    default: fail(DG_ERR_INVALID_ARG, "unsupported N");                                                  \
  }

template <typename T>
void launch_curved_apply(int N, const CurvedArgs<T>& a, int E, cudaStream_t s) {
  if (E == 0) return;
#define DG_CASE(NN)                                                            \
  case NN:                                                                     \
    curved_trace_kernel<NN, T><<<E, NN * NN * NN, 0, s>>>(a);                 \
    curved_apply_kernel<NN, T><<<E, NN * NN * NN, 0, s>>>(a);                 \
    break;
  DG_CURVED_SWITCH(DG_CASE)
#undef DG_CASE
  DG_LAUNCHED(2);
}

template <typename T>
void launch_curved_columns(int N, const CurvedArgs<T>& a, int ov, int nS, int e0, int count, T* A_out,
                           cudaStream_t s) {
  if (count == 0) return;
  DG_REQUIRE(count <= 65535, "at most 65535 subdomains per column launch");
  const dim3 grid(nS, count);
#define DG_CASE(NN)                                                                               \
  case NN:                                                                                        \
    curved_column_kernel<NN, T><<<grid, NN * NN * NN, 0, s>>>(a, ov, nS, e0, A_out);             \
    break;
  DG_CURVED_SWITCH(DG_CASE)
#undef DG_CASE
  DG_LAUNCHED(1);
}

void launch_curved_metric(int N, int64_t E, const double* xyz, const double* D, double* geo64, float* geo32, int* bad,
                          cudaStream_t s) {
  if (E == 0) return;
  const int64_t ndof = E * N * N * N;
#define DG_CASE(NN)                                                                                           \
  case NN:                                                                                                    \
    curved_metric_kernel<NN><<<(unsigned)E, NN * NN * NN, 0, s>>>(xyz, xyz + ndof, xyz + 2 * ndof,          \
                                                                   xyz + 3 * ndof, D, ndof, geo64, geo32, bad); \
    break;
  DG_CURVED_SWITCH(DG_CASE)
#undef DG_CASE
  DG_LAUNCHED(1);
}

void launch_curved_sigma(int N, const int n[3], double penalty, const double* geo64, double* sig64, float* sig32,
                         cudaStream_t s) {
  const int64_t E = (int64_t)n[0] * n[1] * n[2], ndof = E * N * N * N;
  const int64_t work = E * 6 * N * N;
  if (work == 0) return;
#define DG_CASE(NN)                                                                                           \
  case NN:                                                                                                    \
    curved_sigma_kernel<NN><<<grid_for(work, 256), 256, 0, s>>>(n[0], n[1], n[2], penalty, geo64, ndof, sig64, \
                                                               sig32);                                        \
    break;
  DG_CURVED_SWITCH(DG_CASE)
#undef DG_CASE
  DG_LAUNCHED(1);
}

void launch_curved_coarsen(int N, const int cn[3], const int fn[3], const double* C, const double* fine_xyz,
                           double* coarse_xyz, cudaStream_t s) {
  const int64_t fndof = (int64_t)fn[0] * fn[1] * fn[2] * N * N * N;
  const int64_t cndof = (int64_t)cn[0] * cn[1] * cn[2] * N * N * N;
  if (cndof == 0) return;
#define DG_CASE(NN)                                                                                          \
  case NN:                                                                                                   \
    curved_coarsen_kernel<NN><<<grid_for(cndof, 256), 256, 0, s>>>(cn[0], cn[1], cn[2], fn[0], fn[1], fn[2], \
                                                                    C, fine_xyz, fndof, coarse_xyz, cndof); \
    break;
  DG_CURVED_SWITCH(DG_CASE)
#undef DG_CASE
  DG_LAUNCHED(1);
}

void launch_curved_mass(int N, const double* w, const double* geo64, int64_t ndof, double* mass, cudaStream_t s) {
  if (ndof == 0) return;
  curved_mass_kernel<<<grid_for(ndof, 256), 256, 0, s>>>(N, w, geo64, ndof, mass);
  DG_LAUNCHED(1);
}

template void launch_curved_apply<double>(int, const CurvedArgs<double>&, int, cudaStream_t);
template void launch_curved_apply<float>(int, const CurvedArgs<float>&, int, cudaStream_t);
template void launch_curved_columns<double>(int, const CurvedArgs<double>&, int, int, int, int, double*,
                                            cudaStream_t);
template void launch_curved_columns<float>(int, const CurvedArgs<float>&, int, int, int, int, float*, cudaStream_t);

}  // namespace dg
