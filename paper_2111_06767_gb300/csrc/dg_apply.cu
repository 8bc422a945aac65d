// Matrix-free DG operator A u on affine hexahedral LGL elements (Sec. II).
//
// Poisson fluxes (Eq. poisson_fluxform), strong form in two steps (Eqs. dg_op_auxvars and
// dg_op_primal), generalized internal-penalty flux (Eq. numflux) with the penalty of
// Eq. penalty and homogeneous Dirichlet boundary fluxes (Eq. bc), massive form (b = M f).
// Integrals use LGL collocation quadrature: M is diagonal, MD_i = M D_i and the lifting acts
// on face points only.
//
// Per element, with g_d = (2/h_d) Dhat_d u the local gradient:
//   v_d   = g_d + s (u_ext - u_int) / (w_0 h_d)                      on face points of normal s e_d
//   A u   = -M sum_d (2/h_d) Dhat_d v_d
//           - sum_faces Bf [ s/2 (g_ext - g_int) + (sigma_d - 1/(w_0 h_d)) (u_ext - u_int) ]
// where Bf = J_f w_a w_b is the face quadrature weight. At an external face Eq. bc with
// (n F_v)^b = n u_b, u_b = 0, and (n F_u)^b = (n F_u)^int is the ghost state u_ext = -u_int,
// g_ext = g_int, which this kernel uses.
//
// GB300 mapping: EPB elements per CTA (EPB N^3 ~ 256 points), at most 512 threads striding over
// the points; the element block, its gradient and the face brackets stay in shared memory; neighbour face
// data (the neighbour's face value and normal derivative, which needs its whole normal line)
// is read straight from global memory, which L2 serves for the element-ordered sweep.
#include "internal.h"

namespace dg {

template <int N>
struct ApplyShape {
  static constexpr int n3 = N * N * N;
  static constexpr int epb = n3 >= 256 ? 1 : (256 / n3);         // elements per CTA
  static constexpr int threads = epb * n3 > 512 ? 512 : epb * n3;  // points per thread = ceil(epb n3 / threads)
};

template <typename T>
__device__ __forceinline__ T sel3(int d, T a, T b, T c) {
  return d == 0 ? a : (d == 1 ? b : c);
}

template <int N>
__device__ __forceinline__ int face_node(int d, int idx_d, int a1, int a2) {
  // node offset (k*N + j)*N + i of the point with index idx_d along d and tangential indices
  // a1 (the lower tangential dimension) and a2 (the higher one)
  if (d == 0) return (a2 * N + a1) * N + idx_d;
  if (d == 1) return (a2 * N + idx_d) * N + a1;
  return (idx_d * N + a2) * N + a1;
}

template <int N, typename T, int EPB, int NT>
__global__ void __launch_bounds__(NT) apply_kernel(const OpGeom<T> g, const T* __restrict__ Dg,
                                                   const T* __restrict__ wg, const T* __restrict__ u,
                                                   const T* __restrict__ diag, const T* __restrict__ b,
                                                   T* __restrict__ out, int E) {
  constexpr int N2 = N * N, N3 = N * N * N;
  __shared__ T sD[N2];
  __shared__ T sw[N];
  __shared__ T su[EPB][N3];
  __shared__ T sv[EPB][3][N3];
  __shared__ T sfb[EPB][6][N2];

  const int tid = threadIdx.x;
  const int e0 = blockIdx.x * EPB;
  for (int t = tid; t < N2; t += NT) sD[t] = Dg[t];
  for (int t = tid; t < N; t += NT) sw[t] = wg[t];
  for (int t = tid; t < EPB * N3; t += NT) {
    const int el = t / N3;
    su[el][t - el * N3] = e0 + el < E ? u[(int64_t)e0 * N3 + t] : T(0);
  }
  __syncthreads();

  // local gradient g_d = (2/h_d) Dhat_d u
  for (int t = tid; t < EPB * N3; t += NT) {
    const int el = t / N3, p = t - el * N3;
    const int i = p % N, j = (p / N) % N, k = p / N2;
    T gx = 0, gy = 0, gz = 0;
#pragma unroll
    for (int l = 0; l < N; ++l) {
      gx += sD[i * N + l] * su[el][(k * N + j) * N + l];
      gy += sD[j * N + l] * su[el][(k * N + l) * N + i];
      gz += sD[k * N + l] * su[el][(l * N + j) * N + i];
    }
    sv[el][0][p] = g.dxi[0] * gx;
    sv[el][1][p] = g.dxi[1] * gy;
    sv[el][2][p] = g.dxi[2] * gz;
  }
  __syncthreads();

  // face points: lift the auxiliary flux into v_d and form the primal flux bracket
  for (int item = tid; item < EPB * 6 * N2; item += NT) {
    const int el = item / (6 * N2);
    const int rem = item - el * 6 * N2;
    const int f = rem / N2;
    const int ab = rem - f * N2;
    const int a1 = ab % N, a2 = ab / N;
    const int d = f >> 1, side = f & 1;
    const int e = e0 + el;
    if (e >= E) continue;
    const T s = side ? T(1) : T(-1);
    const T dxi = sel3(d, g.dxi[0], g.dxi[1], g.dxi[2]);
    const T lift = sel3(d, g.lift[0], g.lift[1], g.lift[2]);
    const T sigma = sel3(d, g.sigma[0], g.sigma[1], g.sigma[2]);
    const T Jf = sel3(d, g.Jf[0], g.Jf[1], g.Jf[2]);
    const int pf = face_node<N>(d, side ? N - 1 : 0, a1, a2);
    const T u_int = su[el][pf];
    const T g_int = sv[el][d][pf];
    // neighbour across face f
    const int cx = e % g.nx, cy = (e / g.nx) % g.ny, cz = e / (g.nx * g.ny);
    const int cd = sel3(d, cx, cy, cz);
    const int nd = sel3(d, g.nx, g.ny, g.nz);
    const int cn = cd + (side ? 1 : -1);
    T u_ext, g_ext;
    if (cn >= 0 && cn < nd) {
      const int stride = sel3(d, 1, g.nx, g.nx * g.ny);
      const int q = e + (side ? stride : -stride);
      const T* uq = u + (int64_t)q * N3;
      const int opp = side ? 0 : N - 1;
      u_ext = __ldg(uq + face_node<N>(d, opp, a1, a2));
      T acc = 0;
#pragma unroll
      for (int l = 0; l < N; ++l) acc += sD[opp * N + l] * __ldg(uq + face_node<N>(d, l, a1, a2));
      g_ext = dxi * acc;
    } else {
      u_ext = -u_int;  // Dirichlet ghost state of Eq. bc with u_b = 0
      g_ext = g_int;
    }
    const T jump = u_ext - u_int;
    sv[el][d][pf] = g_int + s * jump * lift;
    const T Bf = Jf * sw[a1] * sw[a2];
    sfb[el][f][ab] = Bf * (T(0.5) * s * (g_ext - g_int) + (sigma - lift) * jump);
  }
  __syncthreads();

  // primal step: -M sum_d D_d v_d - ML [(n.v)^* - n.v]
  for (int t = tid; t < EPB * N3; t += NT) {
    const int el = t / N3, p = t - el * N3;
    const int e = e0 + el;
    if (e >= E) continue;
    const int i = p % N, j = (p / N) % N, k = p / N2;
    T dx = 0, dy = 0, dz = 0;
#pragma unroll
    for (int l = 0; l < N; ++l) {
      dx += sD[i * N + l] * sv[el][0][(k * N + j) * N + l];
      dy += sD[j * N + l] * sv[el][1][(k * N + l) * N + i];
      dz += sD[k * N + l] * sv[el][2][(l * N + j) * N + i];
    }
    const T M = g.J * sw[i] * sw[j] * sw[k];
    T res = -M * (g.dxi[0] * dx + g.dxi[1] * dy + g.dxi[2] * dz);
    if (i == 0) res -= sfb[el][0][k * N + j];
    if (i == N - 1) res -= sfb[el][1][k * N + j];
    if (j == 0) res -= sfb[el][2][k * N + i];
    if (j == N - 1) res -= sfb[el][3][k * N + i];
    if (k == 0) res -= sfb[el][4][j * N + i];
    if (k == N - 1) res -= sfb[el][5][j * N + i];
    const int64_t gi = (int64_t)e * N3 + p;
    if (diag) res += diag[gi] * su[el][p];
    out[gi] = b ? b[gi] - res : res;
  }
}

// Column variant: one thread per (i, j) column of N points along z, EPB elements per CTA. The
// z-contractions run in registers (the column's u and g_z), the x- and y-contractions read shared
// memory; each thread also owns the six face points with tangential indices (i, j), so the
// z-faces never touch shared memory and the neighbour z-lines are read coalesced.
template <int N, typename T>
struct ColShape {
  static constexpr int n2 = N * N;
  static constexpr int bytes_per_elem = (3 * N * N * N + 6 * N * N) * (int)sizeof(T);
  static constexpr int by_threads = n2 >= 256 ? 1 : 256 / n2;
  static constexpr int by_smem = (44 * 1024) / bytes_per_elem;
  static constexpr int epb = by_threads < by_smem ? by_threads : (by_smem < 1 ? 1 : by_smem);
  static constexpr int threads = epb * n2;
};

template <int N, typename T, int EPB>
__global__ void __launch_bounds__(EPB* N* N) apply_col_kernel(const OpGeom<T> g, const T* __restrict__ Dg,
                                                             const T* __restrict__ wg, const T* __restrict__ u,
                                                             const T* __restrict__ diag, const T* __restrict__ b,
                                                             T* __restrict__ out, int E) {
  constexpr int N2 = N * N, N3 = N * N * N, NT = EPB * N2;
  __shared__ T sD[N2];
  __shared__ T sw[N];
  __shared__ T su[EPB][N3];
  __shared__ T sv[EPB][2][N3];
  __shared__ T sfb[EPB][6][N2];
  const int tid = threadIdx.x;
  const int el = tid / N2, col = tid - el * N2;
  const int i = col % N, j = col / N;
  const int e0 = blockIdx.x * EPB;
  const int e = e0 + el;
  const bool valid = e < E;
  for (int t = tid; t < N2; t += NT) sD[t] = Dg[t];
  for (int t = tid; t < N; t += NT) sw[t] = wg[t];
  T uk[N], gz[N];
  const T* ue = u + (int64_t)e * N3;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    uk[k] = valid ? ue[(k * N + j) * N + i] : T(0);
    su[el][(k * N + j) * N + i] = uk[k];
  }
  __syncthreads();
  // local gradient: x, y from shared memory, z in registers
#pragma unroll
  for (int k = 0; k < N; ++k) {
    T gx = 0, gy = 0, gzk = 0;
#pragma unroll
    for (int l = 0; l < N; ++l) {
      gx += sD[i * N + l] * su[el][(k * N + j) * N + l];
      gy += sD[j * N + l] * su[el][(k * N + l) * N + i];
      gzk += sD[k * N + l] * uk[l];
    }
    sv[el][0][(k * N + j) * N + i] = g.dxi[0] * gx;
    sv[el][1][(k * N + j) * N + i] = g.dxi[1] * gy;
    gz[k] = g.dxi[2] * gzk;
  }
  __syncthreads();
  // the six face points with tangential indices (a1, a2) = (i, j)
  if (valid) {
    const int cx = e % g.nx, cy = (e / g.nx) % g.ny, cz = e / (g.nx * g.ny);
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const int d = f >> 1, side = f & 1;
      const T s = side ? T(1) : T(-1);
      const int idx = side ? N - 1 : 0, opp = side ? 0 : N - 1;
      // face point and neighbour line offsets (x-faces: y = i, z = j; y-faces: x = i, z = j; z-faces: x = i, y = j)
      int pf, base, stride;
      if (d == 0) { pf = (j * N + i) * N + idx; base = (j * N + i) * N; stride = 1; }
      else if (d == 1) { pf = (j * N + idx) * N + i; base = j * N2 + i; stride = N; }
      else { pf = (idx * N + j) * N + i; base = j * N + i; stride = N2; }
      const T dxi = d == 0 ? g.dxi[0] : (d == 1 ? g.dxi[1] : g.dxi[2]);
      const T lift = d == 0 ? g.lift[0] : (d == 1 ? g.lift[1] : g.lift[2]);
      const T sigma = d == 0 ? g.sigma[0] : (d == 1 ? g.sigma[1] : g.sigma[2]);
      const T Jf = d == 0 ? g.Jf[0] : (d == 1 ? g.Jf[1] : g.Jf[2]);
      const T u_int = d == 2 ? uk[idx] : su[el][pf];
      const T g_int = d == 2 ? gz[idx] : sv[el][d][pf];
      const int cd = d == 0 ? cx : (d == 1 ? cy : cz);
      const int nd = d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);
      const int cn = cd + (side ? 1 : -1);
      T u_ext, g_ext;
      if (cn >= 0 && cn < nd) {
        const int es = d == 0 ? 1 : (d == 1 ? g.nx : g.nx * g.ny);
        const T* uq = u + (int64_t)(e + (side ? es : -es)) * N3 + base;
        u_ext = __ldg(uq + opp * stride);
        T acc = 0;
#pragma unroll
        for (int l = 0; l < N; ++l) acc += sD[opp * N + l] * __ldg(uq + l * stride);
        g_ext = dxi * acc;
      } else {
        u_ext = -u_int;  // Dirichlet ghost state of Eq. bc with u_b = 0
        g_ext = g_int;
      }
      const T jump = u_ext - u_int;
      const T v_face = g_int + s * jump * lift;
      if (d == 2) gz[idx] = v_face;
      else sv[el][d][pf] = v_face;
      sfb[el][f][j * N + i] = Jf * sw[i] * sw[j] * (T(0.5) * s * (g_ext - g_int) + (sigma - lift) * jump);
    }
  }
  __syncthreads();
  if (!valid) return;
  // primal step: -M sum_d D_d v_d - ML [(n.v)^* - n.v]
  T* oe = out + (int64_t)e * N3;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    T dx = 0, dy = 0, dz = 0;
#pragma unroll
    for (int l = 0; l < N; ++l) {
      dx += sD[i * N + l] * sv[el][0][(k * N + j) * N + l];
      dy += sD[j * N + l] * sv[el][1][(k * N + l) * N + i];
      dz += sD[k * N + l] * gz[l];
    }
    const T M = g.J * sw[i] * sw[j] * sw[k];
    T res = -M * (g.dxi[0] * dx + g.dxi[1] * dy + g.dxi[2] * dz);
    if (i == 0) res -= sfb[el][0][k * N + j];
    if (i == N - 1) res -= sfb[el][1][k * N + j];
    if (j == 0) res -= sfb[el][2][k * N + i];
    if (j == N - 1) res -= sfb[el][3][k * N + i];
    if (k == 0) res -= sfb[el][4][j * N + i];
    if (k == N - 1) res -= sfb[el][5][j * N + i];
    const int p = (k * N + j) * N + i;
    if (diag) res += diag[(int64_t)e * N3 + p] * uk[k];
    oe[p] = b ? b[(int64_t)e * N3 + p] - res : res;
  }
}

template <int N, typename T>
static void launch_apply_n(const OpGeom<T>& g, const T* D, const T* w, const T* u, const T* diag, const T* b, T* out,
                           cudaStream_t s) {
  const int E = g.nx * g.ny * g.nz;
  using C = ColShape<N, T>;
  const int blocks = (E + C::epb - 1) / C::epb;
  apply_col_kernel<N, T, C::epb><<<blocks, C::threads, 0, s>>>(g, D, w, u, diag, b, out, E);
}

template <typename T>
void launch_apply(int N, const OpGeom<T>& g, const T* D, const T* w, const T* u, const T* diag, const T* b, T* out,
                  cudaStream_t s) {
  switch (N) {
    case 2: launch_apply_n<2, T>(g, D, w, u, diag, b, out, s); break;
    case 3: launch_apply_n<3, T>(g, D, w, u, diag, b, out, s); break;
    case 4: launch_apply_n<4, T>(g, D, w, u, diag, b, out, s); break;
    case 5: launch_apply_n<5, T>(g, D, w, u, diag, b, out, s); break;
    case 6: launch_apply_n<6, T>(g, D, w, u, diag, b, out, s); break;
    case 7: launch_apply_n<7, T>(g, D, w, u, diag, b, out, s); break;
    case 8: launch_apply_n<8, T>(g, D, w, u, diag, b, out, s); break;
    case 9: launch_apply_n<9, T>(g, D, w, u, diag, b, out, s); break;
    case 10: launch_apply_n<10, T>(g, D, w, u, diag, b, out, s); break;
    default: fail(DG_ERR_INVALID_ARG, "unsupported N");
  }
  DG_LAUNCHED(1);
}

template void launch_apply<double>(int, const OpGeom<double>&, const double*, const double*, const double*,
                                   const double*, const double*, double*, cudaStream_t);
template void launch_apply<float>(int, const OpGeom<float>&, const float*, const float*, const float*, const float*,
                                  const float*, float*, cudaStream_t);

// Diagonal of the LGL mass matrix, M = J w_i w_j w_k (Eq. massmat with collocation quadrature).
template <typename T>
__global__ void mass_kernel(int N, T J, const T* __restrict__ w, int64_t ndof, T* __restrict__ mass) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ndof) return;
  int p = (int)(t % (N * N * N));
  int i = p % N, j = (p / N) % N, k = p / (N * N);
  mass[t] = J * w[i] * w[j] * w[k];
}

template <typename T>
void launch_mass_diag(int N, const OpGeom<T>& g, const T* w, int64_t ndof, T* mass, cudaStream_t s) {
  if (ndof == 0) return;
  mass_kernel<T><<<(unsigned)((ndof + 255) / 256), 256, 0, s>>>(N, g.J, w, ndof, mass);
  DG_LAUNCHED(1);
}
template void launch_mass_diag<double>(int, const OpGeom<double>&, const double*, int64_t, double*, cudaStream_t);
template void launch_mass_diag<float>(int, const OpGeom<float>&, const float*, int64_t, float*, cudaStream_t);

__global__ void coords_kernel(int N, int nx, int ny, double lx, double ly, double lz, double hx, double hy, double hz,
                              const double* __restrict__ x1, int64_t ndof, double* X, double* Y, double* Z) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ndof) return;
  const int N3 = N * N * N;
  int64_t e = t / N3;
  int p = (int)(t - e * N3);
  int i = p % N, j = (p / N) % N, k = p / (N * N);
  int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
  X[t] = lx + hx * (ex + 0.5 * (x1[i] + 1.0));
  Y[t] = ly + hy * (ey + 0.5 * (x1[j] + 1.0));
  Z[t] = lz + hz * (ez + 0.5 * (x1[k] + 1.0));
}

void launch_node_coords(int N, const int n[3], const double lower[3], const double h[3], const double* x1, double* X,
                        double* Y, double* Z, cudaStream_t s) {
  int64_t ndof = (int64_t)n[0] * n[1] * n[2] * N * N * N;
  coords_kernel<<<(unsigned)((ndof + 255) / 256), 256, 0, s>>>(N, n[0], n[1], lower[0], lower[1], lower[2], h[0], h[1],
                                                               h[2], x1, ndof, X, Y, Z);
  DG_LAUNCHED(1);
}

}  // namespace dg
