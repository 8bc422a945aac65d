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
// GB300 mapping: EPB elements per CTA (EPB N^2 ~ 256 threads, one per (i, j) column); the element
// block, its x/y gradients and the face brackets stay in shared memory; neighbour face data (the
// neighbour's face value and normal derivative, which needs its whole normal line) is read straight
// from global memory, which L2 serves for the element-ordered sweep.
#include "internal.h"

namespace dg {

// One thread per (i, j) column of N points along z, EPB elements per CTA. The z-contractions run
// in registers (the column's u and g_z), the x- and y-contractions read shared memory; each thread
// also owns the six face points with tangential indices (i, j), so the z-faces never touch shared
// memory and the neighbour z-lines are read coalesced.
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
                                                             T* __restrict__ out, int E, const SubdomainOut so) {
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
  // residual written straight into the subdomain vectors: column and point-map offset of this
  // element's own subdomain (slot 0) and of each face neighbour's subdomain (slot 1 + (f ^ 1))
  __shared__ int s_col[EPB][7], s_map[EPB][7];
  for (int t = tid; so.rS && t < EPB * 7; t += NT) {
    const int el2 = t / 7, sl = t - el2 * 7;
    const int e2 = e0 + el2;
    int c = -1, m = 0;
    if (e2 < E) {
      int q = e2;
      if (sl > 0) {
        const int f = sl - 1, d = f >> 1;
        int c3[3] = {e2 % g.nx, (e2 / g.nx) % g.ny, e2 / (g.nx * g.ny)};
        const int nd = d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);
        c3[d] += (f & 1) ? 1 : -1;
        q = (c3[d] >= 0 && c3[d] < nd) ? c3[0] + g.nx * (c3[1] + g.ny * c3[2]) : -1;
      }
      if (q >= 0) {
        c = so.col_of_elem[q];
        m = (so.orient[q] * 7 + (sl == 0 ? 0 : 1 + ((sl - 1) ^ 1))) * N * N * N;
      }
    }
    s_col[el2][sl] = c;
    s_map[el2][sl] = m;
  }
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
  // the six face points with tangential indices (a1, a2) = (i, j). Branch-free: a face without a
  // neighbour reads the thread's own element (in bounds) and discards it, so the loads of all six
  // neighbour lines are independent and can be in flight together.
  if (valid) {
    const int cx = e % g.nx, cy = (e / g.nx) % g.ny, cz = e / (g.nx * g.ny);
    T u_ext[6], g_ext[6];
    unsigned external = 0;  // bit f: face f is on the domain boundary
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const int d = f >> 1, side = f & 1;
      const int opp = side ? 0 : N - 1;
      int base, stride;
      if (d == 0) { base = (j * N + i) * N; stride = 1; }
      else if (d == 1) { base = j * N2 + i; stride = N; }
      else { base = j * N + i; stride = N2; }
      const int cd = d == 0 ? cx : (d == 1 ? cy : cz);
      const int nd = d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);
      const int cn = cd + (side ? 1 : -1);
      const bool has = cn >= 0 && cn < nd;
      const int es = d == 0 ? 1 : (d == 1 ? g.nx : g.nx * g.ny);
      const T* uq = u + (int64_t)(has ? e + (side ? es : -es) : e) * N3 + base;
      T acc = 0, ue = 0;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        const T v = __ldg(uq + l * stride);
        acc += sD[opp * N + l] * v;
        if (l == opp) ue = v;
      }
      const T dxi = d == 0 ? g.dxi[0] : (d == 1 ? g.dxi[1] : g.dxi[2]);
      u_ext[f] = ue;
      g_ext[f] = dxi * acc;
      external |= (has ? 0u : 1u) << f;
    }
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const int d = f >> 1, side = f & 1;
      const T s = side ? T(1) : T(-1);
      const int idx = side ? N - 1 : 0;
      int pf;
      if (d == 0) pf = (j * N + i) * N + idx;
      else if (d == 1) pf = (j * N + idx) * N + i;
      else pf = (idx * N + j) * N + i;
      const T lift = d == 0 ? g.lift[0] : (d == 1 ? g.lift[1] : g.lift[2]);
      const T sigma = d == 0 ? g.sigma[0] : (d == 1 ? g.sigma[1] : g.sigma[2]);
      const T Jf = d == 0 ? g.Jf[0] : (d == 1 ? g.Jf[1] : g.Jf[2]);
      const T u_int = d == 2 ? uk[idx] : su[el][pf];
      const T g_int = d == 2 ? gz[idx] : sv[el][d][pf];
      const bool ext = (external >> f) & 1u;
      // Dirichlet ghost state of Eq. bc with u_b = 0 at external faces
      const T ue = ext ? -u_int : u_ext[f];
      const T ge = ext ? g_int : g_ext[f];
      const T jump = ue - u_int;
      const T v_face = g_int + s * jump * lift;
      if (d == 2) gz[idx] = v_face;
      else sv[el][d][pf] = v_face;
      sfb[el][f][j * N + i] = Jf * sw[i] * sw[j] * (T(0.5) * s * (ge - g_int) + (sigma - lift) * jump);
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
    const T val = b ? b[(int64_t)e * N3 + p] - res : res;
    if (!so.rS) {
      oe[p] = val;
    } else {
      // every subdomain row holds exactly one point, so these stores never collide
      const int cc[3] = {i, j, k};
#pragma unroll
      for (int sl = 0; sl < 7; ++sl) {
        const int c = s_col[el][sl];
        if (c < 0) continue;
        if (sl > 0) {
          // only points within N_overlap layers of a face belong to that neighbour's subdomain
          const int f = sl - 1, dd = f >> 1;
          const int depth = (f & 1) ? N - 1 - cc[dd] : cc[dd];
          if (depth >= so.ov) continue;
        }
        const int row = __ldg(so.inv + s_map[el][sl] + p);
        if (row >= 0) static_cast<T*>(so.rS)[(int64_t)c * so.ld + row] = val;
      }
    }
  }
}

template <int N, typename T>
static void launch_apply_n(const OpGeom<T>& g, const T* D, const T* w, const T* u, const T* diag, const T* b, T* out,
                           const SubdomainOut& so, cudaStream_t s) {
  const int E = g.nx * g.ny * g.nz;
  using C = ColShape<N, T>;
  constexpr int kSmall = N * N >= 32 ? 1 : (32 + N * N - 1) / (N * N);  // at least one warp per CTA
  if ((E + C::epb - 1) / C::epb >= 2 * 152 || C::epb <= kSmall) {
    const int blocks = (E + C::epb - 1) / C::epb;
    apply_col_kernel<N, T, C::epb><<<blocks, C::threads, 0, s>>>(g, D, w, u, diag, b, out, E, so);
  } else {
    // small grids: fewer elements per CTA so that every SM gets work
    const int blocks = (E + kSmall - 1) / kSmall;
    apply_col_kernel<N, T, kSmall><<<blocks, kSmall * N * N, 0, s>>>(g, D, w, u, diag, b, out, E, so);
  }
}

template <typename T>
void launch_apply(int N, const OpGeom<T>& g, const T* D, const T* w, const T* u, const T* diag, const T* b, T* out,
                  cudaStream_t s, const SubdomainOut* so_ptr) {
  const SubdomainOut so = so_ptr ? *so_ptr : SubdomainOut{};
  switch (N) {
    case 2: launch_apply_n<2, T>(g, D, w, u, diag, b, out, so, s); break;
    case 3: launch_apply_n<3, T>(g, D, w, u, diag, b, out, so, s); break;
    case 4: launch_apply_n<4, T>(g, D, w, u, diag, b, out, so, s); break;
    case 5: launch_apply_n<5, T>(g, D, w, u, diag, b, out, so, s); break;
    case 6: launch_apply_n<6, T>(g, D, w, u, diag, b, out, so, s); break;
    case 7: launch_apply_n<7, T>(g, D, w, u, diag, b, out, so, s); break;
    case 8: launch_apply_n<8, T>(g, D, w, u, diag, b, out, so, s); break;
    case 9: launch_apply_n<9, T>(g, D, w, u, diag, b, out, so, s); break;
    case 10: launch_apply_n<10, T>(g, D, w, u, diag, b, out, so, s); break;
    default: fail(DG_ERR_INVALID_ARG, "unsupported N");
  }
  DG_LAUNCHED(1);
}

template void launch_apply<double>(int, const OpGeom<double>&, const double*, const double*, const double*,
                                   const double*, const double*, double*, cudaStream_t, const SubdomainOut*);
template void launch_apply<float>(int, const OpGeom<float>&, const float*, const float*, const float*, const float*,
                                  const float*, float*, cudaStream_t, const SubdomainOut*);

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
