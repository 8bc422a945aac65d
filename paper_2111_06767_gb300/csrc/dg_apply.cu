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
// g_ext = g_int, which this kernel uses on Dirichlet faces. On a homogeneous Neumann face of the
// box (Eq. bc with (n F_v)^b = (n F_v)^int and a zero prescribed normal flux (n F_u)^b = 0) the
// ghost state is u_ext = u_int, g_ext = -g_int: no jump, no lifting and a zero numerical flux.
//
// GB300 mapping: one thread per x-line of N points (the N contiguous values of u[e][k][j][:]),
// N^2 threads per element, EPB elements per CTA. Every global access is a coalesced vector access of
// whole lines: the element itself, the two x-neighbour lines at the same (j, k) (kept in registers)
// and the matching lines of the four y/z neighbours (staged in shared memory, which L2 serves for
// the element-ordered sweep). The x-contractions run in registers with Dhat read from constant
// memory; the y- and z-contractions read whole lines from shared memory, which the threads of one
// plane (y) or one column of planes (z) share as broadcasts, with the planes padded so that the
// lines of one access fall into distinct banks.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <set>
#include <type_traits>

#include "bounds.cuh"
#include "internal.h"
#include "lines.cuh"
#include "pdl.cuh"
#include "schwarz_dev.cuh"

namespace dg {

namespace {

// Dhat and the LGL weights of every supported N, concatenated in constant memory, so that the
// x-contraction and the per-point quadrature weights with unrolled (compile-time) indices are
// operands of the FMA instructions themselves.
constexpr int dtab_off(int N) { return (N - 1) * N * (2 * N - 1) / 6 - 1; }  // sum_{m=2}^{N-1} m^2
constexpr int wtab_off(int N) { return N * (N - 1) / 2 - 1; }                 // sum_{m=2}^{N-1} m
constexpr int kDTab = dtab_off(DG_MAX_N + 1), kWTab = wtab_off(DG_MAX_N + 1);
__constant__ double cD64[kDTab];
__constant__ float cD32[kDTab];
__constant__ double cW64[kWTab];
__constant__ float cW32[kWTab];

template <typename T>
struct CTab;
template <>
struct CTab<double> {
  static __device__ __forceinline__ double D(int o) { return cD64[o]; }
  static __device__ __forceinline__ double w(int o) { return cW64[o]; }
};
template <>
struct CTab<float> {
  static __device__ __forceinline__ float D(int o) { return cD32[o]; }
  static __device__ __forceinline__ float w(int o) { return cW32[o]; }
};

// Shared-memory shape. A block holds one element as N planes (k) of N lines (j) of N points (i).
// The plane stride P is padded so that the lines one y-contraction reads at once (one per plane
// of the warp's threads) fall into distinct banks: where a line is a power-of-two fraction of the
// 128-byte bank sweep, P is an odd number of lines (consecutive planes, and with them consecutive
// elements, then land on distinct line slots); otherwise consecutive planes shift by one line.
// Per element: five blocks (u and the four y/z neighbours; the neighbour blocks are later reused
// for v_y, v_z and the face fluxes) and, for each of the four y/z faces, the neighbour's value and
// normal derivative at the face points (N^2 each).
template <int N, typename T>
struct LineShape {
  static constexpr int s = (int)sizeof(T);
  static constexpr int line = N * s;
  static constexpr int P = (128 % line == 0) ? N * (N % 2 == 0 ? N + 1 : N)
                                             : N * N + ((N - N * N) % (128 / s) + (128 / s)) % (128 / s);
  static constexpr int R = N * P;
  static constexpr int n2 = N * N;
  static constexpr int per_elem = (5 * R + 8 * n2) * s + 14 * (int)sizeof(int);
  static constexpr int by_threads = n2 >= 256 ? 1 : 256 / n2;
  static constexpr int by_smem = (47 * 1024) / per_elem;
  static constexpr int cap = by_threads < by_smem ? by_threads : (by_smem < 1 ? 1 : by_smem);
  // largest count up to the cap that fills whole warps, if there is one
  static constexpr int whole(int e) { return e < 1 ? cap : ((e * n2) % 32 == 0 ? e : whole(e - 1)); }
  static constexpr int epb = whole(cap);
};

// Lifting and primal flux at one face point of normal s e_d: from the interior value ui and local
// gradient component gi, the neighbour's value ue and normal derivative ge (has = the neighbour
// exists; otherwise the ghost state of Eq. bc: u_E = -u_i, g_E = g_i on a homogeneous Dirichlet
// face, u_E = u_i, g_E = -g_i on a homogeneous Neumann face (neu), which makes the jump and the
// numerical normal flux vanish), returns the lifted v_d and adds the flux term of the point,
// weighted by the face quadrature weight Bf, to fl.
template <typename T>
__device__ __forceinline__ T face_point(T s, T ui, T gi, T ue, T ge, bool has, bool neu, T lift,
                                        T sigma_minus_lift, T Bf, T& fl) {
  const T uE = has ? ue : (neu ? ui : -ui);
  const T gE = has ? ge : (neu ? -gi : gi);
  const T jump = uE - ui;
  fl -= Bf * (T(0.5) * s * (gE - gi) + sigma_minus_lift * jump);
  return gi + s * jump * lift;
}

// y[i] += d x[i] along a line: in FP32 as packed two-wide FMAs on pairs of points (one instruction
// per pair, same rounding as the scalar FMA), in FP64 scalar.
template <int N, typename T>
__device__ __forceinline__ void axpy_line(T d, const T (&x)[N], T (&y)[N]) {
  if constexpr (std::is_same<T, float>::value) {
    const float2 dd = make_float2(d, d);
#pragma unroll
    for (int i = 0; i + 1 < N; i += 2) {
      const float2 r = __ffma2_rn(dd, make_float2(x[i], x[i + 1]), make_float2(y[i], y[i + 1]));
      y[i] = r.x;
      y[i + 1] = r.y;
    }
    if constexpr (N % 2 == 1) y[N - 1] += d * x[N - 1];
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) y[i] += d * x[i];
  }
}

// One group of EPB elements (block index blk) of the DG apply, for the kernel below and for the
// fused coarse-level smoother; with PDL the set-up before the first read of u overlaps the
// previous kernel on the stream.
template <int N, typename T, int EPB, bool PDL, bool L2ONLY = false>
__device__ __forceinline__ void apply_line_block(const ApplyArgs<T>& A, int blk) {
  const OpGeom<T>& g = A.g;
  const T* __restrict__ Dg = A.D;
  const T* __restrict__ wg = A.w;
  const T* __restrict__ u = A.u;
  const T* __restrict__ diag = A.diag;
  const T* __restrict__ b = A.b;
  T* __restrict__ out = A.out;
  const int E = A.E;
  T* __restrict__ rS = A.rS;
  const int ld = A.ld, ov = A.ov;
  const int* __restrict__ col_of_elem = A.col_of_elem;
  const int* __restrict__ orient = A.orient;
  const int* __restrict__ inv = A.inv;
  using S = LineShape<N, T>;
  using C = CTab<T>;
  constexpr int N2 = N * N, N3 = N2 * N, P = S::P, R = S::R, NT = EPB * N2;
  constexpr int dO = dtab_off(N), wO = wtab_off(N);
  __shared__ __align__(16) T sm[5][EPB][R];
  // y/z face data per face (0..3 = -y, +y, -z, +z): [neighbour value, neighbour normal derivative]
  // [element][tangential point: (k, i) on y faces, (j, i) on z faces]
  __shared__ __align__(16) T sf[4][2][EPB][N2];
  // residual written straight into the subdomain vectors: column and point-map offset of this
  // element's own subdomain (slot 0) and of each face neighbour's subdomain (slot 1 + (f ^ 1))
  __shared__ int s_col[EPB][7], s_map[EPB][7];
  if constexpr (PDL) pdl_launch_dependents();
  const int tid = threadIdx.x;
  const int el = tid / N2, t = tid - el * N2;
  const int j = t % N, k = t / N;
  const int e0 = blk * EPB;
  const int e = e0 + el;
  const bool valid = e < E;
  const int ec = valid ? e : E - 1;  // threads past the end load a real element and store nothing
  const int nx = g.nx, ny = g.ny, nxy = g.nx * g.ny;
  const int cx = ec % nx, cy = (ec / nx) % ny, cz = ec / nxy;
  const bool hxm = cx > 0, hxp = cx + 1 < nx, hym = cy > 0, hyp = cy + 1 < ny, hzm = cz > 0, hzp = cz + 1 < g.nz;
  for (int q = tid; rS && q < EPB * 7; q += NT) {
    const int el2 = q / 7, sl = q - el2 * 7;
    const int e2 = e0 + el2;
    int c = -1, m = 0;
    if (e2 < E) {
      int r = e2;
      if (sl > 0) {
        const int f = sl - 1, d = f >> 1;
        int c3[3] = {e2 % nx, (e2 / nx) % ny, e2 / nxy};
        const int nd = d == 0 ? nx : (d == 1 ? ny : g.nz);
        c3[d] += (f & 1) ? 1 : -1;
        r = (c3[d] >= 0 && c3[d] < nd) ? c3[0] + nx * (c3[1] + ny * c3[2]) : -1;
      }
      if (r >= 0) {
        c = col_of_elem[r];
        m = (orient[r] * 7 + (sl == 0 ? 0 : 1 + ((sl - 1) ^ 1))) * N3;
      }
    }
    s_col[el2][sl] = c;
    s_map[el2][sl] = m;
  }
  // rows j and k of Dhat, scaled by 2/h_y and 2/h_z, and the weights (static data: read before
  // waiting for the previous kernel)
  T Dj[N], Dk[N];
#pragma unroll
  for (int l = 0; l < N; ++l) {
    Dj[l] = g.dxi[1] * __ldg(Dg + j * N + l);
    Dk[l] = g.dxi[2] * __ldg(Dg + k * N + l);
  }
  const T wj = __ldg(wg + j), wk = __ldg(wg + k);
  if constexpr (PDL) pdl_wait();
  // all loads of the thread's seven lines first (a missing neighbour reads the element itself and
  // is replaced by the ghost state), then the shared-memory stores
  const int64_t line = (int64_t)t * N;
  T ul[N], xm[N], xp[N], ym[N], yp[N], zm[N], zp[N];
  gld_line<N, T, L2ONLY>(u + (int64_t)ec * N3 + line, ul);
  gld_line<N, T, L2ONLY>(u + (int64_t)(hxm ? ec - 1 : ec) * N3 + line, xm);
  gld_line<N, T, L2ONLY>(u + (int64_t)(hxp ? ec + 1 : ec) * N3 + line, xp);
  gld_line<N, T, L2ONLY>(u + (int64_t)(hym ? ec - nx : ec) * N3 + line, ym);
  gld_line<N, T, L2ONLY>(u + (int64_t)(hyp ? ec + nx : ec) * N3 + line, yp);
  gld_line<N, T, L2ONLY>(u + (int64_t)(hzm ? ec - nxy : ec) * N3 + line, zm);
  gld_line<N, T, L2ONLY>(u + (int64_t)(hzp ? ec + nxy : ec) * N3 + line, zp);
  const int so = k * P + j * N;  // this thread's line within a block
  sst_line<N>(&sm[0][el][so], ul);
  sst_line<N>(&sm[1][el][so], ym);
  sst_line<N>(&sm[2][el][so], yp);
  sst_line<N>(&sm[3][el][so], zm);
  sst_line<N>(&sm[4][el][so], zp);
  // x-neighbour traces: the value on the shared face and the neighbour's normal derivative there
  const T uxm = xm[N - 1], uxp = xp[0];
  T gxm = T(0), gxp = T(0);
#pragma unroll
  for (int l = 0; l < N; ++l) {
    gxm += C::D(dO + (N - 1) * N + l) * xm[l];
    gxp += C::D(dO + l) * xp[l];
  }
  gxm *= g.dxi[0];
  gxp *= g.dxi[0];
  __syncthreads();
  // y/z face data, one face point per thread and face (all threads share the work): on the y faces
  // the point (i, k) = (j, k), on the z faces the point (i, j) = (k, j)
  {
    T gmy = T(0), gpy = T(0), gmz = T(0), gpz = T(0);
#pragma unroll
    for (int l = 0; l < N; ++l) {
      gmy += C::D(dO + (N - 1) * N + l) * sm[1][el][k * P + l * N + j];
      gpy += C::D(dO + l) * sm[2][el][k * P + l * N + j];
      gmz += C::D(dO + (N - 1) * N + l) * sm[3][el][l * P + j * N + k];
      gpz += C::D(dO + l) * sm[4][el][l * P + j * N + k];
    }
    const int py = k * N + j, pz = j * N + k;
    sf[0][0][el][py] = sm[1][el][k * P + (N - 1) * N + j];
    sf[0][1][el][py] = g.dxi[1] * gmy;
    sf[1][0][el][py] = sm[2][el][k * P + j];
    sf[1][1][el][py] = g.dxi[1] * gpy;
    sf[2][0][el][pz] = sm[3][el][(N - 1) * P + j * N + k];
    sf[2][1][el][pz] = g.dxi[2] * gmz;
    sf[3][0][el][pz] = sm[4][el][j * N + k];
    sf[3][1][el][pz] = g.dxi[2] * gpz;
  }
  // local gradient: x in registers, y and z from the lines of the element block
  T vx[N], vy[N], vz[N], tmp[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T a = T(0);
#pragma unroll
    for (int l = 0; l < N; ++l) a += C::D(dO + i * N + l) * ul[l];
    vx[i] = g.dxi[0] * a;
    vy[i] = T(0);
    vz[i] = T(0);
  }
#pragma unroll
  for (int l = 0; l < N; ++l) {
    sld_line<N>(&sm[0][el][k * P + l * N], tmp);
    axpy_line<N>(Dj[l], tmp, vy);
  }
#pragma unroll
  for (int l = 0; l < N; ++l) {
    sld_line<N>(&sm[0][el][l * P + j * N], tmp);
    axpy_line<N>(Dk[l], tmp, vz);
  }
  // x faces in registers: lifting into v_x at i = 0 and N-1, primal flux into o
  T o[N];
#pragma unroll
  for (int i = 0; i < N; ++i) o[i] = T(0);
  {
    const T Bf = g.Jf[0] * wj * wk, sml = g.sigma[0] - g.lift[0];
    vx[0] = face_point(T(-1), ul[0], vx[0], uxm, gxm, hxm, g.neumann & 1, g.lift[0], sml, Bf, o[0]);
    vx[N - 1] = face_point(T(1), ul[N - 1], vx[N - 1], uxp, gxp, hxp, (g.neumann >> 1) & 1, g.lift[0], sml, Bf,
                           o[N - 1]);
  }
  __syncthreads();  // face data written; every read of the neighbour blocks is done
  sst_line<N>(&sm[1][el][so], vy);
  sst_line<N>(&sm[2][el][so], vz);
  __syncthreads();
  // y/z faces, one point per thread and face: lift v_y (block 1) / v_z (block 2) in shared memory,
  // fluxes into blocks 3 (y faces) and 4 (z faces) at offsets 0 (lower) and N^2 (upper)
  {
    const T Bf = wj * wk;  // w_i w_k on y faces (i = j), w_i w_j on z faces (i = k)
    const int py = k * N + j, pz = j * N + k;
    T fl = T(0);
    T* v = &sm[1][el][k * P + j];
    *v = face_point(T(-1), sm[0][el][k * P + j], *v, sf[0][0][el][py], sf[0][1][el][py], hym, (g.neumann >> 2) & 1,
                    g.lift[1], g.sigma[1] - g.lift[1], g.Jf[1] * Bf, fl);
    sm[3][el][py] = fl;
    fl = T(0);
    v = &sm[1][el][k * P + (N - 1) * N + j];
    *v = face_point(T(1), sm[0][el][k * P + (N - 1) * N + j], *v, sf[1][0][el][py], sf[1][1][el][py], hyp,
                    (g.neumann >> 3) & 1, g.lift[1], g.sigma[1] - g.lift[1], g.Jf[1] * Bf, fl);
    sm[3][el][N2 + py] = fl;
    fl = T(0);
    v = &sm[2][el][j * N + k];
    *v = face_point(T(-1), sm[0][el][j * N + k], *v, sf[2][0][el][pz], sf[2][1][el][pz], hzm, (g.neumann >> 4) & 1,
                    g.lift[2], g.sigma[2] - g.lift[2], g.Jf[2] * Bf, fl);
    sm[4][el][pz] = fl;
    fl = T(0);
    v = &sm[2][el][(N - 1) * P + j * N + k];
    *v = face_point(T(1), sm[0][el][(N - 1) * P + j * N + k], *v, sf[3][0][el][pz], sf[3][1][el][pz], hzp,
                    (g.neumann >> 5) & 1, g.lift[2], g.sigma[2] - g.lift[2], g.Jf[2] * Bf, fl);
    sm[4][el][N2 + pz] = fl;
  }
  __syncthreads();
  // y/z face fluxes of the thread's own points
  if (j == 0) {
    sld_line<N>(&sm[3][el][k * N], tmp);
#pragma unroll
    for (int i = 0; i < N; ++i) o[i] += tmp[i];
  }
  if (j == N - 1) {
    sld_line<N>(&sm[3][el][N2 + k * N], tmp);
#pragma unroll
    for (int i = 0; i < N; ++i) o[i] += tmp[i];
  }
  if (k == 0) {
    sld_line<N>(&sm[4][el][j * N], tmp);
#pragma unroll
    for (int i = 0; i < N; ++i) o[i] += tmp[i];
  }
  if (k == N - 1) {
    sld_line<N>(&sm[4][el][N2 + j * N], tmp);
#pragma unroll
    for (int i = 0; i < N; ++i) o[i] += tmp[i];
  }
  // primal step: -M sum_d D_d v_d - ML [(n.v)^* - n.v]
  T dy[N], dz[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    dy[i] = T(0);
    dz[i] = T(0);
  }
#pragma unroll
  for (int l = 0; l < N; ++l) {
    sld_line<N>(&sm[1][el][k * P + l * N], tmp);
    axpy_line<N>(Dj[l], tmp, dy);
  }
#pragma unroll
  for (int l = 0; l < N; ++l) {
    sld_line<N>(&sm[2][el][l * P + j * N], tmp);
    axpy_line<N>(Dk[l], tmp, dz);
  }
  if (!valid) return;
  const int64_t base = (int64_t)ec * N3 + line;
  T dl[N], bl[N];
  if (diag) gld_line<N>(diag + base, dl);
  if (b) gld_line<N>(b + base, bl);
  T val[N];
  const T M0 = g.J * wj * wk;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T dx = T(0);
#pragma unroll
    for (int l = 0; l < N; ++l) dx += C::D(dO + i * N + l) * vx[l];
    T res = -(M0 * C::w(wO + i)) * (g.dxi[0] * dx + dy[i] + dz[i]) + o[i];
    if (diag) res += dl[i] * ul[i];
    val[i] = b ? bl[i] - res : res;
  }
  if (!rS) {
    gst_line<N>(out + base, val);
    return;
  }
  // every subdomain row holds exactly one point, so these stores never collide; unrolled so that
  // the seven row-table loads are in flight together
#pragma unroll
  for (int sl = 0; sl < 7; ++sl) {
    const int c = s_col[el][sl];
    if (c < 0) continue;
    int lo = 0, hi = N;  // points of the line inside this slot's subdomain (N_overlap layers of a face)
    if (sl > 0) {
      const int f = sl - 1, dd = f >> 1, side = f & 1;
      if (dd == 0) {
        if (side) lo = N - ov;
        else hi = ov;
      } else {
        const int cc = dd == 1 ? j : k;
        if ((side ? N - 1 - cc : cc) >= ov) continue;
      }
    }
    int rows[N];
    gld_line<N>(inv + s_map[el][sl] + t * N, rows);
    if (!DG_IN_BOUNDS(c, E)) continue;
    T* colp = rS + (int64_t)c * ld;
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i >= lo && i < hi && rows[i] >= 0 && DG_IN_BOUNDS(rows[i], ld)) colp[rows[i]] = val[i];
  }
}

template <int N, typename T, int EPB>
__global__ void __launch_bounds__(EPB* N* N) apply_line_kernel(const ApplyArgs<T> A) {
  apply_line_block<N, T, EPB, true>(A, blockIdx.x);
}

// ------------------------------------------------------------------ slice-per-thread apply (N = 4, FP32)
//
// The line kernel's y- and z-contractions read lines of other threads from shared memory, and at
// N = 4 in FP32 its shared-memory wavefronts, not HBM, set the pace. For the plain apply at N = 4
// a thread here owns one x-z slice (fixed y index q: the four x-lines of the four z-planes, 16
// points) of one element: the x- and z-contractions run in registers and the y-contractions take
// the other three slices of the element from the neighbouring lanes with warp shuffles (the four
// threads of an element are consecutive lanes). The four threads of an element load their slices
// as one contiguous 64-byte run per plane, for the element itself and for every neighbour;
// x-neighbours inside the CTA are read back from shared memory (68-word element stride, distinct
// banks); the y-neighbours' normal derivatives at the shared faces are summed over the element's
// four threads with shuffles as well: thread q loads neighbour slice 3 - q, so the thread on the
// face also holds the neighbour's face values.
constexpr int kSliceEPB = 32;     // elements per CTA (128 threads)
constexpr int kSliceStride = 68;  // words per element in shared memory

__device__ __forceinline__ void row4(const float* p, float (&r)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  r[0] = v.x;
  r[1] = v.y;
  r[2] = v.z;
  r[3] = v.w;
}
__device__ __forceinline__ void row4_g(const float* __restrict__ p, float (&r)[4]) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  r[0] = v.x;
  r[1] = v.y;
  r[2] = v.z;
  r[3] = v.w;
}

__global__ void __launch_bounds__(kSliceEPB * 4, 4) apply_slice4_kernel(const ApplyArgs<float> A) {
  constexpr int N = 4, N3 = 64;
  constexpr int dO = dtab_off(N), wO = wtab_off(N);
  using C = CTab<float>;
  __shared__ __align__(16) float su[kSliceEPB * kSliceStride];
  const OpGeom<float>& g = A.g;
  const float* __restrict__ u = A.u;
  const int tid = threadIdx.x;
  const int el = tid >> 2, q = tid & 3;  // element of the CTA, y index of the thread's slice
  const int E = A.E;
  const int e0 = blockIdx.x * kSliceEPB;
  const int n_el = min(kSliceEPB, E - e0);
  const int e = e0 + el;
  const bool valid = el < n_el;
  const int ec = valid ? e : E - 1;  // threads past the end compute on a real element, store nothing
  pdl_launch_dependents();
  pdl_wait();
  const int nx = g.nx, ny = g.ny, nxy = g.nx * g.ny;
  const int cx = ec % nx, cy = (ec / nx) % ny, cz = ec / nxy;
  const bool hxm = cx > 0, hxp = cx + 1 < nx, hym = cy > 0, hyp = cy + 1 < ny, hzm = cz > 0, hzp = cz + 1 < g.nz;
  // own slice: U[kk][i] = u(i, q, kk)
  float U[4][4];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) row4_g(u + (int64_t)ec * N3 + kk * 16 + q * 4, U[kk]);
#pragma unroll
  for (int kk = 0; kk < 4; ++kk)
    *reinterpret_cast<float4*>(&su[el * kSliceStride + kk * 16 + q * 4]) =
        make_float4(U[kk][0], U[kk][1], U[kk][2], U[kk][3]);
  // z-neighbour traces on the slice's face rows (kk = 0: z-, kk = 3: z+), in the thread
  float uzm[4], gzm[4], uzp[4], gzp[4];
  {
    float r[4][4];
#pragma unroll
    for (int l = 0; l < 4; ++l) row4_g(u + (int64_t)(hzm ? ec - nxy : ec) * N3 + l * 16 + q * 4, r[l]);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      uzm[i] = r[3][i];
      float a = 0.f;
#pragma unroll
      for (int l = 0; l < 4; ++l) a += C::D(dO + 3 * N + l) * r[l][i];
      gzm[i] = g.dxi[2] * a;
    }
#pragma unroll
    for (int l = 0; l < 4; ++l) row4_g(u + (int64_t)(hzp ? ec + nxy : ec) * N3 + l * 16 + q * 4, r[l]);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      uzp[i] = r[0][i];
      float a = 0.f;
#pragma unroll
      for (int l = 0; l < 4; ++l) a += C::D(dO + l) * r[l][i];
      gzp[i] = g.dxi[2] * a;
    }
  }
  // y-neighbour traces on the element's y faces (q = 0: y-, q = 3: y+), summed over the element's
  // four threads
  float uyE[4][4], gyE[4][4];
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const int nb = side ? (hyp ? ec + nx : ec) : (hym ? ec - nx : ec);
    const int sl = 3 - q;  // the neighbour slice this thread loads
    float r[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) row4_g(u + (int64_t)nb * N3 + kk * 16 + sl * 4, r[kk]);
    const float cf = C::D(dO + (side ? 0 : 3 * N) + sl) * g.dxi[1];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float a = cf * r[kk][i];
        a += __shfl_xor_sync(0xffffffffu, a, 1);
        a += __shfl_xor_sync(0xffffffffu, a, 2);
        if (q == (side ? 3 : 0)) {  // the face thread: slice 3 - q is the neighbour's face slice
          uyE[kk][i] = r[kk][i];
          gyE[kk][i] = a;
        }
      }
  }
  __syncthreads();  // the CTA's slices are in shared memory
  // x-neighbour lines of this slice (from shared memory inside the CTA)
  float uxm[4], gxm[4], uxp[4], gxp[4];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    float r[4];
    if (hxm && el > 0) row4(&su[(el - 1) * kSliceStride + kk * 16 + q * 4], r);
    else row4_g(u + (int64_t)(hxm ? ec - 1 : ec) * N3 + kk * 16 + q * 4, r);
    uxm[kk] = r[3];
    float a = 0.f;
#pragma unroll
    for (int l = 0; l < 4; ++l) a += C::D(dO + 3 * N + l) * r[l];
    gxm[kk] = g.dxi[0] * a;
    if (hxp && el + 1 < n_el) row4(&su[(el + 1) * kSliceStride + kk * 16 + q * 4], r);
    else row4_g(u + (int64_t)(hxp ? ec + 1 : ec) * N3 + kk * 16 + q * 4, r);
    uxp[kk] = r[0];
    a = 0.f;
#pragma unroll
    for (int l = 0; l < 4; ++l) a += C::D(dO + l) * r[l];
    gxp[kk] = g.dxi[0] * a;
  }
  // local gradient: x along the thread's lines, z across its planes, y across the element's slices
  float vx[4][4], vy[4][4], vz[4][4];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float ax = 0.f, az = 0.f;
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        ax += C::D(dO + i * N + l) * U[kk][l];
        az += C::D(dO + kk * N + l) * U[l][i];
      }
      vx[kk][i] = g.dxi[0] * ax;
      vz[kk][i] = g.dxi[2] * az;
      vy[kk][i] = 0.f;
    }
  // row q of Dhat (times 2/h_y) in partner order: Dy[m] multiplies the slice of thread q ^ m
  float Dy[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    float d = 0.f;
#pragma unroll
    for (int qq = 0; qq < 4; ++qq)  // compile-time constant-memory addresses, selected per lane
      if (qq == q) d = C::D(dO + qq * N + (qq ^ m));
    Dy[m] = g.dxi[1] * d;
  }
  // y across the element's slices: the other three threads' values by warp shuffles
#pragma unroll
  for (int kk = 0; kk < 4; ++kk)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float x = U[kk][i];
      vy[kk][i] = Dy[0] * x + Dy[1] * __shfl_xor_sync(0xffffffffu, x, 1) + Dy[2] * __shfl_xor_sync(0xffffffffu, x, 2) +
                  Dy[3] * __shfl_xor_sync(0xffffffffu, x, 3);
    }
  // faces: lifting into v, primal fluxes into o (Eq. numflux with the ghost states of Eq. bc)
  float o[4][4];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk)
#pragma unroll
    for (int i = 0; i < 4; ++i) o[kk][i] = 0.f;
  const float wq = C::w(wO + q);
  {
    const float smx = g.sigma[0] - g.lift[0], smy = g.sigma[1] - g.lift[1], smz = g.sigma[2] - g.lift[2];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const float Bf = g.Jf[0] * wq * C::w(wO + kk);
      vx[kk][0] = face_point(-1.f, U[kk][0], vx[kk][0], uxm[kk], gxm[kk], hxm, g.neumann & 1, g.lift[0], smx, Bf,
                             o[kk][0]);
      vx[kk][3] = face_point(1.f, U[kk][3], vx[kk][3], uxp[kk], gxp[kk], hxp, (g.neumann >> 1) & 1, g.lift[0], smx,
                             Bf, o[kk][3]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float Bf = g.Jf[2] * C::w(wO + i) * wq;
      vz[0][i] = face_point(-1.f, U[0][i], vz[0][i], uzm[i], gzm[i], hzm, (g.neumann >> 4) & 1, g.lift[2], smz, Bf,
                            o[0][i]);
      vz[3][i] = face_point(1.f, U[3][i], vz[3][i], uzp[i], gzp[i], hzp, (g.neumann >> 5) & 1, g.lift[2], smz, Bf,
                            o[3][i]);
    }
    if (q == 0 || q == 3) {
      const float s = q ? 1.f : -1.f;
      const bool has = q ? hyp : hym;
      const bool neu = (g.neumann >> (q ? 3 : 2)) & 1;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int i = 0; i < 4; ++i)
          vy[kk][i] = face_point(s, U[kk][i], vy[kk][i], uyE[kk][i], gyE[kk][i], has, neu, g.lift[1], smy,
                                 g.Jf[1] * C::w(wO + i) * C::w(wO + kk), o[kk][i]);
    }
  }
  // divergence: y across the slices of the lifted v_y, by warp shuffles
  float dy[4][4];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float x = vy[kk][i];
      dy[kk][i] = Dy[0] * x + Dy[1] * __shfl_xor_sync(0xffffffffu, x, 1) + Dy[2] * __shfl_xor_sync(0xffffffffu, x, 2) +
                  Dy[3] * __shfl_xor_sync(0xffffffffu, x, 3);
    }
  if (!valid) return;
  const int64_t base = (int64_t)ec * N3 + q * 4;
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    float val[4], dl[4], bl[4];
    if (A.diag) row4_g(A.diag + base + kk * 16, dl);
    if (A.b) row4_g(A.b + base + kk * 16, bl);
    const float M0 = g.J * wq * C::w(wO + kk);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float dx = 0.f, dz = 0.f;
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        dx += C::D(dO + i * N + l) * vx[kk][l];
        dz += C::D(dO + kk * N + l) * vz[l][i];
      }
      float res = -(M0 * C::w(wO + i)) * (g.dxi[0] * dx + dy[kk][i] + g.dxi[2] * dz) + o[kk][i];
      if (A.diag) res += dl[i] * U[kk][i];
      val[i] = A.b ? bl[i] - res : res;
    }
    *reinterpret_cast<float4*>(A.out + base + kk * 16) = make_float4(val[0], val[1], val[2], val[3]);
  }
}

// ------------------------------------------------------------------ element-per-thread apply (N = 4, FP32)
//
// At N = 4 an element is 64 values, few enough for one thread to hold the element, one gradient
// component and the result in registers, so the three contractions need no exchange between
// threads at all. A CTA owns a brick of BX x BY x BZ elements. One TMA load stages the brick with a
// one-element halo ((BX+2) x (BY+2) x (BZ+2) elements; elements outside the domain arrive as zeros
// and are replaced by the ghost state) in shared memory, each element padded from 64 to 68 words:
// the 16-byte reads of consecutive elements at one offset then fall into distinct banks. A thread
// reads its element and its six face neighbours from there (a neighbour's normal derivative at the
// shared face needs its whole element), works direction by direction (gradient component, face
// lifting and fluxes, divergence), and the result leaves through the same padded layout with one
// TMA store, which clips elements outside the domain. The flux of a face point enters the per-point
// sum before the mass-matrix scaling, divided by that point's M: Bf / M = Jf_d / (J w_0) at every
// face point of a face normal to d. Values are held as pairs of x-neighbouring points, so that the
// contractions and most face terms run as packed two-wide FP32 FMAs (one instruction per pair):
// the thread's 64-value working set leaves too few warps per SM to hide latency otherwise.
constexpr int kE4Slot = 68;  // words per staged element

template <int BX, int BY, int BZ>
struct E4Shape {
  static constexpr int PX = BX + 2, PY = BY + 2, PZ = BZ + 2;
  static constexpr int THREADS = BX * BY * BZ;
  static constexpr int IN_WORDS = PX * PY * PZ * kE4Slot;
  static constexpr int SMEM = IN_WORDS * 4 + 16 + 128;  // staged box, mbarrier, alignment slack
  static constexpr int PER_SM = (228 * 1024) / (SMEM + 1024) > 8 ? 8 : (228 * 1024) / (SMEM + 1024);
  static_assert(PER_SM >= 1 && SMEM <= 227 * 1024, "staged brick must fit in shared memory");
  static_assert(BX <= 254 && BY <= 254 && BZ <= 254, "TMA boxes are at most 256 elements per dimension");
};

constexpr uint32_t kE4WaitPolls = 1u << 20;  // polls before the staging wait gives up

__device__ __forceinline__ uint32_t e4_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool e4_wait(uint32_t bar, int* err) {
  for (uint32_t it = 0; it < kE4WaitPolls; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P1;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], 0;\n\t"
        "selp.u32 %0, 1, 0, P1;\n\t}"
        : "=r"(ok)
        : "r"(bar)
        : "memory");
    if (ok) return true;
  }
  if (err) atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void ld4p(const float* p, float2 (&r)[2]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  r[0] = make_float2(v.x, v.y);
  r[1] = make_float2(v.z, v.w);
}

__device__ __forceinline__ void ld4s(const float* p, float (&r)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  r[0] = v.x;
  r[1] = v.y;
  r[2] = v.z;
  r[3] = v.w;
}

// Lifting and flux of one face point, as face_point() above, with the flux added to the point's
// pre-mass sum acc (cf = Bf / M of the point).
__device__ __forceinline__ float e4_face(float s, float ui, float gi, float ue, float ge, bool has, bool neu,
                                         float lift, float sml, float cf, float& acc) {
  const float uE = has ? ue : (neu ? ui : -ui);
  const float gE = has ? ge : (neu ? -gi : gi);
  const float jump = uE - ui;
  acc += cf * (0.5f * s * (gE - gi) + sml * jump);
  return gi + s * jump * lift;
}

// Ghost-state blend of one face (Eq. bc): the exterior value is a ue + b ui and the exterior
// normal derivative c ge + d gi, with (a, b, c, d) = (1, 0, 1, 0) where the neighbour exists, else
// (0, -1, 0, 1) on a Dirichlet and (0, 1, 0, -1) on a Neumann face.
struct E4Face {
  float2 a, b, c, d, hs, sl, sml, cf;  // hs = s / 2, sl = s lift (both halves equal)
  __device__ __forceinline__ E4Face(float s, bool has, bool neu, float lift, float sml_, float cf_) {
    const float bb = has ? 0.f : (neu ? 1.f : -1.f);
    a = make_float2(has ? 1.f : 0.f, has ? 1.f : 0.f);
    b = make_float2(bb, bb);
    c = a;
    d = make_float2(-bb, -bb);
    hs = make_float2(0.5f * s, 0.5f * s);
    sl = make_float2(s * lift, s * lift);
    sml = make_float2(sml_, sml_);
    cf = make_float2(cf_, cf_);
  }
  // two face points at once: returns the lifted gradient component, adds the flux to acc
  __device__ __forceinline__ float2 apply(float2 ui, float2 gi, float2 ue, float2 ge, float2& acc) const {
    const float2 uE = __ffma2_rn(a, ue, __fmul2_rn(b, ui));
    const float2 gE = __ffma2_rn(c, ge, __fmul2_rn(d, gi));
    const float2 jump = __fadd2_rn(uE, make_float2(-ui.x, -ui.y));
    const float2 dg = __fadd2_rn(gE, make_float2(-gi.x, -gi.y));
    acc = __ffma2_rn(cf, __ffma2_rn(hs, dg, __fmul2_rn(sml, jump)), acc);
    return __ffma2_rn(sl, jump, gi);
  }
};

template <int BX, int BY, int BZ>
__global__ void __launch_bounds__(BX* BY* BZ, E4Shape<BX, BY, BZ>::PER_SM)
    apply_elem4_kernel(const ApplyArgs<float> A, const __grid_constant__ CUtensorMap mu,
                       const __grid_constant__ CUtensorMap mo, int* __restrict__ err) {
  using S = E4Shape<BX, BY, BZ>;
  using C = CTab<float>;
  constexpr int SL = kE4Slot, PX = S::PX, PY = S::PY;
  constexpr int dO = dtab_off(4), wO = wtab_off(4);
  extern __shared__ __align__(128) unsigned char e4_raw[];
  // 128-byte aligned for TMA; offset from the shared array itself, so that the compiler keeps
  // every access in the shared window (LDS/STS rather than generic loads)
  float* sm = reinterpret_cast<float*>(e4_raw + ((128u - (e4_smem(e4_raw) & 127u)) & 127u));
  const uint32_t bar = e4_smem(sm + S::IN_WORDS);
  const OpGeom<float>& g = A.g;
  const int tid = threadIdx.x;
  const int tx = tid % BX, ty = (tid / BX) % BY, tz = tid / (BX * BY);
  const int nbx = (g.nx + BX - 1) / BX, nby = (g.ny + BY - 1) / BY;
  const int blk = blockIdx.x;
  const int x0 = (blk % nbx) * BX, y0 = ((blk / nbx) % nby) * BY, z0 = (blk / (nbx * nby)) * BZ;
  const int cx = x0 + tx, cy = y0 + ty, cz = z0 + tz;
  const bool hxm = cx > 0, hxp = cx + 1 < g.nx, hym = cy > 0, hyp = cy + 1 < g.ny, hzm = cz > 0, hzp = cz + 1 < g.nz;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  pdl_launch_dependents();
  pdl_wait();
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(S::IN_WORDS * 4)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(e4_smem(sm)),
        "l"(&mu), "r"(0), "r"(x0 - 1), "r"(y0 - 1), "r"(z0 - 1), "r"(bar)
        : "memory");
  }
  if (!__syncthreads_and(e4_wait(bar, err))) {
    if (tid == 0) e4_wait(bar, err);  // let the copy land (bounded) before the CTA leaves
    __syncthreads();
    return;
  }
  const float* me = sm + (((tz + 1) * PY + ty + 1) * PX + tx + 1) * SL;
  constexpr int DX = SL, DY = PX * SL, DZ = PY * PX * SL;  // neighbour offsets in words
  // element, gradient component and pre-mass sum as pairs of x-neighbouring points ([k][j][i / 2]):
  // the y- and z-contractions combine whole pairs with one packed FMA (Dhat entry in both halves)
  float2 U[4][4][2], ACC[4][4][2], G[4][4][2];
#define E4(a, k, j, i) ((i) & 1 ? a[k][j][(i) >> 1].y : a[k][j][(i) >> 1].x)
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float4 v = *reinterpret_cast<const float4*>(me + k * 16 + j * 4);
      U[k][j][0] = make_float2(v.x, v.y);
      U[k][j][1] = make_float2(v.z, v.w);
      ACC[k][j][0] = ACC[k][j][1] = make_float2(0.f, 0.f);
    }
  const float w0 = C::w(wO);
  const float cfx = g.Jf[0] / (g.J * w0), cfy = g.Jf[1] / (g.J * w0), cfz = g.Jf[2] / (g.J * w0);
  const float smx = g.sigma[0] - g.lift[0], smy = g.sigma[1] - g.lift[1], smz = g.sigma[2] - g.lift[2];
  const float2 dy2 = make_float2(g.dxi[1], g.dxi[1]), dz2 = make_float2(g.dxi[2], g.dxi[2]);
  // x: gradient component along the thread's lines, faces from the x-neighbours' lines, divergence.
  // Along a line the pairs multiply 2 x 2 blocks of Dhat: (y0, y1) = (D00, D11) (x0, x1) +
  // (D01, D10) (x1, x0) + (D02, D13) (x2, x3) + (D03, D12) (x3, x2), and likewise for (y2, y3).
  float2 Bx[8];
#pragma unroll
  for (int q = 0; q < 2; ++q)      // output pair
#pragma unroll
    for (int c = 0; c < 2; ++c) {  // input pair
      const int r0 = 2 * q, c0 = 2 * c;
      Bx[4 * q + 2 * c] = make_float2(C::D(dO + r0 * 4 + c0), C::D(dO + (r0 + 1) * 4 + c0 + 1));
      Bx[4 * q + 2 * c + 1] = make_float2(C::D(dO + r0 * 4 + c0 + 1), C::D(dO + (r0 + 1) * 4 + c0));
    }
  const float2 dx2 = make_float2(g.dxi[0], g.dxi[0]);
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 sw[2] = {make_float2(U[k][j][0].y, U[k][j][0].x), make_float2(U[k][j][1].y, U[k][j][1].x)};
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        float2 a = __fmul2_rn(Bx[4 * q], U[k][j][0]);
        a = __ffma2_rn(Bx[4 * q + 1], sw[0], a);
        a = __ffma2_rn(Bx[4 * q + 2], U[k][j][1], a);
        a = __ffma2_rn(Bx[4 * q + 3], sw[1], a);
        G[k][j][q] = __fmul2_rn(dx2, a);
      }
    }
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float r[4];
      ld4s(me - DX + k * 16 + j * 4, r);
      float ge = 0.f;
#pragma unroll
      for (int l = 0; l < 4; ++l) ge += C::D(dO + 12 + l) * r[l];
      G[k][j][0].x = e4_face(-1.f, U[k][j][0].x, G[k][j][0].x, r[3], g.dxi[0] * ge, hxm, g.neumann & 1, g.lift[0],
                             smx, cfx, ACC[k][j][0].x);
      ld4s(me + DX + k * 16 + j * 4, r);
      ge = 0.f;
#pragma unroll
      for (int l = 0; l < 4; ++l) ge += C::D(dO + l) * r[l];
      G[k][j][1].y = e4_face(1.f, U[k][j][1].y, G[k][j][1].y, r[0], g.dxi[0] * ge, hxp, (g.neumann >> 1) & 1,
                             g.lift[0], smx, cfx, ACC[k][j][1].y);
    }
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 sw[2] = {make_float2(G[k][j][0].y, G[k][j][0].x), make_float2(G[k][j][1].y, G[k][j][1].x)};
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        float2 a = __fmul2_rn(Bx[4 * q], G[k][j][0]);
        a = __ffma2_rn(Bx[4 * q + 1], sw[0], a);
        a = __ffma2_rn(Bx[4 * q + 2], G[k][j][1], a);
        a = __ffma2_rn(Bx[4 * q + 3], sw[1], a);
        ACC[k][j][q] = __ffma2_rn(dx2, a, ACC[k][j][q]);
      }
    }
  // y
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          const float d = C::D(dO + j * 4 + l);
          a = __ffma2_rn(make_float2(d, d), U[k][l][p], a);
        }
        G[k][j][p] = __fmul2_rn(dy2, a);
      }
  {
    const E4Face fm(-1.f, hym, (g.neumann >> 2) & 1, g.lift[1], smy, cfy), fp(1.f, hyp, (g.neumann >> 3) & 1,
                                                                            g.lift[1], smy, cfy);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float2 r[4][2];
#pragma unroll
      for (int l = 0; l < 4; ++l) ld4p(me - DY + k * 16 + l * 4, r[l]);
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        float2 ge = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          const float dd = C::D(dO + 12 + l);
          ge = __ffma2_rn(make_float2(dd, dd), r[l][p], ge);
        }
        G[k][0][p] = fm.apply(U[k][0][p], G[k][0][p], r[3][p], __fmul2_rn(dy2, ge), ACC[k][0][p]);
      }
#pragma unroll
      for (int l = 0; l < 4; ++l) ld4p(me + DY + k * 16 + l * 4, r[l]);
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        float2 ge = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          const float dd = C::D(dO + l);
          ge = __ffma2_rn(make_float2(dd, dd), r[l][p], ge);
        }
        G[k][3][p] = fp.apply(U[k][3][p], G[k][3][p], r[0][p], __fmul2_rn(dy2, ge), ACC[k][3][p]);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          const float d = C::D(dO + j * 4 + l);
          a = __ffma2_rn(make_float2(d, d), G[k][l][p], a);
        }
        ACC[k][j][p] = __ffma2_rn(dy2, a, ACC[k][j][p]);
      }
  // z
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          const float d = C::D(dO + k * 4 + l);
          a = __ffma2_rn(make_float2(d, d), U[l][j][p], a);
        }
        G[k][j][p] = __fmul2_rn(dz2, a);
      }
  {
    const E4Face fm(-1.f, hzm, (g.neumann >> 4) & 1, g.lift[2], smz, cfz), fp(1.f, hzp, (g.neumann >> 5) & 1,
                                                                            g.lift[2], smz, cfz);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float2 r[4][2];
#pragma unroll
      for (int l = 0; l < 4; ++l) ld4p(me - DZ + l * 16 + j * 4, r[l]);
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        float2 ge = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          const float dd = C::D(dO + 12 + l);
          ge = __ffma2_rn(make_float2(dd, dd), r[l][p], ge);
        }
        G[0][j][p] = fm.apply(U[0][j][p], G[0][j][p], r[3][p], __fmul2_rn(dz2, ge), ACC[0][j][p]);
      }
#pragma unroll
      for (int l = 0; l < 4; ++l) ld4p(me + DZ + l * 16 + j * 4, r[l]);
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        float2 ge = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          const float dd = C::D(dO + l);
          ge = __ffma2_rn(make_float2(dd, dd), r[l][p], ge);
        }
        G[3][j][p] = fp.apply(U[3][j][p], G[3][j][p], r[0][p], __fmul2_rn(dz2, ge), ACC[3][j][p]);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          const float d = C::D(dO + k * 4 + l);
          a = __ffma2_rn(make_float2(d, d), G[l][j][p], a);
        }
        ACC[k][j][p] = __ffma2_rn(dz2, a, ACC[k][j][p]);
      }
  // A u = -M acc (+ diag u); b - A u with b
  const bool valid = cx < g.nx && cy < g.ny && cz < g.nz;
  const int64_t e = valid ? ((int64_t)cz * g.ny + cy) * g.nx + cx : 0;
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float dl[4], bl[4];
      if (A.diag && valid) row4_g(A.diag + e * 64 + k * 16 + j * 4, dl);
      if (A.b && valid) row4_g(A.b + e * 64 + k * 16 + j * 4, bl);
      const float mjk = -g.J * C::w(wO + j) * C::w(wO + k);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float res = mjk * C::w(wO + i) * E4(ACC, k, j, i);
        if (A.diag && valid) res += dl[i] * E4(U, k, j, i);
        E4(ACC, k, j, i) = (A.b && valid) ? bl[i] - res : res;
      }
    }
#undef E4
  __syncthreads();  // every read of the staged box is done: its first slots take the result
  float* o = sm + tid * SL;
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j)
      *reinterpret_cast<float4*>(o + k * 16 + j * 4) =
          make_float4(ACC[k][j][0].x, ACC[k][j][0].y, ACC[k][j][1].x, ACC[k][j][1].y);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (tid == 0) {
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(&mo),
                 "r"(0), "r"(x0), "r"(y0), "r"(z0), "r"(e4_smem(sm))
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  }
}

// ------------------------------------------------------------------ block-of-lines apply (FP32)
//
// Shared memory serves one word per lane and cycle, so a contraction whose inputs come from other
// threads is bound by the LSU pipe unless every word a thread loads feeds several of its own
// outputs. Here a thread owns B consecutive x-lines: in the first phase B lines along y in one z
// plane k (x-contractions in registers, each y-neighbour row loaded once for B outputs), in the
// second phase B lines along z in one y row j (each z-neighbour row loaded once for B outputs).
// The element, v_y then v_z, and the first phase's partial result pass through shared memory. The
// threads of one block index form warp-uniform groups, so the Dhat rows a thread uses are
// compile-time constants (constant-memory operands). With B = N (one block) a thread holds a whole
// plane and that phase's contraction stays in registers. Neighbour data for the face terms is read
// by the threads that own the face: the x-neighbours' lines of every own line, the y- (z-)
// neighbour's plane (row) of a face the block touches, streamed row by row.
template <int N, int B, int EPB>
struct BlkShape {
  static constexpr int NB = (N + B - 1) / B;  // blocks along the blocked direction
  static constexpr int VW = LineVec<N, float>::per;
  // strides in words: an odd number of vectors, so that the lanes of one vector phase (consecutive
  // planes in the first phase, consecutive rows in the second) hit distinct banks
  static constexpr int LS = ((N / VW) % 2 == 1) ? N : N + VW;
  static constexpr int PS = (((N * LS) / VW) % 2 == 1) ? N * LS : N * LS + VW;
  static constexpr int ES = N * PS;
  static constexpr int GP = (EPB * N + 31) / 32 * 32;  // threads per group, whole warps
  static constexpr int THREADS = NB * GP;
  static constexpr int SMEM = 3 * EPB * ES * (int)sizeof(float);
};

struct BlkElem {
  int64_t base;  // element offset in the vectors (ec N^3)
  int nb[6];     // neighbour element across each face (ec itself where there is none)
  bool has[6];
};

__device__ __forceinline__ BlkElem blk_elem(const OpGeom<float>& g, int ec, int n3) {
  BlkElem c;
  const int nx = g.nx, ny = g.ny, nxy = g.nx * g.ny;
  const int cx = ec % nx, cy = (ec / nx) % ny, cz = ec / nxy;
  c.has[0] = cx > 0;
  c.has[1] = cx + 1 < nx;
  c.has[2] = cy > 0;
  c.has[3] = cy + 1 < ny;
  c.has[4] = cz > 0;
  c.has[5] = cz + 1 < g.nz;
  const int step[3] = {1, nx, nxy};
#pragma unroll
  for (int f = 0; f < 6; ++f) c.nb[f] = c.has[f] ? ec + ((f & 1) ? step[f >> 1] : -step[f >> 1]) : ec;
  c.base = (int64_t)ec * n3;
  return c;
}

// First phase for the group of block jb (warp-uniform): lines j = jb B + jj of plane k. Leaves A u's
// x and y terms (volume and face) of the own lines in the partial-result buffer (the x part goes
// there first, so that it does not hold registers through the y contractions). The Dhat rows of
// the block are read from constant memory with a warp-uniform index.
template <int N, int B, int EPB>
__device__ __forceinline__ void blk_phase_y(const ApplyArgs<float>& A, const BlkElem& c, int jb, int k, bool act,
                                            int el, float* us, float* vs, float* ps) {
  using S = BlkShape<N, B, EPB>;
  using C = CTab<float>;
  constexpr int N2 = N * N, dO = dtab_off(N), wO = wtab_off(N);
  constexpr int NJ = B;  // lines past N (a ragged last block) are computed on zeros and never stored
  constexpr bool ragged = S::NB * B != N;
  const int J0 = jb * B;
  auto ok = [&](int jj) { return !ragged || J0 + jj < N; };
  const OpGeom<float>& g = A.g;
  const float* __restrict__ u = A.u;
  const float wk = C::w(wO + k);  // k is a runtime index: one constant-cache read per thread
  // the CTA's elements (a contiguous run) into their padded shared blocks, with coalesced loads by
  // all threads (a thread's own lines are 128-byte runs one plane apart, so loading them per
  // thread would touch a separate line per lane); past the last element, element E - 1 again
  {
    constexpr int N3 = N2 * N, VE = LineVec<N, float>::per;  // values per vector move
    using V = typename LineVec<N, float>::V;
    const int e0 = blockIdx.x * EPB;
    float* us0 = us - el * S::ES;  // the first element's block
    for (int idx = threadIdx.x; idx < EPB * N3 / VE; idx += S::THREADS) {
      const int el2 = idx / (N3 / VE), o = (idx - el2 * (N3 / VE)) * VE;
      const int e2 = min(e0 + el2, A.E - 1);
      const V v = *reinterpret_cast<const V*>(u + (int64_t)e2 * N3 + o);
      *reinterpret_cast<V*>(us0 + el2 * S::ES + (o / N2) * S::PS + ((o / N) % N) * S::LS + o % N) = v;
    }
  }
  __syncthreads();  // every element is staged
  float U[NJ][N];
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj) {
    if (ok(jj)) {
      sld_line<N>(us + k * S::PS + (J0 + jj) * S::LS, U[jj]);
    } else {
#pragma unroll
      for (int i = 0; i < N; ++i) U[jj][i] = 0.f;
    }
  }
  // x: neighbour traces, gradient, lifting, face fluxes and divergence in registers, line by line;
  // the result goes to the partial-result buffer. An x-neighbour inside the CTA's run is read from
  // its staged block (where it is not the element's neighbour, the face uses the ghost state).
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj) {
    if (!ok(jj)) continue;
    float t[N];
    if (el > 0) sld_line<N>(us - S::ES + k * S::PS + (J0 + jj) * S::LS, t);
    else gld_line<N>(u + (int64_t)c.nb[0] * N2 * N + k * N2 + (J0 + jj) * N, t);
    const float uxm = t[N - 1];
    float gxm = 0.f;
#pragma unroll
    for (int l = 0; l < N; ++l) gxm += C::D(dO + (N - 1) * N + l) * t[l];
    if (el + 1 < EPB) sld_line<N>(us + S::ES + k * S::PS + (J0 + jj) * S::LS, t);
    else gld_line<N>(u + (int64_t)c.nb[1] * N2 * N + k * N2 + (J0 + jj) * N, t);
    const float uxp = t[0];
    float gxp = 0.f;
#pragma unroll
    for (int l = 0; l < N; ++l) gxp += C::D(dO + l) * t[l];
    float vx[N], o[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      float a = 0.f;
#pragma unroll
      for (int l = 0; l < N; ++l) a += C::D(dO + i * N + l) * U[jj][l];
      vx[i] = g.dxi[0] * a;
      o[i] = 0.f;
    }
    const float wj = C::w(wO + J0 + jj);
    const float Bf = g.Jf[0] * wj * wk, sml = g.sigma[0] - g.lift[0];
    vx[0] = face_point(-1.f, U[jj][0], vx[0], uxm, g.dxi[0] * gxm, c.has[0], g.neumann & 1, g.lift[0], sml, Bf, o[0]);
    vx[N - 1] = face_point(1.f, U[jj][N - 1], vx[N - 1], uxp, g.dxi[0] * gxp, c.has[1], (g.neumann >> 1) & 1,
                           g.lift[0], sml, Bf, o[N - 1]);
    const float M0 = g.J * wj * wk;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      float a = 0.f;
#pragma unroll
      for (int l = 0; l < N; ++l) a += C::D(dO + i * N + l) * vx[l];
      o[i] -= (M0 * C::w(wO + i)) * g.dxi[0] * a;
    }
    if (act) sst_line<N>(ps + k * S::PS + (J0 + jj) * S::LS, o);
  }
  __syncthreads();  // the element is in shared memory
  // y gradient: each row of the plane (own rows from registers) feeds the NJ own outputs
  float vy[NJ][N];
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj)
#pragma unroll
    for (int i = 0; i < N; ++i) vy[jj][i] = 0.f;
#pragma unroll
  for (int l = 0; l < N; ++l) {
    float t[N];
    if constexpr (S::NB == 1) {  // one block: the thread holds the whole plane
#pragma unroll
      for (int i = 0; i < N; ++i) t[i] = U[l < NJ ? l : 0][i];
    } else {
      sld_line<N>(us + k * S::PS + l * S::LS, t);
    }
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj) {
      const float d = ok(jj) ? C::D(dO + (J0 + jj) * N + l) : 0.f;
      axpy_line<N>(d, t, vy[jj]);
    }
  }
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj)
#pragma unroll
    for (int i = 0; i < N; ++i) vy[jj][i] *= g.dxi[1];
  // y faces this block touches: neighbour traces (rows of the neighbour's plane k), lifting into
  // v_y, face fluxes into fy
  float fy[2][N];
#pragma unroll
  for (int i = 0; i < N; ++i) fy[0][i] = fy[1][i] = 0.f;
  {
    const float sml = g.sigma[1] - g.lift[1];
    if (J0 == 0) {
      float uym[N], gym[N];
#pragma unroll
      for (int i = 0; i < N; ++i) gym[i] = 0.f;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        float t[N];
        gld_line<N>(u + (int64_t)c.nb[2] * N2 * N + k * N2 + l * N, t);
#pragma unroll
        for (int i = 0; i < N; ++i) {
          gym[i] += C::D(dO + (N - 1) * N + l) * t[i];
          if (l == N - 1) uym[i] = t[i];
        }
      }
#pragma unroll
      for (int i = 0; i < N; ++i)
        vy[0][i] = face_point(-1.f, U[0][i], vy[0][i], uym[i], g.dxi[1] * gym[i], c.has[2], (g.neumann >> 2) & 1,
                              g.lift[1], sml, g.Jf[1] * C::w(wO + i) * wk, fy[0][i]);
    }
    if (J0 + NJ >= N) {  // the block holding the row j = N - 1 (at jj = N - 1 - J0)
      float uyp[N], gyp[N];
#pragma unroll
      for (int i = 0; i < N; ++i) gyp[i] = 0.f;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        float t[N];
        gld_line<N>(u + (int64_t)c.nb[3] * N2 * N + k * N2 + l * N, t);
#pragma unroll
        for (int i = 0; i < N; ++i) {
          gyp[i] += C::D(dO + l) * t[i];
          if (l == 0) uyp[i] = t[i];
        }
      }
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj) {
        if (J0 + jj != N - 1) continue;
#pragma unroll
        for (int i = 0; i < N; ++i)
          vy[jj][i] = face_point(1.f, U[jj][i], vy[jj][i], uyp[i], g.dxi[1] * gyp[i], c.has[3], (g.neumann >> 3) & 1,
                                 g.lift[1], sml, g.Jf[1] * C::w(wO + i) * wk, fy[1][i]);
      }
    }
  }
  // y divergence (other blocks' v_y through shared memory)
  if constexpr (S::NB > 1) {
    if (act) {
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj)
        if (ok(jj)) sst_line<N>(vs + k * S::PS + (J0 + jj) * S::LS, vy[jj]);
    }
    __syncthreads();
  }
  float dy[NJ][N];
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj)
#pragma unroll
    for (int i = 0; i < N; ++i) dy[jj][i] = 0.f;
#pragma unroll
  for (int l = 0; l < N; ++l) {
    float t[N];
    if constexpr (S::NB == 1) {
#pragma unroll
      for (int i = 0; i < N; ++i) t[i] = vy[l < NJ ? l : 0][i];
    } else {
      sld_line<N>(vs + k * S::PS + l * S::LS, t);
    }
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj) {
      const float d = ok(jj) ? C::D(dO + (J0 + jj) * N + l) : 0.f;
      axpy_line<N>(d, t, dy[jj]);
    }
  }
  if (act) {
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj) {
      if (!ok(jj)) continue;
      const float M0 = g.J * C::w(wO + J0 + jj) * wk;
      float r[N];
      sld_line<N>(ps + k * S::PS + (J0 + jj) * S::LS, r);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        r[i] -= (M0 * C::w(wO + i)) * g.dxi[1] * dy[jj][i];
        if (J0 + jj == 0) r[i] += fy[0][i];
        if (J0 + jj == N - 1) r[i] += fy[1][i];
      }
      sst_line<N>(ps + k * S::PS + (J0 + jj) * S::LS, r);
    }
  }
}

// Second phase for the group of block kb (warp-uniform): lines (j, k = kb B + kk). Adds the z terms
// to the partial result and writes A u (b - A u, + diag u) for the own lines.
template <int N, int B, int EPB>
__device__ __forceinline__ void blk_phase_z(const ApplyArgs<float>& A, const BlkElem& c, int kb, int j, bool act,
                                            bool store, const float* us, float* vs, const float* ps,
                                            const int* s_col, const int* s_map) {
  using S = BlkShape<N, B, EPB>;
  using C = CTab<float>;
  constexpr int N2 = N * N, dO = dtab_off(N), wO = wtab_off(N);
  constexpr int NK = B;
  constexpr bool ragged = S::NB * B != N;
  const int K0 = kb * B;
  auto ok = [&](int kk) { return !ragged || K0 + kk < N; };
  const OpGeom<float>& g = A.g;
  const float* __restrict__ u = A.u;
  const float wj = C::w(wO + j);
  // z gradient: each row u(., j, l) of the element feeds the NK own outputs
  float vz[NK][N];
#pragma unroll
  for (int kk = 0; kk < NK; ++kk)
#pragma unroll
    for (int i = 0; i < N; ++i) vz[kk][i] = 0.f;
#pragma unroll
  for (int l = 0; l < N; ++l) {
    float t[N];
    sld_line<N>(us + l * S::PS + j * S::LS, t);
#pragma unroll
    for (int kk = 0; kk < NK; ++kk) {
      const float d = ok(kk) ? C::D(dO + (K0 + kk) * N + l) : 0.f;
      axpy_line<N>(d, t, vz[kk]);
    }
  }
#pragma unroll
  for (int kk = 0; kk < NK; ++kk)
#pragma unroll
    for (int i = 0; i < N; ++i) vz[kk][i] *= g.dxi[2];
  // z faces this block touches: lifting into v_z, face fluxes into fz
  float fz[2][N];
#pragma unroll
  for (int i = 0; i < N; ++i) fz[0][i] = fz[1][i] = 0.f;
  {
    const float sml = g.sigma[2] - g.lift[2];
    if (K0 == 0) {
      float uzm[N], gzm[N], ui[N];
#pragma unroll
      for (int i = 0; i < N; ++i) gzm[i] = 0.f;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        float t[N];
        gld_line<N>(u + (int64_t)c.nb[4] * N2 * N + l * N2 + j * N, t);
#pragma unroll
        for (int i = 0; i < N; ++i) {
          gzm[i] += C::D(dO + (N - 1) * N + l) * t[i];
          if (l == N - 1) uzm[i] = t[i];
        }
      }
      sld_line<N>(us + j * S::LS, ui);
#pragma unroll
      for (int i = 0; i < N; ++i)
        vz[0][i] = face_point(-1.f, ui[i], vz[0][i], uzm[i], g.dxi[2] * gzm[i], c.has[4], (g.neumann >> 4) & 1,
                              g.lift[2], sml, g.Jf[2] * C::w(wO + i) * wj, fz[0][i]);
    }
    if (K0 + NK >= N) {  // the block holding the plane k = N - 1 (at kk = N - 1 - K0)
      float uzp[N], gzp[N], ui[N];
#pragma unroll
      for (int i = 0; i < N; ++i) gzp[i] = 0.f;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        float t[N];
        gld_line<N>(u + (int64_t)c.nb[5] * N2 * N + l * N2 + j * N, t);
#pragma unroll
        for (int i = 0; i < N; ++i) {
          gzp[i] += C::D(dO + l) * t[i];
          if (l == 0) uzp[i] = t[i];
        }
      }
      sld_line<N>(us + (N - 1) * S::PS + j * S::LS, ui);
#pragma unroll
      for (int kk = 0; kk < NK; ++kk) {
        if (K0 + kk != N - 1) continue;
#pragma unroll
        for (int i = 0; i < N; ++i)
          vz[kk][i] = face_point(1.f, ui[i], vz[kk][i], uzp[i], g.dxi[2] * gzp[i], c.has[5], (g.neumann >> 5) & 1,
                                 g.lift[2], sml, g.Jf[2] * C::w(wO + i) * wj, fz[1][i]);
      }
    }
  }
  // z divergence (other blocks' v_z through shared memory; the first-phase reads of v_y ended
  // before the barrier between the phases)
  if constexpr (S::NB > 1) {
    if (act) {
#pragma unroll
      for (int kk = 0; kk < NK; ++kk)
        if (ok(kk)) sst_line<N>(vs + (K0 + kk) * S::PS + j * S::LS, vz[kk]);
    }
    __syncthreads();
  }
  float dz[NK][N];
#pragma unroll
  for (int kk = 0; kk < NK; ++kk)
#pragma unroll
    for (int i = 0; i < N; ++i) dz[kk][i] = 0.f;
#pragma unroll
  for (int l = 0; l < N; ++l) {
    float t[N];
    if constexpr (S::NB == 1) {  // one block: the thread holds the whole row of planes
#pragma unroll
      for (int i = 0; i < N; ++i) t[i] = vz[l < NK ? l : 0][i];
    } else {
      sld_line<N>(vs + l * S::PS + j * S::LS, t);
    }
#pragma unroll
    for (int kk = 0; kk < NK; ++kk) {
      const float d = ok(kk) ? C::D(dO + (K0 + kk) * N + l) : 0.f;
      axpy_line<N>(d, t, dz[kk]);
    }
  }
  if (!store) return;
#pragma unroll
  for (int kk = 0; kk < NK; ++kk) {
    if (!ok(kk)) continue;
    const int k = K0 + kk;
    const int64_t off = c.base + k * N2 + j * N;
    const float M0 = g.J * wj * C::w(wO + k);
    float pr[N], dl[N], bl[N], ul[N], val[N];
    sld_line<N>(ps + k * S::PS + j * S::LS, pr);
    if (A.diag) {
      gld_line<N>(A.diag + off, dl);
      sld_line<N>(us + k * S::PS + j * S::LS, ul);
    }
    if (A.b) gld_line<N>(A.b + off, bl);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      float r = pr[i] - (M0 * C::w(wO + i)) * g.dxi[2] * dz[kk][i];
      if (k == 0) r += fz[0][i];
      if (k == N - 1) r += fz[1][i];
      if (A.diag) r += dl[i] * ul[i];
      val[i] = A.b ? bl[i] - r : r;
    }
    if (!A.rS) {
      gst_line<N>(A.out + off, val);
      continue;
    }
    // written straight into the subdomain vectors: the element's own subdomain (slot 0) and, for
    // points in a face neighbour's overlap layers, that neighbour's subdomain (slot 1 + (f ^ 1)); every
    // subdomain row holds one point, so these stores never collide
    const int t = k * N + j;
#pragma unroll
    for (int sl = 0; sl < 7; ++sl) {
      const int col = s_col[sl];
      if (col < 0) continue;
      int lo = 0, hi = N;
      if (sl > 0) {
        const int f = sl - 1, dd = f >> 1, side = f & 1;
        if (dd == 0) {
          if (side) lo = N - A.ov;
          else hi = A.ov;
        } else {
          const int cc = dd == 1 ? j : k;
          if ((side ? N - 1 - cc : cc) >= A.ov) continue;
        }
      }
      int rows[N];
      gld_line<N>(A.inv + s_map[sl] + t * N, rows);
      if (!DG_IN_BOUNDS(col, A.E)) continue;
      float* colp = A.rS + (int64_t)col * A.ld;
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (i >= lo && i < hi && rows[i] >= 0 && DG_IN_BOUNDS(rows[i], A.ld)) colp[rows[i]] = val[i];
    }
  }
}

template <int N, int B, int EPB>
__global__ void __launch_bounds__(BlkShape<N, B, EPB>::THREADS) apply_blk_kernel(const ApplyArgs<float> A) {
  using S = BlkShape<N, B, EPB>;
  constexpr int N3 = N * N * N;
  extern __shared__ __align__(16) float blk_smem[];
  pdl_launch_dependents();
  pdl_wait();
  const int tid = threadIdx.x;
  const int grp = tid / S::GP, r = tid - grp * S::GP;
  const bool act = r < EPB * N;  // lanes past the last element of the group only take part in barriers
  const int el = act ? r / N : 0, q = act ? r - (r / N) * N : 0;
  const int e = blockIdx.x * EPB + el;
  const int ec = e < A.E ? e : A.E - 1;  // past the end: compute on a real element, store nothing
  const BlkElem c = blk_elem(A.g, ec, N3);
  float* us = blk_smem + el * S::ES;
  float* vs = blk_smem + (EPB + el) * S::ES;
  float* ps = blk_smem + (2 * EPB + el) * S::ES;
  // residual written into the subdomain vectors: column and point-map offset of each element's own
  // subdomain (slot 0) and of each face neighbour's subdomain (slot 1 + (f ^ 1))
  __shared__ int s_col[EPB][7], s_map[EPB][7];
  if (A.rS) {
    const int nx = A.g.nx, ny = A.g.ny, nxy = A.g.nx * A.g.ny;
    for (int qq = tid; qq < EPB * 7; qq += S::THREADS) {
      const int el2 = qq / 7, sl = qq - el2 * 7;
      const int e2 = blockIdx.x * EPB + el2;
      int col = -1, m = 0;
      if (e2 < A.E) {
        int rr = e2;
        if (sl > 0) {
          const int f = sl - 1, d = f >> 1;
          int c3[3] = {e2 % nx, (e2 / nx) % ny, e2 / nxy};
          const int nd = d == 0 ? nx : (d == 1 ? ny : A.g.nz);
          c3[d] += (f & 1) ? 1 : -1;
          rr = (c3[d] >= 0 && c3[d] < nd) ? c3[0] + nx * (c3[1] + ny * c3[2]) : -1;
        }
        if (rr >= 0) {
          col = A.col_of_elem[rr];
          m = (A.orient[rr] * 7 + (sl == 0 ? 0 : 1 + ((sl - 1) ^ 1))) * N3;
        }
      }
      s_col[el2][sl] = col;
      s_map[el2][sl] = m;
    }
  }
  blk_phase_y<N, B, EPB>(A, c, grp, q, act, el, us, vs, ps);
  __syncthreads();  // the partial results (and the subdomain tables) are in shared memory
  const bool store = act && e < A.E;
  blk_phase_z<N, B, EPB>(A, c, grp, q, act, store, us, vs, ps, s_col[el], s_map[el]);
}

// Launch shapes of the block kernel per N: (B, EPB) for variants 5 and 6.
template <int N>
struct BlkConfig;
template <> struct BlkConfig<4> { static constexpr int B5 = 4, E5 = 16, B6 = 4, E6 = 8; };
template <> struct BlkConfig<5> { static constexpr int B5 = 5, E5 = 12, B6 = 5, E6 = 6; };
template <> struct BlkConfig<6> { static constexpr int B5 = 6, E5 = 10, B6 = 3, E6 = 5; };
template <> struct BlkConfig<7> { static constexpr int B5 = 7, E5 = 8, B6 = 4, E6 = 4; };
template <> struct BlkConfig<8> { static constexpr int B5 = 4, E5 = 4, B6 = 2, E6 = 4; };
template <> struct BlkConfig<9> { static constexpr int B5 = 5, E5 = 3, B6 = 3, E6 = 3; };
template <> struct BlkConfig<10> { static constexpr int B5 = 5, E5 = 3, B6 = 4, E6 = 3; };

template <int N, int B, int EPB>
void launch_blk(const ApplyArgs<float>& A, cudaStream_t s) {
  using S = BlkShape<N, B, EPB>;
  if constexpr (S::SMEM > 48 * 1024) {
    static std::mutex mu;
    static std::set<int> done;
    int dev = 0;
    DG_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (!done.count(dev)) {
      DG_CUDA(cudaFuncSetAttribute(apply_blk_kernel<N, B, EPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM));
      done.insert(dev);
    }
  }
  launch_pdl(apply_blk_kernel<N, B, EPB>, dim3((A.E + EPB - 1) / EPB), dim3(S::THREADS), (size_t)S::SMEM, s, A);
}

// Tensor maps of the element-per-thread apply: u (or the result) as a 4-D tensor [nz][ny][nx][64]
// read or written in boxes of (BX, BY, BZ) elements of 68 words (the 4 words past an element are
// outside the tensor: zeros on loads, not written on stores). No swizzle.
PFN_cuTensorMapEncodeTiled_v12000 e4_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      (void)cudaGetLastError();
  });
  return fn;
}

bool e4_map(CUtensorMap* m, const float* base, int nx, int ny, int nz, int bx, int by, int bz) {
  auto fn = e4_encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[4] = {64, (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[3] = {256, 256ull * nx, 256ull * nx * ny};
  const cuuint32_t box[4] = {(cuuint32_t)kE4Slot, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void*)base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// False (nothing launched) where the element-per-thread kernel cannot run this apply: subdomain
// output, buffers not 16-byte aligned, no error flag, or a tensor map the driver does not encode.
template <int BX, int BY, int BZ>
bool launch_elem4(const ApplyArgs<float>& A, int* err, cudaStream_t s) {
  using S = E4Shape<BX, BY, BZ>;
  auto kern = apply_elem4_kernel<BX, BY, BZ>;
  const OpGeom<float>& g = A.g;
  if (A.rS || !err || (((uintptr_t)A.u | (uintptr_t)A.out) & 15)) return false;
  CUtensorMap mu, mo;
  if (!e4_map(&mu, A.u, g.nx, g.ny, g.nz, BX + 2, BY + 2, BZ + 2) || !e4_map(&mo, A.out, g.nx, g.ny, g.nz, BX, BY, BZ))
    return false;
  {
    static std::mutex mu_attr;
    static std::set<int> done;
    int dev = 0;
    DG_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu_attr);
    if (!done.count(dev)) {
      DG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM));
      done.insert(dev);
    }
  }
  const int nb = ((g.nx + BX - 1) / BX) * ((g.ny + BY - 1) / BY) * ((g.nz + BZ - 1) / BZ);
  launch_pdl(kern, dim3(nb), dim3(S::THREADS), (size_t)S::SMEM, s, A, mu, mo, err);
  return true;
}

template <int N, typename T, int EPB>
void launch_apply_epb(const OpGeom<T>& g, const T* D, const T* w, const T* u, const T* diag, const T* b, T* out,
                      const SubdomainOut& so, int E, cudaStream_t s) {
  const ApplyArgs<T> A{g, D, w, u, diag, b, out, E, static_cast<T*>(so.rS), so.ld, so.ov, so.col_of_elem, so.orient,
                       so.inv};
  launch_pdl(apply_line_kernel<N, T, EPB>, dim3((E + EPB - 1) / EPB), dim3(EPB * N * N), 0, s, A);
}

// Launch shapes: elements per CTA from the shared-memory/thread budget (S::epb), the fewest that
// fill a warp (kSmall) and one in between. Variant 0 picks by grid size; 1..3 force one of them
// (the autotuner times them per level).
template <int N, typename T>
void launch_apply_n(const OpGeom<T>& g, const T* D, const T* w, const T* u, const T* diag, const T* b, T* out,
                    const SubdomainOut& so, int variant, int* err, cudaStream_t s) {
  const int E = g.nx * g.ny * g.nz;
  if (E == 0) return;
  constexpr unsigned a = LineVec<N, T>::w - 1;  // lines move in vectors of this many bytes
  DG_REQUIRE(!(((uintptr_t)u | (uintptr_t)diag | (uintptr_t)b | (uintptr_t)out | (uintptr_t)so.rS) & a),
             "DG apply vectors must be aligned to " + std::to_string(a + 1) + " bytes");
  using S = LineShape<N, T>;
  constexpr int kSmall = N * N >= 32 ? 1 : (32 + N * N - 1) / (N * N);  // at least one warp per CTA
  constexpr int kBig = S::epb > kSmall ? S::epb : kSmall;
  constexpr int kMid = (kSmall + kBig) / 2;
  if constexpr (N == 4 && std::is_same<T, float>::value) {
    if (variant == 4 && !so.rS) {
      const ApplyArgs<float> A{g, D, w, u, diag, b, out, E, nullptr, 0, 0, nullptr, nullptr, nullptr};
      launch_pdl(apply_slice4_kernel, dim3((E + kSliceEPB - 1) / kSliceEPB), dim3(kSliceEPB * 4), 0, s, A);
      return;
    }
    if (variant == 7) {
      const ApplyArgs<float> A{g, D, w, u, diag, b, out, E, nullptr, 0, 0, nullptr, nullptr, nullptr};
      if (!so.rS && launch_elem4<8, 4, 4>(A, err, s)) return;
      variant = 0;
    }
  }
  if constexpr (N >= 4 && std::is_same<T, float>::value) {
    if (variant == 5 || variant == 6) {
      const ApplyArgs<float> A{g, D, w, u, diag, b, out, E, static_cast<float*>(so.rS), so.ld, so.ov,
                               so.col_of_elem, so.orient, so.inv};
      using BC = BlkConfig<N>;
      if (variant == 5) launch_blk<N, BC::B5, BC::E5>(A, s);
      else launch_blk<N, BC::B6, BC::E6>(A, s);
      return;
    }
  }
  if (variant >= 4) variant = 0;  // the slice and element kernels cover plain FP32 applies, the block kernel FP32
  if (variant == 0) variant = ((E + kBig - 1) / kBig >= 2 * 152) ? 3 : 1;
  if (variant == 1) launch_apply_epb<N, T, kSmall>(g, D, w, u, diag, b, out, so, E, s);
  else if (variant == 2) launch_apply_epb<N, T, kMid>(g, D, w, u, diag, b, out, so, E, s);
  else launch_apply_epb<N, T, kBig>(g, D, w, u, diag, b, out, so, E, s);
}

// ------------------------------------------------------------------ fused coarse-level smoother
//
// On coarse levels (tens of elements) each of the three kernels of a Schwarz step is limited by its
// own latency, not by work. This kernel runs all steps of one smoothing call in a single
// cooperative launch: residual into r_S (or the gather of b when u = 0), the subdomain solves as a
// CUDA-core GEMM over (class, 16-row) units, the weighted scatter into u, each phase separated by a
// grid-wide barrier. Data written by other CTAs inside the kernel are read through L2 only.

constexpr uint32_t kBarrierPolls = 1u << 22;  // polls before a barrier wait gives up

// Grid-wide barrier over a cooperative launch (all CTAs co-resident). Returns false, with the error
// flag set, if the wait gave up; the caller then leaves the kernel.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned n_blocks, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == n_blocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      uint32_t polls = 0;
      while (*gen == g) {
        if (++polls > kBarrierPolls) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Rows row0 .. row0 + 15 of du_S for every column of one class: 128 threads = 16 rows x 8 K-groups
// of 16; the class's columns are staged in shared memory 8 at a time in 128-wide K tiles; the 8
// partial sums of each output are added in a fixed order.
__device__ __forceinline__ void coarse_gemm_unit(const float* __restrict__ invm, int ld, const float* X, float* Y,
                                                 int4 unit, float alpha) {
  __shared__ __align__(16) float sx[8][136];  // 128 K values per column, one pad word per 16
  __shared__ float red[8][16][9];
  const int tid = threadIdx.x;
  const int kg = tid & 7, r = tid >> 3;  // r < 16 for the first 128 threads
  const int cls = unit.x, row0 = unit.y, col0 = unit.z, ncols = unit.w;
  const float* arow = invm + ((size_t)cls * ld + row0 + r) * ld;
  for (int c0 = 0; c0 < ncols; c0 += 8) {
    const int nc = min(8, ncols - c0);
    float acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = 0.0f;
    for (int kt = 0; kt < ld; kt += 128) {
      __syncthreads();  // sx and red of the previous round are consumed
      for (int q = tid; q < 8 * 128; q += blockDim.x) {
        const int c = q >> 7, kk = q & 127;
        sx[c][kk + (kk >> 4)] = (c < nc && kt + kk < ld) ? __ldcg(X + (size_t)(col0 + c0 + c) * ld + kt + kk) : 0.0f;
      }
      __syncthreads();
      const int kb = kt + kg * 16;
      if (tid < 128 && kb < ld) {
        float a[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 v = __ldg(reinterpret_cast<const float4*>(arow + kb) + q);
          a[4 * q] = v.x;
          a[4 * q + 1] = v.y;
          a[4 * q + 2] = v.z;
          a[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i)
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[c] += a[i] * sx[c][kg * 17 + i];
      }
    }
    if (tid < 128) {
#pragma unroll
      for (int c = 0; c < 8; ++c) red[kg][r][c] = acc[c];
    }
    __syncthreads();
    if (tid < 128) {
      const int rr = tid >> 3, cc = tid & 7;
      if (cc < nc) {
        float sum = 0.0f;
#pragma unroll
        for (int g = 0; g < 8; ++g) sum += red[g][rr][cc];
        Y[(size_t)(col0 + c0 + cc) * ld + row0 + rr] = alpha * sum;
      }
    }
  }
}

template <int N, int EPB>
__global__ void __launch_bounds__(EPB* N* N) coarse_smooth_kernel(const CoarseArgs a) {
  // a wait of an earlier launch gave up and the host has not read the flag yet: skip the work
  // (its inputs are incomplete) instead of waiting again
  if (*reinterpret_cast<volatile int*>(a.err) != 0) return;
  const unsigned G = gridDim.x + (unsigned)a.stall;
  const int E = a.ap.E;
  const int nblk = (E + EPB - 1) / EPB;
  for (int it = 0; it < a.iterations; ++it) {
    if (it == 0 && a.u_zero) {
      for (int col = blockIdx.x; col < E; col += gridDim.x)
        gather_column<float, false>(a.sg, a.ap.b, a.elem_of_col, a.ap.orient, a.map, a.ap.rS, col);
    } else {
      for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        __syncthreads();  // the previous group is done with the shared blocks
        apply_line_block<N, float, EPB, false, true>(a.ap, blk);
      }
    }
    if (!grid_barrier(a.bar, G, a.err)) return;
    for (int un = blockIdx.x; un < a.n_units; un += gridDim.x)
      coarse_gemm_unit(a.invm, a.sg.ld, a.ap.rS, a.duS, a.units[un], a.alpha);
    if (!grid_barrier(a.bar, G, a.err)) return;
    for (int e = blockIdx.x; e < E; e += gridDim.x)
      scatter_element<float, float, false, true>(a.sg, a.duS, a.ap.col_of_elem, a.ap.orient, a.ap.inv, a.shares,
                                                 const_cast<float*>(a.ap.u), e);
    if (it + 1 < a.iterations && !grid_barrier(a.bar, G, a.err)) return;
  }
}

// threads per CTA: whole elements, at least the 128 the GEMM units use
template <int N>
struct CoarseShape {
  static constexpr int epb = (128 + N * N - 1) / (N * N);
  static constexpr int threads = epb * N * N;
};

template <int N>
void launch_coarse_n(const CoarseArgs& a, cudaStream_t s) {
  using CS = CoarseShape<N>;
  static_assert(CS::threads >= 128, "GEMM units need 128 threads");
  int dev = 0, sms = 0, per_sm = 0;
  DG_CUDA(cudaGetDevice(&dev));
  DG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  DG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coarse_smooth_kernel<N, CS::epb>, CS::threads, 0));
  DG_REQUIRE(per_sm >= 1, "fused coarse smoother does not fit on an SM");
  const int E = a.ap.E;
  const int work = std::max(std::max((E + CS::epb - 1) / CS::epb, E), a.n_units);
  const int G = std::min(work, per_sm * sms);
  DG_CUDA(cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), s));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(CS::threads);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  DG_CUDA(cudaLaunchKernelEx(&cfg, coarse_smooth_kernel<N, CS::epb>, a));
}

}  // namespace

void upload_operator_tables() {
  static std::mutex mu;
  static std::set<int> done;
  int dev = 0;
  DG_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (done.count(dev)) return;
  std::vector<double> D(kDTab), W(kWTab);
  for (int N = 2; N <= DG_MAX_N; ++N) {
    const LglTables t = make_lgl(N);
    std::copy(t.D, t.D + N * N, D.begin() + dtab_off(N));
    std::copy(t.w, t.w + N, W.begin() + wtab_off(N));
  }
  const std::vector<float> D32(D.begin(), D.end()), W32(W.begin(), W.end());
  DG_CUDA(cudaMemcpyToSymbol(cD64, D.data(), sizeof(double) * kDTab));
  DG_CUDA(cudaMemcpyToSymbol(cD32, D32.data(), sizeof(float) * kDTab));
  DG_CUDA(cudaMemcpyToSymbol(cW64, W.data(), sizeof(double) * kWTab));
  DG_CUDA(cudaMemcpyToSymbol(cW32, W32.data(), sizeof(float) * kWTab));
  done.insert(dev);
}

template <typename T>
void launch_apply(int N, const OpGeom<T>& g, const T* D, const T* w, const T* u, const T* diag, const T* b, T* out,
                  cudaStream_t s, const SubdomainOut* so_ptr, int variant, int* err) {
  const SubdomainOut so = so_ptr ? *so_ptr : SubdomainOut{};
  switch (N) {
    case 2: launch_apply_n<2, T>(g, D, w, u, diag, b, out, so, variant, err, s); break;
    case 3: launch_apply_n<3, T>(g, D, w, u, diag, b, out, so, variant, err, s); break;
    case 4: launch_apply_n<4, T>(g, D, w, u, diag, b, out, so, variant, err, s); break;
    case 5: launch_apply_n<5, T>(g, D, w, u, diag, b, out, so, variant, err, s); break;
    case 6: launch_apply_n<6, T>(g, D, w, u, diag, b, out, so, variant, err, s); break;
    case 7: launch_apply_n<7, T>(g, D, w, u, diag, b, out, so, variant, err, s); break;
    case 8: launch_apply_n<8, T>(g, D, w, u, diag, b, out, so, variant, err, s); break;
    case 9: launch_apply_n<9, T>(g, D, w, u, diag, b, out, so, variant, err, s); break;
    case 10: launch_apply_n<10, T>(g, D, w, u, diag, b, out, so, variant, err, s); break;
    default: fail(DG_ERR_INVALID_ARG, "unsupported N");
  }
  DG_LAUNCHED(1);
}

template void launch_apply<double>(int, const OpGeom<double>&, const double*, const double*, const double*,
                                   const double*, const double*, double*, cudaStream_t, const SubdomainOut*, int, int*);
template void launch_apply<float>(int, const OpGeom<float>&, const float*, const float*, const float*, const float*,
                                  const float*, float*, cudaStream_t, const SubdomainOut*, int, int*);

// static shared memory of the fused kernel stays within 48 KiB up to N = 8
bool coarse_smooth_available(int N) { return N >= 2 && N <= 8; }

void launch_coarse_smooth(int N, const CoarseArgs& a, cudaStream_t s) {
  DG_REQUIRE(a.sg.ld % 16 == 0, "fused coarse smoother needs a 16-aligned subdomain stride");
  switch (N) {
    case 2: launch_coarse_n<2>(a, s); break;
    case 3: launch_coarse_n<3>(a, s); break;
    case 4: launch_coarse_n<4>(a, s); break;
    case 5: launch_coarse_n<5>(a, s); break;
    case 6: launch_coarse_n<6>(a, s); break;
    case 7: launch_coarse_n<7>(a, s); break;
    case 8: launch_coarse_n<8>(a, s); break;
    default: fail(DG_ERR_INVALID_ARG, "fused coarse smoother supports N <= 8");
  }
  DG_LAUNCHED(1);
}


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
