// Device building blocks of the Schwarz data movement (Sec. III.D.5), shared by the per-step
// kernels of schwarz.cu and the fused coarse-level smoother: the table-driven gather of one
// subdomain column and the weighted scatter into one element. Both run with every thread of the
// calling CTA (any block size of at least 32) and may be called back to back on the same CTA.
#pragma once

#include "bounds.cuh"
#include "internal.h"
#include "pdl.cuh"

namespace dg {

// Face neighbour of element e across face f (-1 at the domain boundary).
__device__ __forceinline__ int nbr_elem(const SubdomainGeom& g, int e, int f) {
  const int c0 = e % g.n[0], c1 = (e / g.n[0]) % g.n[1], c2 = e / (g.n[0] * g.n[1]);
  int c[3] = {c0, c1, c2};
  const int d = f >> 1;
  c[d] += (f & 1) ? 1 : -1;
  if (c[d] < 0 || c[d] >= g.n[d]) return -1;
  return c[0] + g.n[0] * (c[1] + g.n[1] * c[2]);
}

// Index of the node at position idx_d along d and (a1, a2) along the other two dimensions in
// increasing order (the face layout shared by neighbours across a face of normal d).
template <int N>
__device__ __forceinline__ int node_of(int d, int idx_d, int a1, int a2) {
  int c0, c1, c2;
  if (d == 0) { c0 = idx_d; c1 = a1; c2 = a2; }
  else if (d == 1) { c0 = a1; c1 = idx_d; c2 = a2; }
  else { c0 = a1; c1 = a2; c2 = idx_d; }
  return (c2 * N + c1) * N + c0;
}

// Subdomain row of point p of slot s (0 centre, 1 + f the neighbour across face f) in the
// unreflected point order, or -1 if outside S.
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

// r_S column `col` = R_S r through the point map of the subdomain's orientation. With PDL the
// neighbour look-up overlaps the previous kernel.
template <typename T, bool PDL>
__device__ __forceinline__ void gather_column(const SubdomainGeom& g, const T* __restrict__ r,
                                              const int* __restrict__ elem_of_col, const int* __restrict__ orient,
                                              const int* __restrict__ map, T* __restrict__ rS, int col) {
  __shared__ int nb[7];
  const int e = elem_of_col[col];
  __syncthreads();  // the previous call on this CTA is done with nb
  if (threadIdx.x < 7) nb[threadIdx.x] = threadIdx.x == 0 ? e : nbr_elem(g, e, threadIdx.x - 1);
  __syncthreads();
  const int nS = g.nS, ld = g.ld, N3 = g.N * g.N * g.N;
  const int* m = map + (size_t)orient[e] * nS;
  T* out = rS + (size_t)col * ld;
  // the point map (static) is read before waiting for the previous kernel
  for (int q = threadIdx.x, first = 1; first || q < ld; q += blockDim.x, first = 0) {
    int64_t src = -1;
    if (q < nS) {
      const int code = __ldg(m + q);
      const int sl = code >> 16;
      const int el = DG_IN_BOUNDS(sl, 7) ? nb[sl] : -1;
      if (el >= 0 && DG_IN_BOUNDS((int64_t)el * N3 + (code & 0xFFFF), (int64_t)g.E * N3))
        src = (int64_t)el * N3 + (code & 0xFFFF);
    }
    if constexpr (PDL) {
      if (first) pdl_wait();
    }
    if (q < ld) out[q] = src >= 0 ? r[src] : T(0);
  }
}

// u(element q) += sum over the subdomains containing its points of w_S du_S. L2ONLY: du_S and u
// were written by other CTAs of the same kernel (read through L2 only).
template <typename T, typename TU, bool PDL, bool L2ONLY = false>
__device__ __forceinline__ void scatter_element(const SubdomainGeom& g, const T* __restrict__ duS,
                                                const int* __restrict__ col_of_elem, const int* __restrict__ orient,
                                                const int* __restrict__ inv, const T* __restrict__ shares,
                                                TU* __restrict__ u, int q) {
  __shared__ int s_col[7], s_inv[7], s_pat;
  const int N3 = g.N * g.N * g.N, ld = g.ld;
  __syncthreads();  // the previous call on this CTA is done with the shared look-ups
  if (threadIdx.x < 7) {
    const int f = threadIdx.x - 1;
    const int e = threadIdx.x == 0 ? q : nbr_elem(g, q, f);
    if (e >= 0) {
      s_col[threadIdx.x] = col_of_elem[e];
      // own subdomain: slot 0 of q's orientation; neighbour e sees q across its actual face
      // opposite to f, i.e. in slot 1 + (f ^ 1) of e's orientation
      const int slot = threadIdx.x == 0 ? 0 : 1 + (f ^ 1);
      s_inv[threadIdx.x] = (orient[e] * 7 + slot) * N3;
    } else {
      s_col[threadIdx.x] = -1;
      s_inv[threadIdx.x] = 0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int pat = 0;
    for (int f = 0; f < 6; ++f) pat |= (s_col[1 + f] >= 0) << f;
    s_pat = pat;
  }
  __syncthreads();
  const T* sh0 = shares + (size_t)s_pat * N3 * 7;
  // per point: the static look-ups (subdomain rows and weight shares) first, before waiting for the
  // previous kernel, then the seven du_S reads issued together
  for (int p = threadIdx.x, first = 1; first || p < N3; p += blockDim.x, first = 0) {
    const bool act = p < N3;
    int64_t idx[7];
    T w[7];
    if (act) {
      const T* sh = sh0 + (size_t)p * 7;
      // the neighbour across face f covers this point only within N_overlap layers of that face
      const int c[3] = {p % g.N, (p / g.N) % g.N, p / (g.N * g.N)};
#pragma unroll
      for (int sl = 0; sl < 7; ++sl) {
        bool in = s_col[sl] >= 0;
        if (sl > 0) {
          const int f = sl - 1, cd = c[f >> 1];
          in = in && ((f & 1) ? g.N - 1 - cd : cd) < g.ov;
        }
        const int row = in ? __ldg(inv + s_inv[sl] + p) : -1;
        idx[sl] = row >= 0 && DG_IN_BOUNDS(row, ld) && DG_IN_BOUNDS(s_col[sl], g.E) ? (int64_t)s_col[sl] * ld + row
                                                                                   : -1;
        w[sl] = row >= 0 ? sh[sl] : T(0);
      }
    }
    if constexpr (PDL) {
      if (first) pdl_wait();
    }
    if (!act) continue;
    T v[7];
#pragma unroll
    for (int sl = 0; sl < 7; ++sl) v[sl] = idx[sl] >= 0 ? (L2ONLY ? __ldcg(duS + idx[sl]) : duS[idx[sl]]) : T(0);
    TU* up = u + (int64_t)q * N3 + p;
    const TU u0 = L2ONLY ? __ldcg(up) : *up;
    T acc = w[0] * v[0];
#pragma unroll
    for (int sl = 1; sl < 7; ++sl) acc += w[sl] * v[sl];
    *up = u0 + (TU)acc;
  }
}

}  // namespace dg
