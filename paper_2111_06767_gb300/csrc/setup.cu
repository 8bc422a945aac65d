// Domain construction: LGL tables, the multigrid hierarchy (Sec. III.C.1), Schwarz subdomain
// index and weight tables (Sec. III.D) and the explicit subdomain inverses (Sec. III.E).
//
// Subdomain classes: on a uniform box the subdomain operator A_S of element e depends only on
// which of its faces have neighbours and, for each neighbour, whether that neighbour's far face
// (the one pointing away from e) is an external boundary. Up to reflections and exchanges of
// equal-width dimensions (the operator's symmetries) the subdomains fall into a handful of
// classes, each with one explicit inverse built once (see classify_schwarz).
//
// Weights (Eqs. schwarz_weight_prod, schwarz_weight_function): quintic smoothstep phi,
// w(xi) = (phi((xi + 1)/delta) - phi((xi - 1)/delta)) / 2, delta = 1 + x_{N_ov}. The edge and
// corner weight missing from the product is handed to face neighbours: per point the product
// prod_d (a_d + b_d^+ + b_d^-) = 1 (a_d = w(xi_d), b_d^+- = w(xi_d -+ 2)) is expanded, a term with
// m >= 1 neighbour factors goes 1/m to each of those face neighbours' subdomains; a side without
// a neighbour replaces its phi term by +-1 so that a_d absorbs it.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#include <cstdlib>
#include <cstring>

#include "domain.h"

namespace dg {

namespace {

const int kPerms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

double smoothstep(double x) {
  if (x >= 1.0) return 1.0;
  if (x <= -1.0) return -1.0;
  const double x2 = x * x;
  return x * (15.0 - 10.0 * x2 + 3.0 * x2 * x2) / 8.0;
}

double weight1d(double xi, double delta) { return 0.5 * (smoothstep((xi + 1.0) / delta) - smoothstep((xi - 1.0) / delta)); }

// shares[s] for s = 0 (own subdomain) and 1 + f (neighbour across face f) at one point.
void point_shares(const LglTables& t, int ov, const bool has_lo[3], const bool has_hi[3], const int idx[3],
                  double shares[7]) {
  const double delta = ov < t.N ? 1.0 + t.x[ov] : 2.0;
  double a[3], bm[3], bp[3];
  for (int d = 0; d < 3; ++d) {
    const double xi = t.x[idx[d]];
    const double lo = has_lo[d] ? smoothstep((xi + 1.0) / delta) : 1.0;
    const double hi = has_hi[d] ? smoothstep((xi - 1.0) / delta) : -1.0;
    a[d] = 0.5 * (lo - hi);
    bm[d] = has_lo[d] ? weight1d(xi + 2.0, delta) : 0.0;
    bp[d] = has_hi[d] ? weight1d(xi - 2.0, delta) : 0.0;
  }
  for (int s = 0; s < 7; ++s) shares[s] = 0.0;
  for (int cx = 0; cx < 3; ++cx)
    for (int cy = 0; cy < 3; ++cy)
      for (int cz = 0; cz < 3; ++cz) {
        const int ch[3] = {cx, cy, cz};
        double term = 1.0;
        int owners[3], m = 0;
        for (int d = 0; d < 3; ++d) {
          if (ch[d] == 0) term *= a[d];
          else if (ch[d] == 1) { term *= bm[d]; owners[m++] = 1 + 2 * d; }
          else { term *= bp[d]; owners[m++] = 2 + 2 * d; }
        }
        if (m == 0) shares[0] += term;
        else
          for (int q = 0; q < m; ++q) shares[owners[q]] += term / m;
      }
}

template <typename T>
void upload(DevBuf<T>& buf, const std::vector<T>& host, cudaStream_t s) {
  buf.alloc(host.size());
  if (!host.empty()) DG_CUDA(cudaMemcpyAsync(buf.get(), host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice, s));
}

template <typename T>
void upload_arr(DevBuf<T>& buf, const double* src, int n, cudaStream_t s) {
  std::vector<T> h(src, src + n);
  upload(buf, h, s);
}

// Per-level subdomain classes and column order (cheap: done at creation).
//
// Per dimension a subdomain sees, on each side, a Dirichlet box face (code 0), a Neumann box face
// (3), a neighbour whose far face is internal (1), or a neighbour whose far face is a Dirichlet (2)
// or Neumann (4) box face. A_S depends only on these six codes (uniform affine elements). The DG
// operator is invariant under reflecting a dimension and under swapping dimensions of equal element
// width (with the boundary types moving along), so every subdomain is mapped
// to a canonical orientation: each dimension reflected so that its lower code is the smaller,
// then dimensions of equal width sorted by their code pair. Subdomains with equal canonical codes
// share one explicit inverse, stored in the canonical point order; the gather and scatter kernels
// apply each subdomain's reflection/permutation on the fly.
void classify_schwarz(dg_domain* dom, Level& L) {
  const int N = dom->N, ov = dom->desc.overlap;
  const int N3 = N * N * N;
  SchwarzLevel& sw = L.sw;
  sw.nS = N3 + 6 * ov * N * N;
  sw.ld = (sw.nS + 31) / 32 * 32;
  sw.geom = SubdomainGeom{{L.n[0], L.n[1], L.n[2]}, L.E, N, ov, sw.nS, sw.ld};
  const int E = L.E;
  const int neu = dom->desc.neumann_faces;
  auto is_nbr = [](int code) { return code == 1 || code == 2 || code == 4; };
  std::vector<int> key(E), xform(E);
  for (int e = 0; e < E; ++e) {
    const int c[3] = {e % L.n[0], (e / L.n[0]) % L.n[1], e / (L.n[0] * L.n[1])};
    int lo[3], hi[3], flip[3];
    for (int d = 0; d < 3; ++d) {
      const int n = L.n[d];
      const int neu_lo = (neu >> (2 * d)) & 1, neu_hi = (neu >> (2 * d + 1)) & 1;
      lo[d] = c[d] > 0 ? (c[d] - 1 == 0 ? (neu_lo ? 4 : 2) : 1) : (neu_lo ? 3 : 0);
      hi[d] = c[d] < n - 1 ? (c[d] + 1 == n - 1 ? (neu_hi ? 4 : 2) : 1) : (neu_hi ? 3 : 0);
      flip[d] = lo[d] > hi[d];
      if (flip[d]) std::swap(lo[d], hi[d]);
    }
    // canonical axis a <- actual axis perm[a]; only dimensions of equal width may be exchanged
    int perm[3] = {0, 1, 2};
    auto pair_key = [&](int d) { return lo[d] * 5 + hi[d]; };
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j + 1 < 3 - i; ++j) {
        const int a = perm[j], b = perm[j + 1];
        if (L.h[a] == L.h[b] && pair_key(a) > pair_key(b)) std::swap(perm[j], perm[j + 1]);
      }
    int k = 0, fl = 0;
    for (int a = 0; a < 3; ++a) {
      k = k * 25 + pair_key(perm[a]);
      fl |= flip[perm[a]] << a;
    }
    int pi = 0;
    while (!(kPerms[pi][0] == perm[0] && kPerms[pi][1] == perm[1] && kPerms[pi][2] == perm[2])) ++pi;
    key[e] = k;
    xform[e] = pi * 8 + fl;
    if (dom->curved) {  // mapped elements: every subdomain is its own class, in its own orientation
      key[e] = e;
      xform[e] = 0;
    }
  }
  std::map<int, int> cls_id;
  for (int e = 0; e < E; ++e) cls_id.emplace(key[e], 0);
  int nc = 0;
  sw.class_key.clear();
  for (auto& kv : cls_id) {
    kv.second = nc++;
    sw.class_key.push_back(kv.first);
  }
  sw.n_classes = nc;
  sw.class_of.resize(E);
  sw.class_count.assign(nc, 0);
  for (int e = 0; e < E; ++e) {
    sw.class_of[e] = cls_id[key[e]];
    sw.class_count[sw.class_of[e]]++;
  }
  sw.class_first.assign(nc, 0);
  for (int c = 1; c < nc; ++c) sw.class_first[c] = sw.class_first[c - 1] + sw.class_count[c - 1];
  sw.position.resize(E);
  std::vector<int> elem_of_col(E);
  {
    std::vector<int> fill = sw.class_first;
    for (int e = 0; e < E; ++e) {
      sw.position[e] = fill[sw.class_of[e]]++;
      elem_of_col[sw.position[e]] = e;
    }
  }
  // canonical patch of every class (slot 0 centre, 1 + f neighbour across canonical face f)
  sw.patch.assign((size_t)nc * 49, -2);
  for (auto& kv : cls_id) {
    if (dom->curved) break;  // curved subdomain matrices are built from the grid itself
    int codes[3][2];  // [canonical axis][side]
    int k = kv.first;
    for (int a = 2; a >= 0; --a) {
      codes[a][0] = (k % 25) / 5;
      codes[a][1] = k % 5;
      k /= 25;
    }
    int* P = &sw.patch[(size_t)kv.second * 49];
    for (int s = 0; s < 7; ++s) P[42 + s] = 0;
    P[42] = 1;
    for (int f = 0; f < 6; ++f) {
      const int a = f >> 1, side = f & 1;
      const int cd = codes[a][side];
      P[f] = is_nbr(cd) ? 1 + f : (cd == 0 ? -1 : -3);
      P[42 + 1 + f] = is_nbr(cd);
      if (!is_nbr(cd)) continue;
      const int back = 2 * a + (1 - side);
      for (int ff = 0; ff < 6; ++ff) {
        const int aa = ff >> 1, ss = ff & 1;
        if (ff == back) P[(1 + f) * 6 + ff] = 0;                 // faces the centre
        else if (ff == f) P[(1 + f) * 6 + ff] = cd == 2 ? -1 : (cd == 4 ? -3 : -2);  // far face
        else P[(1 + f) * 6 + ff] = is_nbr(codes[aa][ss]) ? -2 : (codes[aa][ss] == 0 ? -1 : -3);  // as the centre's
      }
    }
  }
  cudaStream_t s = dom->stream;
  upload(sw.elem_of_col, elem_of_col, s);
  upload(sw.col_of_elem, sw.position, s);
  {
    std::vector<int> class_of_col(E);
    for (int e = 0; e < E; ++e) class_of_col[sw.position[e]] = sw.class_of[e];
    upload(sw.class_of_col, class_of_col, s);
  }
  upload(sw.xform_of_elem, xform, s);
  // Rows (and columns) of a class's inverse in the slots of missing neighbours have no coupling to
  // the rest (identity block): K chunks and row tiles that meet no present slot are skipped, and
  // tiles whose rows lie only there just write zeros (zero flag, bit 30 of the tile's first word).
  const int slot_rows = ov * N * N;
  auto present = [&](int c, int r0, int r1) {  // does row range [r0, r1) meet a present slot?
    if (dom->curved) return true;
    for (int sl = 0; sl < 7; ++sl) {
      if (!sw.patch[(size_t)c * 49 + 42 + sl]) continue;
      const int a = sl == 0 ? 0 : N3 + (sl - 1) * slot_rows, b = sl == 0 ? N3 : a + slot_rows;
      if (r0 < b && a < r1) return true;
    }
    return false;
  };
  sw.class_nS.assign(nc, sw.nS);
  sw.alg_inv = sw.alg_vec = sw.alg_mac = 0;
  for (int c = 0; c < nc; ++c) {
    if (!dom->curved) {
      sw.class_nS[c] = N3;
      for (int f = 0; f < 6; ++f) sw.class_nS[c] += sw.patch[(size_t)c * 49 + 43 + f] ? slot_rows : 0;
    }
    const double n = sw.class_nS[c], m = sw.class_count[c];
    sw.alg_inv += dom->curved ? m * n * n : n * n;  // curved: one inverse per subdomain
    sw.alg_vec += m * n;
    sw.alg_mac += m * n * n;
  }
  for (int bk : {16, 32}) {
    const int per = sw.ld / bk + 1, nck = dom->curved ? 0 : nc;  // curved levels use no class GEMM
    std::vector<int> kc((size_t)nck * per, 0);
    for (int c = 0; c < nck; ++c) {
      int* k = &kc[(size_t)c * per];
      for (int q = 0; q < sw.ld / bk; ++q)
        if (present(c, q * bk, (q + 1) * bk)) k[1 + k[0]++] = q;
    }
    upload(bk == 16 ? sw.kchunks16 : sw.kchunks32, kc, s);
  }
  auto tile = [&](int c, int r0, int rows, int c0, int wcode) {
    const int zero = present(c, r0, std::min(r0 + rows, sw.ld)) ? 0 : 1;
    return make_int4(c | (wcode << 24) | (zero << 30), r0, sw.class_first[c] + c0, sw.class_count[c] - c0);
  };
  // CUDA-core tiles: 64 columns while more than 48 are left, then 32 and/or 16
  std::vector<int4> tiles;
  for (int c = 0; c < (dom->curved ? 0 : nc); ++c)
    for (int r0 = 0; r0 < sw.ld; r0 += 64)
      for (int c0 = 0; c0 < sw.class_count[c];) {
        const int left = sw.class_count[c] - c0;
        const int w = left > 48 ? 64 : (left > 16 ? 32 : 16);
        tiles.push_back(tile(c, r0, 64, c0, w == 64 ? 0 : (w == 32 ? 1 : 2)));
        c0 += w;
      }
  sw.n_tiles = (int)tiles.size();
  upload(sw.tiles, tiles, s);
  std::vector<int4> tiles_tc;
  for (int c = 0; c < (dom->curved ? 0 : nc); ++c)
    for (int r0 = 0; r0 < sw.ld; r0 += 128)
      for (int c0 = 0; c0 < sw.class_count[c]; c0 += 64) tiles_tc.push_back(tile(c, r0, 128, c0, 0));
  sw.n_tiles_tc = (int)tiles_tc.size();
  upload(sw.tiles_tc, tiles_tc, s);
  std::vector<int4> tiles_tc128;
  for (int c = 0; c < (dom->curved ? 0 : nc); ++c)
    for (int r0 = 0; r0 < sw.ld; r0 += 128)
      for (int c0 = 0; c0 < sw.class_count[c]; c0 += 128) tiles_tc128.push_back(tile(c, r0, 128, c0, 0));
  sw.n_tiles_tc128 = (int)tiles_tc128.size();
  upload(sw.tiles_tc128, tiles_tc128, s);
  std::vector<int4> tiles_tc256;
  for (int c = 0; c < (dom->curved ? 0 : nc); ++c)
    for (int r0 = 0; r0 < sw.ld; r0 += 128)
      for (int c0 = 0; c0 < sw.class_count[c]; c0 += 256) tiles_tc256.push_back(tile(c, r0, 128, c0, 0));
  sw.n_tiles_tc256 = (int)tiles_tc256.size();
  upload(sw.tiles_tc256, tiles_tc256, s);
  std::vector<int4> units;
  for (int c = 0; c < (dom->curved ? 0 : nc); ++c)
    for (int r0 = 0; r0 < sw.ld; r0 += 16) units.push_back(make_int4(c, r0, sw.class_first[c], sw.class_count[c]));
  sw.n_units = (int)units.size();
  upload(sw.units, units, s);
  sw.bar.alloc(2);
  DG_CUDA(cudaMemsetAsync(sw.bar.get(), 0, sw.bar.bytes(), s));
}

// Point maps of the 48 subdomain orientations (orientation o = 8 perm + flips: canonical axis a is
// actual axis kPerms[perm][a], reflected if bit a of flips): map[o][q] = (actual slot << 16) |
// actual point of canonical subdomain row q; inv[o][slot][p] = canonical row of point p of that
// actual slot, -1 outside the subdomain.
void build_orientation_tables(dg_domain* dom) {
  const int N = dom->N, N2 = N * N, N3 = N2 * N, ov = dom->desc.overlap;
  const int nS = N3 + 6 * ov * N2;
  std::vector<int> map((size_t)48 * nS), inv((size_t)48 * 7 * N3, -1);
  for (int pi = 0; pi < 6; ++pi)
    for (int fl = 0; fl < 8; ++fl) {
      const int o = pi * 8 + fl;
      const int* perm = kPerms[pi];
      int invp[3];
      for (int a = 0; a < 3; ++a) invp[perm[a]] = a;
      for (int q = 0; q < nS; ++q) {
        int cc[3], slot = 0;
        if (q < N3) {
          cc[0] = q % N;
          cc[1] = (q / N) % N;
          cc[2] = q / N2;
        } else {
          const int rr = q - N3, fc = rr / (ov * N2), k = rr - fc * ov * N2;
          const int depth = k / N2, a2 = (k / N) % N, a1 = k % N;
          const int a = fc >> 1, sc = fc & 1;
          const int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
          cc[a] = sc ? depth : N - 1 - depth;
          cc[t1] = a1;
          cc[t2] = a2;
          const int d = perm[a];
          const int sa = ((fl >> a) & 1) ? 1 - sc : sc;
          slot = 1 + 2 * d + sa;
        }
        int ca[3];
        for (int d = 0; d < 3; ++d) {
          const int a = invp[d];
          ca[d] = ((fl >> a) & 1) ? N - 1 - cc[a] : cc[a];
        }
        const int p = (ca[2] * N + ca[1]) * N + ca[0];
        map[(size_t)o * nS + q] = (slot << 16) | p;
        inv[((size_t)o * 7 + slot) * N3 + p] = q;
      }
    }
  upload(dom->orient_map, map, dom->stream);
  upload(dom->orient_inv, inv, dom->stream);
}

// Schwarz weight shares of every point for the 64 patterns of existing face neighbours.
void build_shares(dg_domain* dom) {
  const int N = dom->N, N3 = N * N * N, ov = dom->desc.overlap;
  std::vector<double> sh((size_t)64 * N3 * 7);
  for (int pat = 0; pat < 64; ++pat) {
    bool has_lo[3], has_hi[3];
    for (int d = 0; d < 3; ++d) {
      has_lo[d] = (pat >> (2 * d)) & 1;
      has_hi[d] = (pat >> (2 * d + 1)) & 1;
    }
    for (int p = 0; p < N3; ++p) {
      const int c[3] = {p % N, (p / N) % N, p / (N * N)};
      point_shares(dom->lgl, ov, has_lo, has_hi, c, &sh[((size_t)pat * N3 + p) * 7]);
    }
  }
  if (dom->mixed) {
    std::vector<float> s32(sh.begin(), sh.end());
    upload(dom->shares32, s32, dom->stream);
  } else {
    upload(dom->shares64, sh, dom->stream);
  }
}

template <typename T>
void alloc_work(LevelWork<T>& w, const Level& L, cudaStream_t s) {
  w.b.alloc(L.ndof);
  w.u.alloc(L.ndof);
  w.r.alloc(L.ndof);
  w.rS.alloc((size_t)L.E * L.sw.ld);
  w.duS.alloc((size_t)L.E * L.sw.ld);
  // rows of r_S that no point maps to (missing neighbours, stride padding) stay zero for good: the
  // fused residual writes only mapped rows
  DG_CUDA(cudaMemsetAsync(w.rS.get(), 0, w.rS.bytes(), s));
}

}  // namespace

// Curved elements or a variable coefficient: the level-0 node coordinates (the caller's, else the
// box's) and coefficient (the caller's, else 1), the coarse levels' nodes and coefficient on the
// interpolated fine fields (per coarsened dimension the coarse node xi_c lies in the lower child,
// xi_c <= 0, at child coordinate 2 xi_c + 1, or in the upper one at 2 xi_c - 1), then per level the
// nodal metric and the face-node penalty; the mass diagonal w_p J_p of level 0.
void setup_curved_geometry(dg_domain* dom, const double* host_xyz, const double* host_coef) {
  const int N = dom->N;
  cudaStream_t s = dom->stream;
  const LglTables& t = dom->lgl;
  const Level& L0 = dom->levels[0];
  const size_t n0 = (size_t)L0.ndof;
  DevBuf<double> xyz(4 * n0);  // x, y, z, K
  if (host_xyz) {
    DG_CUDA(cudaMemcpyAsync(xyz.get(), host_xyz, 3 * n0 * sizeof(double), cudaMemcpyHostToDevice, s));
    DG_CUDA(cudaMemcpyAsync(dom->X.get(), xyz.get(), n0 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    DG_CUDA(cudaMemcpyAsync(dom->Y.get(), xyz.get() + n0, n0 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    DG_CUDA(cudaMemcpyAsync(dom->Z.get(), xyz.get() + 2 * n0, n0 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else {
    launch_node_coords(N, L0.n, dom->desc.lower, L0.h, dom->x1.get(), dom->X.get(), dom->Y.get(), dom->Z.get(), s);
    DG_CUDA(cudaMemcpyAsync(xyz.get(), dom->X.get(), n0 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    DG_CUDA(cudaMemcpyAsync(xyz.get() + n0, dom->Y.get(), n0 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    DG_CUDA(cudaMemcpyAsync(xyz.get() + 2 * n0, dom->Z.get(), n0 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  if (host_coef) {
    DG_CUDA(cudaMemcpyAsync(xyz.get() + 3 * n0, host_coef, n0 * sizeof(double), cudaMemcpyHostToDevice, s));
  } else {
    launch_fill<double>((int64_t)n0, 1.0, xyz.get() + 3 * n0, s);
  }
  // coarsening weights: [lower child][c][q], [upper child][c][q], identity, upper-half flag per node
  std::vector<double> C(3 * N * N + N, 0.0);
  auto lagrange = [&](int q, double x) {
    double v = 1.0;
    for (int m = 0; m < N; ++m)
      if (m != q) v *= (x - t.x[m]) / (t.x[q] - t.x[m]);
    return v;
  };
  for (int c = 0; c < N; ++c) {
    const bool upper = t.x[c] > 0.0;
    for (int q = 0; q < N; ++q) {
      C[(upper ? N * N : 0) + c * N + q] = lagrange(q, upper ? 2.0 * t.x[c] - 1.0 : 2.0 * t.x[c] + 1.0);
      C[2 * N * N + c * N + q] = c == q ? 1.0 : 0.0;
    }
    C[3 * N * N + c] = upper ? 1.0 : 0.0;
  }
  DevBuf<double> dC;
  upload(dC, C, s);
  DevBuf<int> bad(1);
  DG_CUDA(cudaMemsetAsync(bad.get(), 0, sizeof(int), s));
  DevBuf<double> cur = std::move(xyz);
  for (size_t l = 0; l < dom->levels.size(); ++l) {
    Level& L = dom->levels[l];
    if (l > 0) {
      DevBuf<double> next(4 * (size_t)L.ndof);
      launch_curved_coarsen(N, L.n, dom->levels[l - 1].n, dC.get(), cur.get(), next.get(), s);
      cur = std::move(next);
    }
    L.geo64.alloc(11 * (size_t)L.ndof);
    L.geo32.alloc(11 * (size_t)L.ndof);
    launch_curved_metric(N, L.E, cur.get(), dom->D64.get(), L.geo64.get(), L.geo32.get(), bad.get(), s);
    const size_t nf = (size_t)L.E * 6 * N * N;
    L.sig64.alloc(nf);
    L.sig32.alloc(nf);
    launch_curved_sigma(N, L.n, dom->desc.penalty, L.geo64.get(), L.sig64.get(), L.sig32.get(), s);
    L.trace32.alloc(nf);
    L.trace64.alloc(nf);
  }
  launch_curved_mass(N, dom->w64.get(), L0.geo64.get(), L0.ndof, dom->mass.get(), s);
  int h_bad = 0;
  DG_CUDA(cudaMemcpyAsync(&h_bad, bad.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  DG_REQUIRE(h_bad != 1, "node coordinates give a folded or left-handed element (Jacobian determinant <= 0)");
  DG_REQUIRE(h_bad != 2, "the coefficient must be positive at every node");
}

void domain_setup(dg_domain* dom) {
  const dg_domain_desc& d = dom->desc;
  DG_REQUIRE(d.N >= 2 && d.N <= DG_MAX_N, "N must be in [2, 10]");
  for (int i = 0; i < 3; ++i) {
    DG_REQUIRE(d.n[i] >= 1 && d.n[i] <= 4096, "element counts must be in [1, 4096]");
    DG_REQUIRE(d.upper[i] > d.lower[i], "upper must exceed lower");
  }
  DG_REQUIRE(d.penalty > 0, "penalty must be positive");
  DG_REQUIRE(d.overlap >= 1 && d.overlap <= d.N - 1, "overlap must be in [1, N-1]");
  DG_REQUIRE(d.presmooth >= 0 && d.postsmooth >= 0 && d.presmooth + d.postsmooth >= 1, "need smoothing steps");
  DG_REQUIRE(d.precision == DG_PRECISION_FP64 || d.precision == DG_PRECISION_MIXED, "bad precision");
  DG_REQUIRE(d.problem == DG_PROBLEM_POISSON || d.problem == DG_PROBLEM_PUNCTURE, "bad problem");
  DG_REQUIRE(d.mg_levels >= 0 && d.mg_levels <= DG_MAX_LEVELS, "mg_levels must be in [0, 8]");
  DG_REQUIRE(d.neumann_faces >= 0 && d.neumann_faces < 63,
             "neumann_faces must be a mask of box faces with at least one Dirichlet face");
  DG_REQUIRE(d.subdomain_gemm >= DG_GEMM_DEFAULT && d.subdomain_gemm <= DG_GEMM_TENSOR_TF32, "bad subdomain_gemm");
  DG_REQUIRE(d.subdomain_gemm != DG_GEMM_TENSOR_TF32 || d.precision == DG_PRECISION_MIXED,
             "tensor-core subdomain GEMM needs a MIXED domain");
  DG_REQUIRE(d.problem != DG_PROBLEM_PUNCTURE || (d.n_punctures >= 0 && d.n_punctures <= DG_MAX_PUNCTURES),
             "bad puncture count");
  DG_REQUIRE((!d.node_xyz && !d.coef) || d.problem == DG_PROBLEM_POISSON,
             "curved elements and variable coefficients are supported for POISSON only");
  const int64_t ndof = (int64_t)d.n[0] * d.n[1] * d.n[2] * d.N * d.N * d.N;
  DG_REQUIRE(ndof < (int64_t)1 << 31, "problem too large for 32-bit point indices");
  dom->N = d.N;
  dom->mixed = d.precision == DG_PRECISION_MIXED;
  dom->curved = d.node_xyz != nullptr || d.coef != nullptr;
  dom->mapped = d.node_xyz != nullptr;
  dom->use_tc = dom->mixed && d.subdomain_gemm != DG_GEMM_SIMT;
  {
    const char* v = std::getenv("DG_COARSE_FUSED");
    dom->coarse_fused = v && std::strcmp(v, "1") == 0 && !dom->curved;
  }
  if (dom->use_tc && !tc_gemm_available()) {
    DG_REQUIRE(d.subdomain_gemm != DG_GEMM_TENSOR_TF32, "tensor-core GEMM requested but TMA encoding is unavailable");
    dom->use_tc = false;
  }
  dom->err_flag.alloc(1);
  DG_CUDA(cudaMemsetAsync(dom->err_flag.get(), 0, sizeof(int), dom->stream));
  dom->lgl = make_lgl(d.N);
  upload_operator_tables();
  keep_pool_memory();
  cudaStream_t s = dom->stream;
  const LglTables& t = dom->lgl;
  const int N = d.N;
  upload_arr(dom->D64, t.D, N * N, s);
  upload_arr(dom->w64, t.w, N, s);
  upload_arr(dom->Ilo64, t.I_lo, N * N, s);
  upload_arr(dom->Ihi64, t.I_hi, N * N, s);
  upload_arr(dom->x1, t.x, N, s);
  upload_arr(dom->D32, t.D, N * N, s);
  upload_arr(dom->w32, t.w, N, s);
  upload_arr(dom->Ilo32, t.I_lo, N * N, s);
  upload_arr(dom->Ihi32, t.I_hi, N * N, s);
  // hierarchy: halve every even dimension per level
  int n[3] = {d.n[0], d.n[1], d.n[2]};
  for (;;) {
    Level L;
    for (int i = 0; i < 3; ++i) {
      L.n[i] = n[i];
      L.h[i] = (d.upper[i] - d.lower[i]) / n[i];
    }
    L.E = n[0] * n[1] * n[2];
    L.ndof = (int64_t)L.E * N * N * N;
    L.g64 = make_geom<double>(L.n, L.h, N, d.penalty, t, d.neumann_faces);
    L.g32 = make_geom<float>(L.n, L.h, N, d.penalty, t, d.neumann_faces);
    dom->levels.push_back(std::move(L));
    if ((int)dom->levels.size() == (d.mg_levels ? d.mg_levels : DG_MAX_LEVELS)) break;
    if (n[0] % 2 && n[1] % 2 && n[2] % 2) break;
    for (int i = 0; i < 3; ++i)
      if (n[i] % 2 == 0) n[i] /= 2;
  }
  const Level& L0 = dom->levels[0];
  dom->X.alloc(L0.ndof);
  dom->Y.alloc(L0.ndof);
  dom->Z.alloc(L0.ndof);
  dom->mass.alloc(L0.ndof);
  if (dom->curved) {
    setup_curved_geometry(dom, d.node_xyz, d.coef);
    dom->desc.node_xyz = nullptr;  // the caller's buffers are not kept
    dom->desc.coef = nullptr;
  } else {
    launch_node_coords(N, L0.n, d.lower, L0.h, dom->x1.get(), dom->X.get(), dom->Y.get(), dom->Z.get(), s);
    launch_mass_diag<double>(N, L0.g64, dom->w64.get(), L0.ndof, dom->mass.get(), s);
  }
  for (auto& L : dom->levels) classify_schwarz(dom, L);
  build_shares(dom);
  build_orientation_tables(dom);
  if (d.problem == DG_PROBLEM_PUNCTURE) {
    dom->alpha.alloc(L0.ndof);
    dom->beta.alloc(L0.ndof);
    dom->lin64.alloc(L0.ndof);
    if (dom->mixed) dom->lin32.alloc(L0.ndof);
    launch_puncture_fields(L0.ndof, dom->X.get(), dom->Y.get(), dom->Z.get(), d.n_punctures, d.punctures,
                           dom->alpha.get(), dom->beta.get(), s);
  }
  DG_CUDA(cudaStreamSynchronize(s));
}

// Explicit inverses and work vectors of one level, built on first use (Sec. III.E: construction
// cost amortised over all later solves).
namespace {

// Library-wide store of built inverses. Every term of the affine Poisson DG operator scales with
// the element size in 3-D (mass h^3 x derivatives h^-2, face mass h^2 x penalty and lifting h^-1),
// so A_S(h) = h_x A_S(h / h_x) and one inverse built at h_x = 1 serves every grid with the same
// aspect ratios, order, overlap, penalty and boundary pattern: A_S(h)^-1 = (1/h_x) A_S(h/h_x)^-1.
// Entries live until the process exits (bounded by kCacheCap; beyond it new inverses are built
// but not kept).
struct InvKey {
  int dev, N, ov, key, fp64;
  double penalty, a1, a2;
  bool operator<(const InvKey& o) const {
    return std::tie(dev, N, ov, key, fp64, penalty, a1, a2) <
           std::tie(o.dev, o.N, o.ov, o.key, o.fp64, o.penalty, o.a1, o.a2);
  }
};
constexpr size_t kCacheCap = size_t(8) << 30;
std::mutex g_inv_mu;
std::map<InvKey, void*>* g_inv = new std::map<InvKey, void*>();  // device buffers of ld^2 entries
size_t g_inv_bytes = 0;

}  // namespace

namespace {
// Curved elements: the explicit inverse of every subdomain's own A_S (row-major, compact n_S x n_S),
// built column by column from the curved operator on its patch, inverted in place by Gauss-Jordan
// without pivoting (the symmetric part of A_S is positive definite, so no pivot vanishes).
template <typename T>
void build_curved_inverses(dg_domain* dom, Level& L, DevBuf<T>& inv, const T* geo, const T* sig, const T* D,
                           const T* w, cudaStream_t s) {
  const int nS = L.sw.nS, E = L.E;
  const size_t n2 = (size_t)nS * nS;
  inv.alloc((size_t)E * n2);
  CurvedArgs<T> a{};
  for (int i = 0; i < 3; ++i) a.n[i] = L.n[i];
  a.neumann = dom->desc.neumann_faces;
  a.ndof = L.ndof;
  a.geo = geo;
  a.sigma = sig;
  a.D = D;
  a.w = w;
  constexpr int kBatch = 65535;  // grid limits of the column and Gauss-Jordan launches
  for (int e0 = 0; e0 < E; e0 += kBatch) {
    const int cnt = std::min(kBatch, E - e0);
    launch_curved_columns<T>(dom->N, a, dom->desc.overlap, nS, e0, cnt, inv.get() + (size_t)e0 * n2, s);
    launch_invert_spd_batched<T>(inv.get() + (size_t)e0 * n2, nS, cnt, s);
  }
}
}  // namespace

// Explicit inverses and work vectors of one level, built on first use (Sec. III.E: construction
// cost amortised over all later solves).
void ensure_schwarz(dg_domain* dom, int level) {
  Level& L = dom->levels[level];
  SchwarzLevel& sw = L.sw;
  if (sw.built) return;
  if (dom->curved) {
    cudaStream_t s = dom->stream;
    sw.inv_scale = 1.0;
    if (dom->mixed) {
      build_curved_inverses<float>(dom, L, sw.inv32, L.geo32.get(), L.sig32.get(), dom->D32.get(), dom->w32.get(), s);
      if (dom->desc.subdomain_gemm != DG_GEMM_SIMT) {
        // the smoother streams every inverse once per step: keep them in FP16 (scaled per subdomain),
        // the input precision of the tensor-core path; "simt" keeps FP32
        sw.inv16.alloc((size_t)L.E * sw.nS * sw.nS);
        sw.inv16_scale.alloc(L.E);
        launch_to_half_scaled(sw.inv32.get(), sw.nS, L.E, sw.inv16.get(), sw.inv16_scale.get(), s);
        DG_CUDA(cudaStreamSynchronize(s));
        sw.inv32.release();
      }
      alloc_work(L.w32, L, s);
    } else {
      build_curved_inverses<double>(dom, L, sw.inv64, L.geo64.get(), L.sig64.get(), dom->D64.get(), dom->w64.get(),
                                    s);
      alloc_work(L.w64, L, s);
    }
    DG_CUDA(cudaStreamSynchronize(s));
    sw.built = true;
    dom->bytes = domain_device_bytes(dom);
    return;
  }
  const int N = dom->N, ov = dom->desc.overlap, nS = sw.nS, nc = sw.n_classes;
  cudaStream_t s = dom->stream;
  DG_CUDA(cudaStreamSynchronize(s));
  const int ld = sw.ld;
  const size_t esz = dom->mixed ? sizeof(float) : sizeof(double);
  const size_t mat = (size_t)ld * ld * esz;
  int dev = 0;
  DG_CUDA(cudaGetDevice(&dev));
  const double hx = L.h[0];
  sw.inv_scale = 1.0 / hx;
  if (dom->mixed) sw.inv32.alloc((size_t)nc * ld * ld);
  else sw.inv64.alloc((size_t)nc * ld * ld);
  char* dst = dom->mixed ? (char*)sw.inv32.get() : (char*)sw.inv64.get();
  std::vector<int> missing;
  std::vector<InvKey> keys(nc);
  {
    // cached entries are never freed, so their copies may run after the lock is released
    std::lock_guard<std::mutex> lk(g_inv_mu);
    for (int c = 0; c < nc; ++c) {
      keys[c] = InvKey{dev, N, ov, sw.class_key[c], dom->mixed ? 0 : 1, dom->desc.penalty, L.h[1] / hx, L.h[2] / hx};
      auto it = g_inv->find(keys[c]);
      if (it != g_inv->end())
        DG_CUDA(cudaMemcpyAsync(dst + c * mat, it->second, mat, cudaMemcpyDeviceToDevice, s));
      else
        missing.push_back(c);
    }
  }
  if (!missing.empty()) {
    // build the missing classes at unit width: A_S column by column, then Gauss-Jordan in FP64
    const int nm = (int)missing.size();
    std::vector<int> patch((size_t)nm * 49);
    for (int i = 0; i < nm; ++i)
      std::copy(sw.patch.begin() + (size_t)missing[i] * 49, sw.patch.begin() + (size_t)(missing[i] + 1) * 49,
                patch.begin() + (size_t)i * 49);
    DevBuf<int> d_patch;
    upload(d_patch, patch, s);
    const double hu[3] = {1.0, L.h[1] / hx, L.h[2] / hx};
    DevBuf<char> built((size_t)nm * mat);
    if (dom->mixed) {
      // stored in FP32 for an FP32/TF32 smoother: built and inverted in FP32 (A_S is well
      // conditioned; GB300's FP32 rate is ~60x its FP64 rate)
      const OpGeom<float> gu = make_geom<float>(L.n, hu, N, dom->desc.penalty, dom->lgl);
      DevBuf<float> c32((size_t)nm * nS * nS);
      launch_build_subdomain_matrices<float>(N, ov, gu, dom->D32.get(), dom->w32.get(), d_patch.get(), nm, nS,
                                             c32.get(), s);
      launch_invert_spd_batched<float>(c32.get(), nS, nm, s);
      launch_pad_convert<float, float>(c32.get(), nS, ld, nm, (float*)built.get(), s);
    } else {
      const OpGeom<double> gu = make_geom<double>(L.n, hu, N, dom->desc.penalty, dom->lgl);
      DevBuf<double> compact((size_t)nm * nS * nS);
      launch_build_subdomain_matrices<double>(N, ov, gu, dom->D64.get(), dom->w64.get(), d_patch.get(), nm, nS,
                                              compact.get(), s);
      launch_invert_spd_batched<double>(compact.get(), nS, nm, s);
      launch_pad_convert<double, double>(compact.get(), nS, ld, nm, (double*)built.get(), s);
    }
    for (int i = 0; i < nm; ++i)
      DG_CUDA(cudaMemcpyAsync(dst + missing[i] * mat, built.get() + i * mat, mat, cudaMemcpyDeviceToDevice, s));
    // keep a copy for later domains (built outside the lock; another thread may have won the race)
    for (int i = 0; i < nm; ++i) {
      {
        std::lock_guard<std::mutex> lk(g_inv_mu);
        if (g_inv->count(keys[missing[i]]) || g_inv_bytes + mat > kCacheCap) continue;
        g_inv_bytes += mat;
      }
      void* keep = nullptr;
      if (cudaMallocAsync(&keep, mat, s) != cudaSuccess) {
        (void)cudaGetLastError();
        std::lock_guard<std::mutex> lk(g_inv_mu);
        g_inv_bytes -= mat;
        continue;
      }
      DG_CUDA(cudaMemcpyAsync(keep, built.get() + i * mat, mat, cudaMemcpyDeviceToDevice, s));
      DG_CUDA(cudaStreamSynchronize(s));
      std::lock_guard<std::mutex> lk(g_inv_mu);
      if (!g_inv->emplace(keys[missing[i]], keep).second) {
        cudaFreeAsync(keep, s);
        g_inv_bytes -= mat;
      }
    }
    DG_CUDA(cudaStreamSynchronize(s));
  }
  if (dom->mixed) alloc_work(L.w32, L, s);
  else alloc_work(L.w64, L, s);
  DG_CUDA(cudaStreamSynchronize(s));
  sw.built = true;
  dom->bytes = domain_device_bytes(dom);
}

size_t domain_device_bytes(const dg_domain* dom) {
  size_t b = dom->D64.bytes() + dom->w64.bytes() + dom->Ilo64.bytes() + dom->Ihi64.bytes() + dom->x1.bytes() +
             dom->D32.bytes() + dom->w32.bytes() + dom->Ilo32.bytes() + dom->Ihi32.bytes() + dom->X.bytes() +
             dom->Y.bytes() + dom->Z.bytes() + dom->mass.bytes() + dom->alpha.bytes() + dom->beta.bytes() +
             dom->lin64.bytes() + dom->lin32.bytes() + dom->V.bytes() + dom->Zb.bytes() + dom->w.bytes() +
             dom->r.bytes() + dom->du.bytes() + dom->ut.bytes() + dom->rt.bytes() + dom->tmp.bytes() +
             dom->partial.bytes() + dom->dots.bytes() + dom->vin32.bytes() + dom->shares64.bytes() +
             dom->shares32.bytes() + dom->orient_map.bytes() + dom->orient_inv.bytes() + dom->vin64.bytes() +
             dom->vout64.bytes() + dom->err_flag.bytes();
  for (const auto& L : dom->levels) {
    const auto& sw = L.sw;
    b += L.geo64.bytes() + L.geo32.bytes() + L.sig64.bytes() + L.sig32.bytes() + L.trace64.bytes() +
         L.trace32.bytes();
    b += sw.elem_of_col.bytes() + sw.col_of_elem.bytes() + sw.class_of_col.bytes() + sw.xform_of_elem.bytes() +
         sw.inv64.bytes() +
         sw.inv32.bytes() + sw.inv16.bytes() + sw.inv16_scale.bytes() + sw.tiles.bytes() + sw.tiles_tc.bytes() +
         sw.tiles_tc128.bytes() + sw.tiles_tc256.bytes() +
         sw.units.bytes() + sw.bar.bytes();
    for (auto* p : {&L.w64.b, &L.w64.u, &L.w64.r, &L.w64.rS, &L.w64.duS, &L.w64.gV, &L.w64.gZ, &L.w64.gW, &L.w64.gD,
                    &L.w64.gH, &L.w64.linA, &L.w64.linv})
      b += p->bytes();
    for (auto* p : {&L.w32.b, &L.w32.u, &L.w32.r, &L.w32.rS, &L.w32.duS, &L.w32.gV, &L.w32.gZ, &L.w32.gW, &L.w32.gD,
                    &L.w32.gH, &L.w32.linA, &L.w32.linv})
      b += p->bytes();
  }
  return b;
}

}  // namespace dg
