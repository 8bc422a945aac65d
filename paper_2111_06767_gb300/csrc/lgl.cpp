// Legendre-Gauss-Lobatto tables for the element-local operators (Sec. II, Eqs. field_expansion,
// lagrprod) and the multigrid prolongation (Eq. prol). Host code, computed once per order N.
//
// Points: x_0 = -1, x_{N-1} = +1 and the N-2 roots of P'_{N-1}, found by Newton's method on
// q(x) = P'_{N-1}(x) in long double from Chebyshev-Gauss-Lobatto starting points.
// Weights: w_k = 2 / (N (N-1) P_{N-1}(x_k)^2).
// Differentiation: barycentric form D_kl = (b_l / b_k) / (x_k - x_l), D_kk = -sum_{l != k} D_kl,
// with barycentric weights b_j = 1 / prod_{m != j} (x_j - x_m).
// Interpolation to arbitrary points: barycentric formula of the second kind, exact at the nodes.
#include <cmath>

#include "internal.h"

namespace dg {

namespace {

// P_n(x), P_n'(x) and P_n''(x) by the Bonnet recurrence and its derivatives.
void legendre3(int n, long double x, long double& p, long double& dp, long double& d2p) {
  long double p0 = 1, p1 = x, d0 = 0, d1 = 1, s0 = 0, s1 = 0;
  if (n == 0) { p = 1; dp = 0; d2p = 0; return; }
  for (int k = 2; k <= n; ++k) {
    long double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
    long double d2 = ((2 * k - 1) * (p1 + x * d1) - (k - 1) * d0) / k;
    long double s2 = ((2 * k - 1) * (2 * d1 + x * s1) - (k - 1) * s0) / k;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2; s0 = s1; s1 = s2;
  }
  p = p1; dp = d1; d2p = s1;
}

long double lagrange_bary(int N, const long double* x, const long double* b, int j, long double t) {
  for (int m = 0; m < N; ++m)
    if (t == x[m]) return m == j ? 1.0L : 0.0L;
  long double num = 0, den = 0;
  for (int m = 0; m < N; ++m) {
    long double c = b[m] / (t - x[m]);
    den += c;
    if (m == j) num = c;
  }
  return num / den;
}

}  // namespace

LglTables make_lgl(int N) {
  DG_REQUIRE(N >= 2 && N <= DG_MAX_N, "N must be in [2, DG_MAX_N]");
  LglTables t;
  t.N = N;
  const int p = N - 1;
  const long double pi = 3.141592653589793238462643383279502884L;
  long double x[DG_MAX_N], b[DG_MAX_N];
  x[0] = -1.0L;
  x[N - 1] = 1.0L;
  for (int k = 1; k < N - 1; ++k) {
    long double xi = -cosl(pi * k / p);
    for (int it = 0; it < 100; ++it) {
      long double P, dP, d2P;
      legendre3(p, xi, P, dP, d2P);
      long double step = dP / d2P;
      xi -= step;
      if (fabsl(step) < 1e-19L) break;
    }
    x[k] = xi;
  }
  // symmetrise the point set exactly
  for (int k = 0; k < N / 2; ++k) {
    long double a = 0.5L * (x[N - 1 - k] - x[k]);
    x[k] = -a;
    x[N - 1 - k] = a;
  }
  if (N % 2) x[N / 2] = 0.0L;
  for (int k = 0; k < N; ++k) {
    long double P, dP, d2P;
    legendre3(p, x[k], P, dP, d2P);
    t.x[k] = (double)x[k];
    t.w[k] = (double)(2.0L / (N * (N - 1) * P * P));
  }
  for (int j = 0; j < N; ++j) {
    long double prod = 1;
    for (int m = 0; m < N; ++m)
      if (m != j) prod *= (x[j] - x[m]);
    b[j] = 1.0L / prod;
  }
  for (int k = 0; k < N; ++k) {
    long double diag = 0;
    for (int l = 0; l < N; ++l) {
      if (l == k) continue;
      long double v = (b[l] / b[k]) / (x[k] - x[l]);
      t.D[k * N + l] = (double)v;
      diag -= v;
    }
    t.D[k * N + k] = (double)diag;
  }
  for (int tt = 0; tt < N; ++tt) {
    long double lo = 0.5L * (x[tt] - 1.0L), hi = 0.5L * (x[tt] + 1.0L);
    for (int j = 0; j < N; ++j) {
      t.I_lo[tt * N + j] = (double)lagrange_bary(N, x, b, j, lo);
      t.I_hi[tt * N + j] = (double)lagrange_bary(N, x, b, j, hi);
    }
  }
  return t;
}

template <typename T>
OpGeom<T> make_geom(const int n[3], const double h[3], int N, double penalty, const LglTables& t, int neumann) {
  OpGeom<T> g;
  g.neumann = neumann;
  g.nx = n[0];
  g.ny = n[1];
  g.nz = n[2];
  g.J = (T)(h[0] * h[1] * h[2] / 8.0);
  for (int d = 0; d < 3; ++d) {
    g.dxi[d] = (T)(2.0 / h[d]);
    double jf = 1.0;
    for (int e = 0; e < 3; ++e)
      if (e != d) jf *= 0.5 * h[e];
    g.Jf[d] = (T)jf;
    g.sigma[d] = (T)(penalty * (double)N * (double)N / h[d]);
    g.lift[d] = (T)(1.0 / (t.w[0] * h[d]));
  }
  return g;
}

template OpGeom<double> make_geom<double>(const int*, const double*, int, double, const LglTables&, int);
template OpGeom<float> make_geom<float>(const int*, const double*, int, double, const LglTables&, int);

}  // namespace dg
