// Puncture-method source terms (Sec. V lists puncture problems among those the solver handles;
// the paper gives no formulas, so this is the textbook Brandt-Bruegmann form):
//   1/alpha = sum_n m_n / (2 r_n),
//   A^ij    = sum_n 3/(2 r_n^2) [P^i l^j + P^j l^i - (delta^ij - l^i l^j) P.l],  l = (x - C_n) / r_n,
//   beta    = alpha^7 A_ij A^ij / 8,
//   S(u)    = -beta (1 + alpha (1 + u))^-7,   S'(u) = 7 alpha beta (1 + alpha (1 + u))^-8.
// The nonlinear operator is A(u) = A_Delta u + M S(u) (massive form), linearized as
// A_Delta + M diag(S'(u)) (Eq. linearized).
#include "internal.h"

namespace dg {

struct PunctureSet {
  int n;
  dg_puncture p[DG_MAX_PUNCTURES];
};

__global__ void puncture_fields_kernel(int64_t n, const double* __restrict__ X, const double* __restrict__ Y,
                                       const double* __restrict__ Z, PunctureSet ps, double* __restrict__ alpha,
                                       double* __restrict__ beta) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const double x[3] = {X[t], Y[t], Z[t]};
    double inv_alpha = 0.0;
    double A[3][3] = {};
    for (int q = 0; q < ps.n; ++q) {
      double l[3], r2 = 0.0;
      for (int d = 0; d < 3; ++d) {
        l[d] = x[d] - ps.p[q].position[d];
        r2 += l[d] * l[d];
      }
      const double r = sqrt(r2);
      for (int d = 0; d < 3; ++d) l[d] /= r;
      inv_alpha += ps.p[q].mass / (2.0 * r);
      const double* P = ps.p[q].momentum;
      const double Pl = P[0] * l[0] + P[1] * l[1] + P[2] * l[2];
      const double c = 1.5 / r2;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
          A[a][b] += c * (P[a] * l[b] + P[b] * l[a] - ((a == b ? 1.0 : 0.0) - l[a] * l[b]) * Pl);
    }
    double AA = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) AA += A[a][b] * A[a][b];
    const double al = 1.0 / inv_alpha;
    const double a2 = al * al, a4 = a2 * a2;
    alpha[t] = al;
    beta[t] = a4 * a2 * al * AA * 0.125;
  }
}

void launch_puncture_fields(int64_t n, const double* x, const double* y, const double* z, int np, const dg_puncture* p,
                            double* alpha, double* beta, cudaStream_t s) {
  PunctureSet ps;
  ps.n = np;
  for (int q = 0; q < np; ++q) ps.p[q] = p[q];
  puncture_fields_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, s>>>(n, x, y, z, ps, alpha,
                                                                                               beta);
  DG_LAUNCHED(1);
}

__global__ void puncture_residual_kernel(int64_t n, const double* __restrict__ Au, const double* __restrict__ u,
                                         const double* __restrict__ b, const double* __restrict__ mass,
                                         const double* __restrict__ alpha, const double* __restrict__ beta,
                                         double* __restrict__ r) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const double psi = 1.0 + alpha[t] * (1.0 + u[t]);
    const double p2 = psi * psi, p4 = p2 * p2;
    const double S = -beta[t] / (p4 * p2 * psi);
    r[t] = (b ? b[t] : 0.0) - (Au[t] + mass[t] * S);
  }
}

void launch_puncture_residual(int64_t n, const double* Au, const double* u, const double* b, const double* mass,
                              const double* alpha, const double* beta, double* r, cudaStream_t s) {
  puncture_residual_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, s>>>(n, Au, u, b, mass,
                                                                                                 alpha, beta, r);
  DG_LAUNCHED(1);
}

__global__ void puncture_lin_kernel(int64_t n, const double* __restrict__ u, const double* __restrict__ mass,
                                    const double* __restrict__ alpha, const double* __restrict__ beta,
                                    double* __restrict__ lin64, float* __restrict__ lin32) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const double psi = 1.0 + alpha[t] * (1.0 + u[t]);
    const double p2 = psi * psi, p4 = p2 * p2;
    const double dS = 7.0 * alpha[t] * beta[t] / (p4 * p4);
    const double v = mass[t] * dS;
    lin64[t] = v;
    if (lin32) lin32[t] = (float)v;
  }
}

void launch_puncture_linearization(int64_t n, const double* u, const double* mass, const double* alpha,
                                   const double* beta, double* lin64, float* lin32, cudaStream_t s) {
  puncture_lin_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, s>>>(n, u, mass, alpha, beta,
                                                                                            lin64, lin32);
  DG_LAUNCHED(1);
}

}  // namespace dg
