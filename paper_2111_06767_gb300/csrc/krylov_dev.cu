// Device-resident flexible GMRES (Sec. III.B; Saad, Iterative Methods, Alg. 9.6): the Hessenberg
// column, its Givens rotations, the residual estimate and the stopping decision are computed on
// the GPU, so an iteration needs no host round trip and a whole solve can be one CUDA graph whose
// Arnoldi loop is a conditional WHILE node (the rotation kernel sets the loop condition).
//
// Every kernel here reads the iteration index j (and the column count m = j + 1) from the solve's
// state in device memory rather than from launch arguments, so the same captured launches serve
// every iteration: V_j and Z_j are addressed as V + j ld and Z + j ld inside the kernels. The
// reductions are the same fixed-shape two-pass trees as the host-driven solver's multi-dot
// (per-block partial sums over the same chunks, summed in the same order), so the inner products,
// and with them the Krylov basis, are the same bit for bit.
#include "internal.h"
#include "pdl.cuh"

namespace dg {

namespace {
constexpr int kThreads = 256;
inline int grid_for(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, 152 * 8));
}
}  // namespace

// r0 = ||b - A x0||, reference norm, g_0 = beta, V_0 scale; sets the loop condition.
__global__ void kr_start_kernel(KrylovState* st, double tol, int max_it, int rel_to_b, const double* __restrict__ nrm2,
                                double* __restrict__ g, cudaGraphConditionalHandle loop) {
  pdl_launch_dependents();
  pdl_wait();  // the state and vectors come from the previous kernel
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->tol = tol;
  st->max_it = max_it;
  st->rel_to_b = rel_to_b;
  const double beta = sqrt(fmax(nrm2[0], 0.0));
  const double ref = st->rel_to_b ? sqrt(fmax(nrm2[1], 0.0)) : beta;
  st->beta = beta;
  st->tol_abs = st->tol * ref;
  st->j = 0;
  st->k = 0;
  st->runs = 0;
  st->est = beta;
  g[0] = beta;
  int status = KR_RUNNING;
  if (!isfinite(beta)) status = KR_BREAKDOWN;
  else if (beta <= st->tol_abs || beta == 0.0) status = KR_CONVERGED;
  else if (st->max_it <= 0) status = KR_CAP;
  st->status = status;
  st->scale = status == KR_RUNNING ? 1.0 / beta : 0.0;
  cudaGraphSetConditional(loop, status == KR_RUNNING ? 1u : 0u);
}

// V_j = scale x while the loop runs (j and scale from the state)
__global__ void kr_scale_into_v_kernel(int64_t n, const double* __restrict__ x, const KrylovState* __restrict__ st,
                                       double* __restrict__ V, int64_t ld) {
  pdl_launch_dependents();
  pdl_wait();  // the state and vectors come from the previous kernel
  if (st->status != KR_RUNNING) return;
  const double a = st->scale;
  double* v = V + (int64_t)st->j * ld;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = a * x[i];
}

// the preconditioner's input: V_j, in FP32 (MIXED) or FP64
template <typename T>
__global__ void kr_load_v_kernel(int64_t n, const double* __restrict__ V, int64_t ld,
                                 const KrylovState* __restrict__ st, T* __restrict__ out) {
  pdl_launch_dependents();
  pdl_wait();  // the state and vectors come from the previous kernel
  const double* v = V + (int64_t)st->j * ld;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (T)v[i];
}

// Z_j = z (the flexible basis keeps every preconditioned vector) and zfix = z, the fixed input of
// the operator apply that follows
template <typename T>
__global__ void kr_store_z_kernel(int64_t n, const T* __restrict__ z, const KrylovState* __restrict__ st,
                                  double* __restrict__ Z, int64_t ld, double* __restrict__ zfix) {
  pdl_launch_dependents();
  pdl_wait();  // the state and vectors come from the previous kernel
  double* zj = Z + (int64_t)st->j * ld;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)z[i];
    zj[i] = v;
    zfix[i] = v;
  }
}

// partial[k * blocks + bx] = this block's chunk of V_k . w for k <= j: the host solver's multi-dot
// partial pass with the vector count read from the state (rows k > j of the grid exit at once)
__global__ void kr_multidot_partial_kernel(int64_t n, const double* __restrict__ V, int64_t ld,
                                           const double* __restrict__ w, const KrylovState* __restrict__ st,
                                           double* __restrict__ partial, int blocks) {
  pdl_launch_dependents();
  pdl_wait();  // the state and vectors come from the previous kernel
  const int k = blockIdx.y;
  if (k > st->j) return;
  __shared__ double red[kThreads / 32];
  const double* v = V + (int64_t)k * ld;
  const int64_t chunk = (n + blocks - 1) / blocks;
  const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  double acc = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += v[i] * w[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += red[q];
    partial[(int64_t)k * blocks + blockIdx.x] = t;
  }
}

__global__ void kr_multidot_final_kernel(const double* __restrict__ partial, const KrylovState* __restrict__ st,
                                         double* __restrict__ out, int blocks) {
  pdl_launch_dependents();
  pdl_wait();  // the state and vectors come from the previous kernel
  const int k = blockIdx.x;
  if (k > st->j) return;
  __shared__ double red[kThreads / 32];
  double acc = 0.0;
  for (int q = threadIdx.x; q < blocks; q += blockDim.x) acc += partial[(int64_t)k * blocks + q];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += red[q];
    out[k] = t;
  }
}

// w -= sum_{k <= j} h[k] V_k
__global__ void kr_sub_comb_kernel(int64_t n, const double* __restrict__ V, int64_t ld, const double* __restrict__ h,
                                   const KrylovState* __restrict__ st, double* __restrict__ w) {
  pdl_launch_dependents();
  pdl_wait();  // the state and vectors come from the previous kernel
  const int m = st->j + 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = w[i];
    for (int k = 0; k < m; ++k) acc -= h[k] * V[(int64_t)k * ld + i];
    w[i] = acc;
  }
}

// Column j of the Hessenberg matrix from the two Gram-Schmidt passes, the previous rotations
// applied to it, the new rotation, the residual estimate |g_{j+1}| and the stopping decision; while
// the loop continues, the scale 1 / h_{j+1,j} of the next basis vector and j + 1. One thread.
__global__ void kr_givens_kernel(KrylovState* st, double* __restrict__ H, int ldh, double* __restrict__ cs,
                                 double* __restrict__ sn, double* __restrict__ g, const double* __restrict__ h1,
                                 const double* __restrict__ h2, const double* __restrict__ nrm2,
                                 const volatile int* cancel, cudaGraphConditionalHandle loop) {
  pdl_launch_dependents();
  pdl_wait();  // the state and vectors come from the previous kernel
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (st->status != KR_RUNNING) {
    cudaGraphSetConditional(loop, 0u);
    return;
  }
  const int j = st->j;
  st->runs = j + 1;
  double* col = H + (int64_t)j * ldh;
  for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
  const double hn = sqrt(fmax(0.0, nrm2[0]));
  col[j + 1] = hn;
  for (int i = 0; i < j; ++i) {  // previous rotations
    const double a = col[i], c = col[i + 1];
    col[i] = cs[i] * a + sn[i] * c;
    col[i + 1] = -sn[i] * a + cs[i] * c;
  }
  const double den = hypot(col[j], col[j + 1]);
  int status = KR_RUNNING;
  if (den == 0.0 || !isfinite(den)) {
    status = KR_BREAKDOWN;  // column j is unusable: the update keeps the k = j columns before it
  } else {
    cs[j] = col[j] / den;
    sn[j] = col[j + 1] / den;
    col[j] = den;
    col[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    st->k = j + 1;
    const double est = fabs(g[j + 1]);
    st->est = est;
    if (!isfinite(est)) status = KR_BREAKDOWN;
    else if (est <= st->tol_abs || hn == 0.0) status = KR_CONVERGED;
    else if (j + 1 >= st->max_it) status = KR_CAP;
    else if (cancel && *cancel) status = KR_CANCELLED;
  }
  st->status = status;
  if (status == KR_RUNNING) {
    st->scale = 1.0 / hn;
    st->j = j + 1;
  }
  cudaGraphSetConditional(loop, status == KR_RUNNING ? 1u : 0u);
}

// y = R^-1 g over the k completed columns (back substitution). One thread.
__global__ void kr_trisolve_kernel(const KrylovState* __restrict__ st, const double* __restrict__ H, int ldh,
                                   const double* __restrict__ g, double* __restrict__ y) {
  pdl_launch_dependents();
  pdl_wait();  // the state and vectors come from the previous kernel
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k = st->k;
  for (int i = k - 1; i >= 0; --i) {
    double acc = g[i];
    for (int l = i + 1; l < k; ++l) acc -= H[(int64_t)l * ldh + i] * y[l];
    y[i] = acc / H[(int64_t)i * ldh + i];
  }
}

// x += sum_{l < k} y[l] Z_l
__global__ void kr_add_comb_kernel(int64_t n, const double* __restrict__ Z, int64_t ld, const double* __restrict__ y,
                                   const KrylovState* __restrict__ st, double* __restrict__ x) {
  pdl_launch_dependents();
  pdl_wait();  // the state and vectors come from the previous kernel
  const int m = st->k;
  if (m == 0) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = x[i];
    for (int l = 0; l < m; ++l) acc += y[l] * Z[(int64_t)l * ld + i];
    x[i] = acc;
  }
}

// ------------------------------------------------------------------ launchers
//
// Every kernel above waits for its predecessor (griddepcontrol.wait) before touching the state or
// the vectors, so they can be launched with programmatic dependent launch (DG_PDL_KRYLOV=1; off by
// default, see pdl_krylov_enabled).

void launch_kr_start(KrylovState* st, double tol, int max_it, bool rel_to_b, const double* nrm2, double* g,
                     cudaGraphConditionalHandle loop, cudaStream_t s) {
  const PdlScope pdl(pdl_krylov_enabled());
  launch_pdl(kr_start_kernel, dim3(1), dim3(32), 0, s, st, tol, max_it, rel_to_b ? 1 : 0, nrm2, g, loop);
  DG_LAUNCHED(1);
}

// The outcome of one captured solve as 8 doubles: completed columns, status, loop bodies run,
// ||b - A x0||, the reference norm, the final ||b - A x||, the stopping threshold.
__global__ void kr_report_kernel(const KrylovState* __restrict__ st, const double* __restrict__ nrm2,
                                 double* __restrict__ out) {
  pdl_launch_dependents();
  pdl_wait();  // the state and vectors come from the previous kernel
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  out[0] = st->k;
  out[1] = st->status;
  out[2] = st->runs;
  out[3] = st->beta;
  out[4] = st->rel_to_b ? sqrt(fmax(nrm2[1], 0.0)) : st->beta;
  out[5] = sqrt(fmax(nrm2[2], 0.0));
  out[6] = st->tol_abs;
  out[7] = 0.0;
}
void launch_kr_report(const KrylovState* st, const double* nrm2, double* out, cudaStream_t s) {
  const PdlScope pdl(pdl_krylov_enabled());
  launch_pdl(kr_report_kernel, dim3(1), dim3(32), 0, s, st, nrm2, out);
  DG_LAUNCHED(1);
}
void launch_kr_scale_into_v(int64_t n, const double* x, const KrylovState* st, double* V, int64_t ld, cudaStream_t s) {
  const PdlScope pdl(pdl_krylov_enabled());
  launch_pdl(kr_scale_into_v_kernel, dim3(grid_for(n)), dim3(kThreads), 0, s, n, x, st, V, ld);
  DG_LAUNCHED(1);
}
template <typename T>
void launch_kr_load_v(int64_t n, const double* V, int64_t ld, const KrylovState* st, T* out, cudaStream_t s) {
  const PdlScope pdl(pdl_krylov_enabled());
  launch_pdl(kr_load_v_kernel<T>, dim3(grid_for(n)), dim3(kThreads), 0, s, n, V, ld, st, out);
  DG_LAUNCHED(1);
}
template void launch_kr_load_v<float>(int64_t, const double*, int64_t, const KrylovState*, float*, cudaStream_t);
template void launch_kr_load_v<double>(int64_t, const double*, int64_t, const KrylovState*, double*, cudaStream_t);
template <typename T>
void launch_kr_store_z(int64_t n, const T* z, const KrylovState* st, double* Z, int64_t ld, double* zfix,
                       cudaStream_t s) {
  const PdlScope pdl(pdl_krylov_enabled());
  launch_pdl(kr_store_z_kernel<T>, dim3(grid_for(n)), dim3(kThreads), 0, s, n, z, st, Z, ld, zfix);
  DG_LAUNCHED(1);
}
template void launch_kr_store_z<float>(int64_t, const float*, const KrylovState*, double*, int64_t, double*,
                                       cudaStream_t);
template void launch_kr_store_z<double>(int64_t, const double*, const KrylovState*, double*, int64_t, double*,
                                        cudaStream_t);
void launch_kr_multidot(int64_t n, int cap, const double* V, int64_t ld, const double* w, const KrylovState* st,
                        double* partial, double* out, cudaStream_t s) {
  const PdlScope pdl(pdl_krylov_enabled());
  const int blocks = multidot_partial_blocks();
  launch_pdl(kr_multidot_partial_kernel, dim3(blocks, cap), dim3(kThreads), 0, s, n, V, ld, w, st, partial,
             blocks);
  launch_pdl(kr_multidot_final_kernel, dim3(cap), dim3(kThreads), 0, s, partial, st, out, blocks);
  DG_LAUNCHED(2);
}
void launch_kr_sub_comb(int64_t n, const double* V, int64_t ld, const double* h, const KrylovState* st, double* w,
                        cudaStream_t s) {
  const PdlScope pdl(pdl_krylov_enabled());
  launch_pdl(kr_sub_comb_kernel, dim3(grid_for(n)), dim3(kThreads), 0, s, n, V, ld, h, st, w);
  DG_LAUNCHED(1);
}
void launch_kr_givens(KrylovState* st, double* H, int ldh, double* cs, double* sn, double* g, const double* h1,
                      const double* h2, const double* nrm2, const volatile int* cancel,
                      cudaGraphConditionalHandle loop, cudaStream_t s) {
  const PdlScope pdl(pdl_krylov_enabled());
  launch_pdl(kr_givens_kernel, dim3(1), dim3(32), 0, s, st, H, ldh, cs, sn, g, h1, h2, nrm2, cancel, loop);
  DG_LAUNCHED(1);
}
void launch_kr_trisolve(const KrylovState* st, const double* H, int ldh, const double* g, double* y, cudaStream_t s) {
  const PdlScope pdl(pdl_krylov_enabled());
  launch_pdl(kr_trisolve_kernel, dim3(1), dim3(32), 0, s, st, H, ldh, g, y);
  DG_LAUNCHED(1);
}
void launch_kr_add_comb(int64_t n, const double* Z, int64_t ld, const double* y, const KrylovState* st, double* x,
                        cudaStream_t s) {
  const PdlScope pdl(pdl_krylov_enabled());
  launch_pdl(kr_add_comb_kernel, dim3(grid_for(n)), dim3(kThreads), 0, s, n, Z, ld, y, st, x);
  DG_LAUNCHED(1);
}

}  // namespace dg
