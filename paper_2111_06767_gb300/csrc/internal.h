// Internal declarations of the GB300 DG elliptic library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <functional>
#include <memory>
#include <string>
#include <vector>

#include "../../include/dg_elliptic.h"

namespace dg {

// ------------------------------------------------------------------ errors

struct Error {
  dg_status status;
  std::string message;
};

// Throwing is confined to host setup/orchestration code; every extern "C" entry point catches
// and converts to a dg_status, so nothing escapes the ABI.
[[noreturn]] void fail(dg_status st, const std::string& msg);
void cuda_check(cudaError_t e, const char* what, const char* file, int line);
#define DG_CUDA(x) ::dg::cuda_check((x), #x, __FILE__, __LINE__)
// Counts kernels this library launched (process-wide) and checks the launch.
void count_launches(int64_t k);
int64_t launches_total();
#define DG_LAUNCHED(k)                      \
  do {                                      \
    ::dg::count_launches(k);                \
    DG_CUDA(cudaGetLastError());            \
  } while (0)
// Message of the latest call on this thread that had no domain handle (dg_domain_create that
// failed, dg_dot_noalloc); dg_last_error(NULL) returns it.
void set_null_handle_error(const std::string& msg);
const char* null_handle_error();
#define DG_REQUIRE(cond, msg)                                  \
  do {                                                         \
    if (!(cond)) ::dg::fail(DG_ERR_INVALID_ARG, (msg));        \
  } while (0)

// ------------------------------------------------------------------ device memory

// Stream on which this thread's library allocations are made: the domain's stream while an entry
// point runs (set by AllocStreamScope), else the legacy default stream. Allocation and release are
// stream-ordered (cudaMallocAsync / cudaFreeAsync), so one domain's set-up or teardown does not
// wait for the work of domains on other streams, as cudaMalloc / cudaFree would.
cudaStream_t alloc_stream();
// Programmatic dependent launch for the launches made on this thread while a scope with on = true
// is alive (pdl_enabled() in pdl.cuh); pdl_vcycle_mode(): which FP32 V-cycle launches open one
// (DG_PDL_COARSE: 0 none, 1 the coarse levels' smoothing, 2 every level and the transfers, 3 the
// coarse levels and the fine level's scatter).
struct PdlScope {
  bool on;
  explicit PdlScope(bool on_);
  ~PdlScope();
  PdlScope(const PdlScope&) = delete;
  PdlScope& operator=(const PdlScope&) = delete;
};
int pdl_vcycle_mode();
bool pdl_krylov_enabled();  // the device-resident FGMRES kernels (DG_PDL_KRYLOV=1 turns it on)

struct AllocStreamScope {
  cudaStream_t prev;
  explicit AllocStreamScope(cudaStream_t s);
  ~AllocStreamScope();
};
// Keep freed memory in this process's default pool of the current device (once per device).
void keep_pool_memory();

// Owning device buffer, move-only. alloc() returns once the memory is usable from any stream
// (it synchronises the allocation stream); release() is ordered after that stream's work, and
// the owner makes sure other streams are done with the buffer before (the domain joins its
// private stream into its main stream after every use).
template <typename T>
struct DevBuf {
  T* ptr = nullptr;
  size_t count = 0;
  cudaStream_t st = nullptr;
  DevBuf() = default;
  explicit DevBuf(size_t n) { alloc(n); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : ptr(o.ptr), count(o.count), st(o.st) { o.ptr = nullptr; o.count = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); ptr = o.ptr; count = o.count; st = o.st; o.ptr = nullptr; o.count = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  void alloc(size_t n);
  void release() {
    if (ptr) cudaFreeAsync(ptr, st);
    ptr = nullptr;
    count = 0;
  }
  size_t bytes() const { return count * sizeof(T); }
  T* get() const { return ptr; }
};

template <typename T>
void DevBuf<T>::alloc(size_t n) {
  release();
  if (n == 0) return;
  st = alloc_stream();
  cudaError_t e = cudaMallocAsync(&ptr, n * sizeof(T), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    if (ptr) cudaFreeAsync(ptr, st);
    ptr = nullptr;
    (void)cudaGetLastError();
    fail(DG_ERR_OOM, "allocation of " + std::to_string(n * sizeof(T)) + " bytes failed: " + cudaGetErrorString(e));
  }
  count = n;
}

// ------------------------------------------------------------------ LGL tables (host)

struct LglTables {
  int N = 0;
  double x[DG_MAX_N] = {};
  double w[DG_MAX_N] = {};
  double D[DG_MAX_N * DG_MAX_N] = {};        // D[k*N + l] = l_l'(x_k)
  double I_lo[DG_MAX_N * DG_MAX_N] = {};     // child on the lower half: l_j((x_t - 1)/2), [t*N + j]
  double I_hi[DG_MAX_N * DG_MAX_N] = {};     // upper half: l_j((x_t + 1)/2)
};
LglTables make_lgl(int N);
// Dhat and the LGL weights of every N in constant memory, uploaded once per device.
void upload_operator_tables();

// ------------------------------------------------------------------ operator geometry

// Everything an element apply needs besides the data; uniform affine elements per level.
template <typename T>
struct OpGeom {
  int nx, ny, nz;
  T dxi[3];      // 2 / h_d : d xi / d x
  T J;           // volume Jacobian h_x h_y h_z / 8
  T Jf[3];       // face Jacobian of faces normal to d: product of the tangential h/2
  T sigma[3];    // penalty C N^2 / h_d (Eq. penalty, equal neighbours)
  T lift[3];     // 1 / (w_0 h_d): L = M^-1 ML at a face node is 2 lift[d]
  int neumann;   // bit f: box face f (= 2 d + side) is homogeneous Neumann, else Dirichlet
};

template <typename T>
OpGeom<T> make_geom(const int n[3], const double h[3], int N, double penalty, const LglTables& t, int neumann = 0);

// ------------------------------------------------------------------ kernels (launchers)

// Optional destination of the apply: instead of `out`, write every result point into the subdomain
// vectors that contain it (rows from the orientation point maps), i.e. the Schwarz gather fused
// into the residual computation.
struct SubdomainOut {
  void* rS = nullptr;            // T*: [columns][ld]
  int ld = 0;
  int ov = 0;                    // N_overlap
  const int* col_of_elem = nullptr;
  const int* orient = nullptr;   // orientation index per element
  const int* inv = nullptr;      // [48][7][N^3] canonical row or -1
};

// Everything one DG apply reads and writes (rS != nullptr: write into the subdomain vectors).
template <typename T>
struct ApplyArgs {
  OpGeom<T> g;
  const T* D;
  const T* w;
  const T* u;
  const T* diag;
  const T* b;
  T* out;
  int E;
  T* rS;
  int ld, ov;
  const int* col_of_elem;
  const int* orient;
  const int* inv;
};

// out = A u (+ diag * u)  or, with b != nullptr, out = b - (A u + diag * u). variant: launch shape
// (0 chosen by grid size, 1..3 few / middle / many elements per CTA; FP32 only: 4 the N = 4
// slice-per-thread kernel, 5 and 6 the block-of-lines kernel, 7 the N = 4 element-per-thread kernel,
// whose bounded staging wait raises *err if it gives up; a variant that cannot serve the call runs
// as 0).
template <typename T>
void launch_apply(int N, const OpGeom<T>& g, const T* D, const T* w, const T* u, const T* diag, const T* b, T* out,
                  cudaStream_t s, const SubdomainOut* so = nullptr, int variant = 0, int* err = nullptr);
constexpr int kApplyVariants = 3;

// Build explicit subdomain matrices A_S for a set of classes (column-major == row-major by symmetry).
template <typename T>
void launch_build_subdomain_matrices(int N, int overlap, const OpGeom<T>& g, const T* D, const T* w,
                                     const int* d_patch_info, int n_classes, int nS, T* A_out, cudaStream_t s);
// In-place Gauss-Jordan inversion of n_classes SPD matrices of size n (no pivoting).
template <typename T>
void launch_invert_spd_batched(T* A, int n, int n_classes, cudaStream_t s);

// Schwarz data movement. Subdomain columns are class-sorted; rows follow the subdomain point order.
struct SubdomainGeom {
  int n[3];
  int E, N, ov, nS;
  int ld;  // column stride of subdomain vectors and row stride of inverses: nS rounded up to 32
};
template <typename T>
void launch_gather_tab(const SubdomainGeom& g, const T* r, const int* elem_of_col, const int* orient, const int* map,
                       T* rS, cudaStream_t s);
template <typename T, typename TU>
void launch_scatter_tab(const SubdomainGeom& g, const T* duS, const int* col_of_elem, const int* orient,
                        const int* inv, const T* shares, TU* u, cudaStream_t s);
template <typename S, typename T>
void launch_pad_convert(const S* src, int n, int ld, int n_classes, T* dst, cudaStream_t s);

// Fused coarse-level smoother (FP32): `iterations` Schwarz steps on one level in a single
// cooperative launch, the phases (residual into r_S, subdomain solves, weighted scatter) separated
// by grid-wide barriers.
struct CoarseArgs {
  ApplyArgs<float> ap;       // residual r = b - A u written into r_S (ap.rS)
  SubdomainGeom sg;
  const int* elem_of_col;    // gather of the first step when u = 0
  const int* map;
  const float* shares;       // scatter weights
  float* duS;
  const float* invm;         // class inverses [class][ld][ld] (unit width)
  float alpha;               // 1 / h_x
  const int4* units;         // (class, first of 16 rows, first column, columns) per GEMM work unit
  int n_units;
  unsigned* bar;             // barrier state (arrivals, generation), zeroed before the launch
  int* err;                  // set if a barrier wait gave up
  int iterations;
  int u_zero;                // first step gathers b (u = 0)
  int stall;                 // extra arrivals every barrier waits for: 0, or 1 to make every wait run out
                             // (the generation flag is then never advanced; the timeout test's switch)
};
bool coarse_smooth_available(int N);
void launch_coarse_smooth(int N, const CoarseArgs& a, cudaStream_t s);

// Tensor-core (tcgen05, TF32) class GEMM; Y columns of ld values, n_cols columns in X and Y.
bool tc_gemm_available();
// split: K split across a cluster of 1, 2, 4 or 8 CTAs; 0 picks it from the tile count. bn: tile
// width, 64 or 256 (d_tiles must list tiles of that width). d_kchunks: per class [count, indices of
// the 32-wide K chunks that meet a present slot], ld / 32 + 1 ints per class.
void launch_class_gemm_tc(const float* inv, int n_classes, const float* X, float* Y, int ld, int n_cols,
                          const int4* d_tiles, int n_tiles, const int* d_kchunks, int* err, float alpha,
                          cudaStream_t s, int split = 0, int bn = 64);
// Splits the tensor-core GEMM accepts for this shape (each CTA keeps >= 4 K chunks).
std::vector<int> tc_gemm_splits(int ld);

// Launch-shape autotuning: the first time a kernel shape (key) is seen in the process, time each
// candidate (run(c) launches it once on stream s) and keep the fastest; later calls return the
// kept choice. candidates[0] is the heuristic default, used alone when DG_AUTOTUNE=0 or while s is
// being captured into a graph.
bool tune_log();  // DG_TUNE_LOG=1
int autotune(const std::vector<int64_t>& key, const std::vector<int>& candidates,
             const std::function<void(int)>& run, cudaStream_t s);

// Subdomain GMRES for linearized problems (columns of n_S values, E columns per basis vector).
template <typename T>
void launch_sub_normalize(int E, int nS, const T* rS, T* V0, T* beta, cudaStream_t s);
template <typename T>
void launch_sub_arnoldi(int E, int nS, int j, int m, const T* D, T* V, const T* Z, T* H, cudaStream_t s);
template <typename T>
void launch_sub_lsq_combine(int E, int nS, int m, const T* beta, const T* H, const T* Z, T* duS, cudaStream_t s);

// Curved (mapped) elements and variable coefficients: metric [11][ndof] (J, then G^j_i = dxi^j/dx^i
// at 1 + 3 j + i, then the coefficient K at 10), penalty
// at every face node [E][6][N^2], outward normal fluxes of u at every face node [E][6][N^2].
template <typename T>
struct CurvedArgs {
  int n[3];
  int neumann;
  int64_t ndof;
  const T* geo;
  const T* sigma;
  const T* D;
  const T* w;
  const T* u;
  const T* b;
  T* out;
  T* trace;
};
// out = A u (or b - A u): the trace pass, then the operator pass.
template <typename T>
void launch_curved_apply(int N, const CurvedArgs<T>& a, int E, cudaStream_t s);
// Row-major subdomain matrices A_S of subdomains e0 .. e0 + count - 1 into A_out.
template <typename T>
void launch_curved_columns(int N, const CurvedArgs<T>& a, int ov, int nS, int e0, int count, T* A_out,
                           cudaStream_t s);
void launch_curved_metric(int N, int64_t E, const double* xyz, const double* D, double* geo64, float* geo32, int* bad,
                          cudaStream_t s);
void launch_curved_sigma(int N, const int n[3], double penalty, const double* geo64, double* sig64, float* sig32,
                         cudaStream_t s);
void launch_curved_coarsen(int N, const int cn[3], const int fn[3], const double* C, const double* fine_xyz,
                           double* coarse_xyz, cudaStream_t s);
void launch_curved_mass(int N, const double* w, const double* geo64, int64_t ndof, double* mass, cudaStream_t s);

// Per-subdomain linearized inverses (finest level of a linearized problem): assemble
// M_c = A_{class(c)} + diag(d_S[:, c]) (compact n_S x n_S per column), then du_S = Minv_c r_S.
template <typename T>
void launch_lin_assemble(const T* A, const int* class_of_col, const T* dS, int nS, int ld, int E, T* M,
                         cudaStream_t s);
template <typename T>
void launch_lin_gemv(const T* Minv, const T* rS, int nS, int ld, int E, T* duS, cudaStream_t s);
// FP16 copies of E compact n_S x n_S FP32 matrices, each scaled by its largest magnitude (scale[c]),
// and du_S = scale Minv16 r_S with FP32 vectors and sums.
void launch_to_half_scaled(const float* src, int nS, int E, uint16_t* dst, float* scale, cudaStream_t s);
void launch_lin_gemv_half(const uint16_t* Minv, const float* scale, const float* rS, int nS, int ld, int E,
                          float* duS, cudaStream_t s);

// Multigrid transfers (per dimension: 0 lower half, 1 upper half, 2 full).
template <typename T>
void launch_prolongate_add(int N, const int nf[3], const int nc[3], const T* Ilo, const T* Ihi, const T* uc, T* uf,
                           cudaStream_t s);
template <typename T>
void launch_restrict(int N, const int nf[3], const int nc[3], const T* Ilo, const T* Ihi, const T* rf, T* bc,
                     cudaStream_t s);

// Vector kernels.
template <typename T>
void launch_axpby(int64_t n, T a, const T* x, T b, T* y, cudaStream_t s);  // y = a x + b y
template <typename T>
void launch_fill(int64_t n, T v, T* y, cudaStream_t s);  // y = v
void launch_convert_d2f(int64_t n, const double* x, float* y, cudaStream_t s);
void launch_convert_f2d(int64_t n, const float* x, double* y, cudaStream_t s);
void launch_add_f2d(int64_t n, const float* x, double* y, cudaStream_t s);  // y += x
void launch_scale_mul(int64_t n, const double* a, const double* b, double* y, cudaStream_t s);  // y = a .* b
// Deterministic multi-dot: out[k] = sum_i V[k*ld + i] * w[i] for k < m (two-pass reduction).
void launch_multidot(int64_t n, int m, const double* V, int64_t ld, const double* w, double* partial, double* out,
                     cudaStream_t s);
// w -= sum_k h[k] V[k*ld + i]
void launch_subtract_combination(int64_t n, int m, const double* V, int64_t ld, const double* h, double* w,
                                 cudaStream_t s);
// x += sum_k y[k] Z[k*ld + i]
void launch_add_combination(int64_t n, int m, const double* Z, int64_t ld, const double* y, double* x, cudaStream_t s);
int multidot_partial_blocks();

// Device-resident flexible GMRES (krylov_dev.cu): the state of one solve, in device memory.
enum { KR_RUNNING = 0, KR_CONVERGED = 1, KR_BREAKDOWN = 2, KR_CAP = 3, KR_CANCELLED = 4 };
struct KrylovState {
  int j;           // column the running iteration computes (V_j, Z_j)
  int k;           // completed columns
  int status;      // KR_*
  int max_it;      // columns allowed (input)
  int rel_to_b;    // tolerance relative to ||b|| (input) instead of ||b - A x0||
  int runs;        // loop bodies executed (Arnoldi iterations attempted)
  double tol;      // relative tolerance (input)
  double tol_abs;  // absolute threshold on the residual estimate
  double beta;     // ||b - A x0||
  double scale;    // factor of the next basis vector: 1 / beta, then 1 / h_{j+1,j}
  double est;      // latest residual estimate |g_k|
};
void launch_kr_start(KrylovState* st, double tol, int max_it, bool rel_to_b, const double* nrm2, double* g,
                     cudaGraphConditionalHandle loop, cudaStream_t s);
void launch_kr_report(const KrylovState* st, const double* nrm2, double* out, cudaStream_t s);
void launch_kr_scale_into_v(int64_t n, const double* x, const KrylovState* st, double* V, int64_t ld, cudaStream_t s);
template <typename T>
void launch_kr_load_v(int64_t n, const double* V, int64_t ld, const KrylovState* st, T* out, cudaStream_t s);
template <typename T>
void launch_kr_store_z(int64_t n, const T* z, const KrylovState* st, double* Z, int64_t ld, double* zfix,
                       cudaStream_t s);
void launch_kr_multidot(int64_t n, int cap, const double* V, int64_t ld, const double* w, const KrylovState* st,
                        double* partial, double* out, cudaStream_t s);
void launch_kr_sub_comb(int64_t n, const double* V, int64_t ld, const double* h, const KrylovState* st, double* w,
                        cudaStream_t s);
void launch_kr_givens(KrylovState* st, double* H, int ldh, double* cs, double* sn, double* g, const double* h1,
                      const double* h2, const double* nrm2, const volatile int* cancel,
                      cudaGraphConditionalHandle loop, cudaStream_t s);
void launch_kr_trisolve(const KrylovState* st, const double* H, int ldh, const double* g, double* y, cudaStream_t s);
void launch_kr_add_comb(int64_t n, const double* Z, int64_t ld, const double* y, const KrylovState* st, double* x,
                        cudaStream_t s);

// Puncture source terms.
void launch_puncture_fields(int64_t n, const double* x, const double* y, const double* z, int np,
                            const dg_puncture* p, double* alpha, double* beta, cudaStream_t s);
// r = b - (Au + M S(u)) where Au is given; lin = M S'(u)
void launch_puncture_residual(int64_t n, const double* Au, const double* u, const double* b, const double* mass,
                              const double* alpha, const double* beta, double* r, cudaStream_t s);
void launch_puncture_linearization(int64_t n, const double* u, const double* mass, const double* alpha,
                                   const double* beta, double* lin64, float* lin32, cudaStream_t s);
template <typename T>
void launch_mass_diag(int N, const OpGeom<T>& g, const T* w, int64_t ndof, T* mass, cudaStream_t s);
void launch_node_coords(int N, const int n[3], const double lower[3], const double h[3], const double* x1,
                        double* X, double* Y, double* Z, cudaStream_t s);

}  // namespace dg
