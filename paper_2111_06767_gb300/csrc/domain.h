// Domain state: geometry, multigrid hierarchy, Schwarz subdomain tables and inverses, solver
// workspace. Host-side definitions shared by the setup, solver and C-ABI translation units.
#pragma once

#include <atomic>

#include <vector_types.h>

#include "internal.h"

namespace dg {

struct SchwarzLevel {
  int nS = 0;                      // padded subdomain size N^3 + 6 N_ov N^2
  int ld = 0;                      // storage stride: nS rounded up to 32
  int n_classes = 0;               // distinct A_S (boundary-contact patterns)
  bool built = false;              // inverses built (lazily, on first smoothing)
  SubdomainGeom geom{};
  std::vector<int> class_count;    // subdomains per class
  std::vector<int> class_first;    // first subdomain column of each class
  std::vector<int> position;       // element -> subdomain column (class-sorted)
  std::vector<int> class_of;       // element -> class
  std::vector<int> patch;          // per class: 49 ints describing the representative's patch
  std::vector<int> class_key;      // per class: canonical boundary-code key
  double inv_scale = 1.0;          // stored inverses are built at unit element width: A_S^-1 = inv_scale x stored
  DevBuf<int> elem_of_col;         // subdomain column -> element
  DevBuf<int> col_of_elem;         // element -> subdomain column
  DevBuf<int> class_of_col;        // subdomain column -> class
  DevBuf<int> xform_of_elem;       // orientation index 8 perm + flips (canonical -> actual frame)
  DevBuf<double> inv64;            // [n_classes][nS][nS] explicit inverses (FP64 mode)
  DevBuf<float> inv32;             // FP32 copies (mixed mode)
  DevBuf<uint16_t> inv16;          // curved MIXED domains: per-subdomain inverses in FP16, each scaled
  DevBuf<float> inv16_scale;       //   by its largest magnitude (kept here)
  DevBuf<int4> tiles;              // SIMT GEMM tiles (class | width code << 24 | zero << 30, row0, col0,
  int n_tiles = 0;                 //   columns left): 64 rows x 64, 32 or 16 columns
  DevBuf<int> kchunks16;           // per class: [count, K chunks of 16 that meet a present slot]
  DevBuf<int> kchunks32;           // the same for chunks of 32 (tensor-core GEMM)
  std::vector<int> class_nS;       // per class: rows of the slots present (its real subdomain size)
  double alg_inv = 0, alg_vec = 0, alg_mac = 0;  // sum_c nS_c^2, sum_c E_c nS_c, sum_c E_c nS_c^2
  DevBuf<int4> tiles_tc;           // tensor-core GEMM tiles: 128 rows x 64 columns
  int n_tiles_tc = 0;
  DevBuf<int4> tiles_tc128;        // tensor-core GEMM tiles: 128 rows x 128 columns
  int n_tiles_tc128 = 0;
  DevBuf<int4> tiles_tc256;        // tensor-core GEMM tiles: 128 rows x 256 columns (one read of a
  int n_tiles_tc256 = 0;           //   128-row slab of the inverse per class of at most 256 columns)
  DevBuf<int4> units;              // fused coarse smoother GEMM units: 16 rows x all columns of a class
  int n_units = 0;
  DevBuf<unsigned> bar;            // fused coarse smoother barrier state
};

template <typename T>
struct LevelWork {
  DevBuf<T> b, u, r, rS, duS;
  // puncture subdomain GMRES (finest level only)
  DevBuf<T> gV, gZ, gW, gD, gH;
  // per-subdomain linearized inverses (finest level only): class matrices A_S at the actual
  // element widths [n_classes][nS][nS] and the inverses of A_S + D_S [E][nS][nS]
  DevBuf<T> linA, linv;
};

struct Level {
  int n[3] = {0, 0, 0};
  int E = 0;
  int64_t ndof = 0;
  double h[3] = {0, 0, 0};
  OpGeom<double> g64{};
  OpGeom<float> g32{};
  // curved elements: metric, face-node penalty, face-node normal fluxes (scratch of every apply)
  DevBuf<double> geo64, sig64, trace64;
  DevBuf<float> geo32, sig32, trace32;
  SchwarzLevel sw;
  LevelWork<double> w64;
  LevelWork<float> w32;
  // autotuned launch shapes (-1: not yet tuned): DG apply [FP64, FP32][plain, fused into r_S],
  // tensor-core GEMM split and tile width, CUDA-core GEMM split [FP32, FP64]
  int apply_variant[2][2] = {{-1, -1}, {-1, -1}};
  int gemm_split = -1;
  int simt_split[2] = {-1, -1};
};

// Event-based per-phase timing of launches (dg_profile_*).
struct Profiler {
  bool on = false;
  struct Rec {
    cudaEvent_t a, b;
    int phase;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  dg_phase_stats acc[DG_PHASE_COUNT] = {};
  // records captured into the V-cycle graph: event nodes re-recorded by every replay
  bool capturing = false;
  std::vector<Rec> graph_recs;
  dg_phase_stats graph_acc[DG_PHASE_COUNT] = {};
  cudaEvent_t get();
  void clear();
  void drop_graph_records();
  void add_graph_replay();  // after a replay has completed: accumulate its event times
  ~Profiler();
};

// Brackets one launch (or a group of launches) of a phase with events when profiling is on.
class PhaseScope {
 public:
  PhaseScope(Profiler& p, int phase, cudaStream_t s, double bytes, double flops);
  ~PhaseScope();

 private:
  Profiler& p_;
  int phase_;
  cudaStream_t s_;
  cudaEvent_t a_ = nullptr;
};

}  // namespace dg

struct dg_domain {
  dg_domain_desc desc{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  int N = 0;
  bool mixed = false;
  bool curved = false;  // per-element operators: mapped elements or a variable coefficient
  bool mapped = false;  // node coordinates given at creation (the operator is then not symmetric)
  dg::LglTables lgl;
  dg::DevBuf<double> D64, w64, Ilo64, Ihi64, x1;
  dg::DevBuf<float> D32, w32, Ilo32, Ihi32;
  std::vector<dg::Level> levels;
  dg::DevBuf<double> X, Y, Z, mass;
  dg::DevBuf<double> shares64;  // Schwarz weight shares [64 neighbour patterns][N^3][7]
  dg::DevBuf<float> shares32;
  dg::DevBuf<int> orient_map;   // [48][nS]: canonical subdomain row -> (actual slot, point)
  dg::DevBuf<int> orient_inv;   // [48][7][N^3]: (actual slot, point) -> canonical row or -1
  // puncture
  dg::DevBuf<double> alpha, beta, lin64;
  dg::DevBuf<float> lin32;
  bool lin_set = false;
  // Krylov workspace
  int kcap = 0;
  dg::DevBuf<double> V, Zb, w, r, du, ut, rt, tmp, partial, dots;
  dg::DevBuf<float> vin32;
  size_t bytes = 0;
  int subdomain_iterations = 3;
  dg::Profiler prof;
  int subdomain_solver = 0;  // linearized finest-level subdomain problems: 0 GMRES, 1 per-subdomain inverses
  const std::atomic<bool>* cancel = nullptr;  // set by a serving worker: stop between Krylov iterations
  bool linv_current = false; // per-subdomain inverses built for the current linearization
  bool use_tc = false;       // subdomain GEMM on tcgen05 tensor cores (MIXED)
  bool coarse_fused = false; // fused cooperative smoother on coarse levels (DG_COARSE_FUSED=1 turns it on)
  int barrier_stall = 0;     // DG_TEST_BARRIER_STALL=1 (read when a solve starts): the fused smoother's
                             // barriers wait for one CTA more than launched, so every wait runs out
  dg::DevBuf<int> err_flag;       // set by device code whose bounded wait gave up
  // the V-cycle replayed as one CUDA graph (fixed input/output buffers; captured on the second use)
  bool graphs = true;
  int vcycle_calls = 0;
  cudaGraphExec_t vgraph = nullptr;
  bool vgraph_lin = false;
  bool vgraph_prof = false;
  int vgraph_stall = 0;
  int64_t vgraph_kernels = 0;  // kernels in the captured graph (counted again at every replay)
  int vgraph_m = -1;
  int vgraph_sub = -1;
  dg::DevBuf<double> vin64, vout64;
  cudaStream_t gstream = nullptr;  // private stream the graph is captured on and replayed in
  cudaEvent_t gev_in = nullptr, gev_out = nullptr;
  // A whole FGMRES solve as one CUDA graph (device-resident Hessenberg/Givens, the Arnoldi loop a
  // conditional WHILE node): built when a solve with the same key has run once host-driven.
  cudaGraphExec_t sgraph = nullptr;
  std::vector<int64_t> sgraph_key, skey_seen;
  int kr_cap = 0;
  int64_t sgraph_body_kernels = 0, sgraph_fixed_kernels = 0;  // kernels per loop body / outside it
  dg::DevBuf<dg::KrylovState> kst;
  dg::DevBuf<double> kbuf;            // H, rotations, g, y, inner products, norms of the captured solve
  dg::DevBuf<double> kb, kx, zfix;    // the graph's fixed b and x, and the operator input Z_j
  cudaStream_t gstream2 = nullptr;    // second capture stream (the loop body)
  int* cancel_host = nullptr;         // mapped pinned flag the rotation kernel reads (serving cancel)
  dg::DevBuf<double> host_f, host_b, host_u;  // device copies for elliptic_solve_host
  int* cancel_dev = nullptr;
  ~dg_domain() {
    if (sgraph) cudaGraphExecDestroy(sgraph);
    if (gstream2) cudaStreamDestroy(gstream2);
    if (cancel_host) cudaFreeHost(cancel_host);
    if (vgraph) cudaGraphExecDestroy(vgraph);
    if (gev_in) cudaEventDestroy(gev_in);
    if (gev_out) cudaEventDestroy(gev_out);
    if (gstream) cudaStreamDestroy(gstream);
  }
};

namespace dg {

void domain_setup(dg_domain* dom);
dg_batch* batch_create(dg_domain* const* doms, const double* const* b, double* const* u, int count, double tol,
                       const dg_solve_opts& o);
void batch_run(dg_batch* bt, cudaStream_t s, dg_solve_report* reps);
void batch_destroy(dg_batch* bt);
void profile_read(dg_domain* dom, dg_phase_stats* out);
void ensure_schwarz(dg_domain* dom, int level);
size_t domain_device_bytes(const dg_domain* dom);

// level operators
void apply_level(dg_domain* dom, int level, const double* u, double* out, const double* b, bool with_lin,
                 cudaStream_t s, const SubdomainOut* so = nullptr);
void apply_level_f32(dg_domain* dom, int level, const float* u, float* out, const float* b, bool with_lin,
                     cudaStream_t s, const SubdomainOut* so = nullptr);
template <typename T>
void schwarz_smooth(dg_domain* dom, int level, const T* b, T* u, int iterations, bool u_is_zero, cudaStream_t s);
template <typename T>
void vcycle(dg_domain* dom, const T* r, T* z, cudaStream_t s);
void precondition(dg_domain* dom, int mode, const double* v, double* z, cudaStream_t s);

dg_status solve(dg_domain* dom, const double* b, double* u, double tol, const dg_solve_opts& o, dg_solve_report* rep);

}  // namespace dg
