/*
 * dg_elliptic.h - C ABI of the GB300 DG multigrid-Schwarz elliptic solver.
 *
 * The library solves the DG-discretized elliptic problem  A u = b  (Sec. II, Eq. matrix_eq)
 * of arXiv 2111.06767 with flexible GMRES (Sec. III.B) preconditioned by one geometric
 * multigrid V-cycle per iteration (Sec. III.C) whose smoother is the additive Schwarz method
 * with element-centred overlapping subdomains (Sec. III.D) and explicit subdomain inverses
 * (Sec. III.E). Nonlinear problems A(u) = b are solved by Newton-Raphson with a line search
 * (Sec. III.A, Eq. linearized). Only the matrix-vector product A u is ever formed (Sec. II).
 *
 * Conventions shared by every call:
 *  - Pointers named u, b, r, f, Au, z are DEVICE pointers to FP64 (or FP32 where the name says
 *    so) nodal vectors of n_dof entries, owned by the caller, laid out element-major:
 *    element e = ex + n[0] * (ey + n[1] * ez), and inside an element node (k, j, i) at offset
 *    (k * N + j) * N + i, i along x fastest. Nodes are the N Legendre-Gauss-Lobatto points per
 *    dimension of each affine element (Sec. II, Eq. field_expansion).
 *  - `stream` is a cudaStream_t passed as void*; NULL means the domain's stream, which is the
 *    stream given to dg_domain_create (NULL there: the legacy default stream). Calls are
 *    asynchronous on that stream unless stated otherwise.
 *  - Every call returns a dg_status; none aborts or traps. On failure the per-handle message
 *    dg_last_error() says why. A failed CUDA call leaves the handle usable only for destroy.
 *  - One domain is used from one host thread at a time; server calls are thread-safe.
 */
#ifndef DG_ELLIPTIC_H
#define DG_ELLIPTIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dg_status {
  DG_OK = 0,
  DG_PENDING = 1,             /* served request still running */
  DG_ERR_INVALID_ARG = -1,    /* bad descriptor, size, pointer or level */
  DG_ERR_OOM = -2,            /* device or host allocation failed */
  DG_ERR_CUDA = -3,           /* a CUDA runtime call failed */
  DG_ERR_NOT_CONVERGED = -4,  /* iteration limit reached before the tolerance */
  DG_ERR_BREAKDOWN = -5,      /* non-finite residual or Krylov breakdown without convergence */
  DG_ERR_TIMEOUT = -6,        /* a bounded device wait gave up */
  DG_ERR_BUSY = -7,           /* serving queue full: retry later */
  DG_ERR_NOT_FOUND = -8,      /* unknown serving ticket */
  DG_ERR_CANCELLED = -9       /* served request cancelled before it finished */
} dg_status;

enum { DG_MAX_N = 10, DG_MAX_LEVELS = 8, DG_MAX_PUNCTURES = 4 };

enum dg_precision {
  DG_PRECISION_FP64 = 0,  /* every operation in FP64 */
  DG_PRECISION_MIXED = 1  /* V-cycle (smoother, subdomain inverses, transfers) in FP32 under FP64 FGMRES */
};

enum dg_problem {
  DG_PROBLEM_POISSON = 0,  /* -Laplace u = f, Eq. poisson_fluxform */
  DG_PROBLEM_PUNCTURE = 1  /* -Laplace u - beta (1 + alpha (1 + u))^-7 = 0, puncture method */
};

typedef struct dg_puncture {
  double position[3];
  double mass;       /* bare mass */
  double momentum[3];/* Bowen-York linear momentum */
} dg_puncture;

/* Problem and discretization: an axis-aligned box split uniformly into n[0] x n[1] x n[2] affine
 * elements with N LGL points per dimension, homogeneous Dirichlet boundaries (Eq. bc),
 * internal-penalty parameter C (Eq. penalty). */
typedef struct dg_domain_desc {
  double lower[3];
  double upper[3];
  int32_t n[3];        /* elements per dimension, >= 1 */
  int32_t N;           /* LGL points per dimension, 2..DG_MAX_N */
  double penalty;      /* C > 0 */
  int32_t precision;   /* enum dg_precision */
  int32_t mg_levels;   /* 0: coarsen 2->1 along every even dimension while possible; else at most this many */
  int32_t overlap;     /* N_overlap, 1..N-1 (Sec. III.D.1) */
  int32_t presmooth;   /* Schwarz steps before restriction (and at the coarsest level) */
  int32_t postsmooth;  /* Schwarz steps after prolongation (and at the coarsest level) */
  int32_t problem;     /* enum dg_problem */
  int32_t n_punctures; /* DG_PROBLEM_PUNCTURE only, 0..DG_MAX_PUNCTURES */
  dg_puncture punctures[DG_MAX_PUNCTURES];
  int32_t subdomain_gemm; /* how du_S = A_S^-1 r_S is applied in a MIXED domain: enum dg_subdomain_gemm */
  int32_t neumann_faces;  /* bit f set: box face f (0 -x, 1 +x, 2 -y, 3 +y, 4 -z, 5 +z) carries the homogeneous
                             Neumann condition n.grad u = 0 of Eq. bc (interior auxiliary flux, zero
                             prescribed normal flux) instead of homogeneous Dirichlet; at least one
                             face must stay Dirichlet (the pure Neumann operator is singular) */
  const double* node_xyz; /* NULL: the affine box. Otherwise curved (mapped) elements (POISSON only): host
                             pointer to 3 n_dof doubles, the physical x, then y, then z coordinates of every
                             LGL node in the element-major layout, each element mapped isoparametrically
                             (Sec. II with the metric terms of Eqs. massmat, stiffmat, liftop); read only
                             during dg_domain_create. Shared face nodes must coincide; a folded or
                             left-handed element is DG_ERR_INVALID_ARG. Every subdomain then has its own
                             explicit inverse (E n_S^2 values per level) */
  const double* coef;     /* NULL: K = 1. Otherwise the operator is -div(K grad u) (fluxes F_u = K v in
                             Eq. fluxform, the penalty flux of Eq. numflux on K u; POISSON only): host pointer
                             to n_dof positive values of K at the nodes, read only during dg_domain_create;
                             the coarse levels interpolate it. As for curved elements, every subdomain then
                             has its own explicit inverse */
} dg_domain_desc;

enum dg_subdomain_gemm {
  DG_GEMM_DEFAULT = 0,      /* MIXED: tensor cores (TF32 inputs, FP32 accumulate); FP64: FP64 SIMT */
  DG_GEMM_SIMT = 1,         /* FP32 (or FP64) CUDA-core GEMM */
  DG_GEMM_TENSOR_TF32 = 2   /* tcgen05 tensor cores, TF32 inputs, FP32 accumulate (MIXED only) */
};

typedef struct dg_layout {
  int64_t n_dof;                        /* nodal values per vector on the finest level */
  int32_t n_elements;
  int32_t N;
  int32_t n[3];
  int32_t mg_levels;                    /* levels actually built */
  int32_t level_n[DG_MAX_LEVELS][3];    /* elements per dimension on every level */
  int32_t n_classes[DG_MAX_LEVELS];     /* distinct explicit subdomain inverses per level */
  int32_t subdomain_size;               /* padded subdomain size n_S = N^3 + 6 N_overlap N^2 */
  const double* x;                      /* device, library-owned: node coordinates, n_dof each */
  const double* y;
  const double* z;
  size_t device_bytes;                  /* device memory the domain holds */
} dg_layout;

typedef struct dg_solve_opts {
  int32_t max_iterations;      /* Krylov iterations per linear solve (no restart); default 200 */
  int32_t precondition;        /* 0 none, 1 Schwarz only (presmooth+postsmooth steps), 2 multigrid V-cycle (default) */
  double linear_tol;           /* PUNCTURE: relative tolerance of each linearized solve; default 1e-4 */
  int32_t max_newton_steps;    /* PUNCTURE: default 20 */
  int32_t subdomain_iterations;/* PUNCTURE: GMRES iterations per subdomain solve; default 3 */
  int32_t relative_to_b;       /* 0: tol relative to ||b - A u0|| (default); 1: relative to ||b|| */
  int32_t krylov;              /* 0: flexible GMRES (Sec. III.B, default); 1: flexible conjugate gradients
                                  (one search direction, three reductions per iteration; the operator is
                                  SPD for both problems): r = b - A x, z = M r,
                                  p = z - (z.A p_old / p_old.A p_old) p_old, alpha = p.r / p.A p */
  int32_t subdomain_solver;    /* PUNCTURE, finest level: 0 GMRES on A_S + D_S preconditioned by the Poisson
                                  class inverse (Sec. III.E's Laplacian approximation, default); 1 the
                                  explicit inverse of every subdomain's A_S + D_S, rebuilt at every
                                  linearization (E n_S^2 values of the smoother's precision on the device) */
} dg_solve_opts;

typedef struct dg_solve_report {
  int32_t status;              /* dg_status of the solve */
  int32_t iterations;          /* total Krylov iterations (summed over Newton steps) */
  int32_t newton_steps;
  int32_t line_search_steps;
  double initial_residual;     /* ||b - A(u0)||_2 */
  double final_residual;       /* ||b - A(u)||_2 recomputed in FP64 at exit */
  double relative_residual;    /* final / reference norm */
  double seconds;              /* host wall time of the call */
} dg_solve_report;

/* Build a domain: geometry, LGL tables, the multigrid hierarchy, Schwarz subdomains and their
 * explicit inverses (Sec. III.E: built column by column from the matrix-free subdomain operator,
 * inverted once, amortised over every later solve). The library owns all device state and uses
 * `cuda_stream` (NULL: the legacy default stream) for its work. Synchronous. */
dg_status dg_domain_create(const dg_domain_desc* desc, void* cuda_stream, struct dg_domain** out);
/* Free everything the domain holds. NULL-safe. */
void dg_domain_destroy(struct dg_domain* dom);
/* Sizes and the library-owned node coordinates, so that callers can fill f and b. */
dg_status dg_domain_layout(const struct dg_domain* dom, dg_layout* out);
/* Host-side node coordinates of the grid a descriptor defines (no domain, no GPU work): fills the
 * caller's host arrays x, y, z of n_dof = n[0] n[1] n[2] N^3 doubles each in the element-major
 * layout, so that a client can evaluate its source before submitting a served request. */
dg_status dg_layout_coordinates_host(const dg_domain_desc* desc, double* x, double* y, double* z);
/* Copy the node coordinates into caller-owned device buffers x, y, z (n_dof doubles each). */
dg_status dg_copy_coordinates(const struct dg_domain* dom, double* x, double* y, double* z, void* stream);
/* Message of the last failed call on this handle ("" if none). Thread-unsafe per handle. */
const char* dg_last_error(const struct dg_domain* dom);

/* Au = A u on the finest level, FP64 (Sec. II, Eqs. dg_op_auxvars and dg_op_primal with the
 * internal-penalty flux Eq. numflux and the homogeneous Dirichlet fluxes of Eq. bc). For a
 * PUNCTURE domain with a linearization set (dg_set_linearization) this is the linearized
 * operator A + M diag(S'(u_lin)). u and Au must not alias. The kernel moves whole lines of N
 * values, so u and Au must be aligned to gcd(16, N sizeof(value)) bytes, as every cudaMalloc or
 * PyTorch buffer and every whole-vector offset into one is; otherwise DG_ERR_INVALID_ARG. The same
 * holds for dg_apply_f32 and dg_apply_level. */
dg_status dg_apply(struct dg_domain* dom, const double* u, double* Au, void* stream);
/* Same operator in FP32 on multigrid level `level` (0 = finest). */
dg_status dg_apply_f32(struct dg_domain* dom, int32_t level, const float* u, float* Au, void* stream);
/* FP64 operator on level `level` (the rediscretized A_l of Eq. mg_problem). */
dg_status dg_apply_level(struct dg_domain* dom, int32_t level, const double* u, double* Au, void* stream);

/* b = M f, the right-hand side of Eq. dg_op_primal for nodal source values f. */
dg_status dg_rhs(struct dg_domain* dom, const double* f, double* b, void* stream);

/* Restriction b_coarse = R r_fine from level `level` to level+1, R = P^T (Sec. III.C.2). */
dg_status dg_mg_restrict(struct dg_domain* dom, int32_t level, const double* r_fine, double* b_coarse, void* stream);
/* u_fine += P u_coarse from level level+1 to `level` (Eq. prol). */
dg_status dg_mg_prolongate_add(struct dg_domain* dom, int32_t level, const double* u_coarse, double* u_fine, void* stream);

/* `iterations` additive Schwarz steps on level `level`, updating u in place (Sec. III.D.5):
 * r = b - A u; r_S = R_S r; du_S = A_S^-1 r_S; u += sum_S R_S^T (w_S du_S). In a MIXED domain
 * the subdomain work runs in FP32 and only u's update is accumulated in FP64. */
dg_status dg_schwarz_smooth(struct dg_domain* dom, int32_t level, const double* b, double* u, int32_t iterations,
                            void* stream);

/* z = one multigrid V-cycle applied to r from a zero initial guess (the preconditioner of
 * Sec. III.C.3, with presmooth/postsmooth Schwarz steps on every level, both at the coarsest). */
dg_status dg_vcycle(struct dg_domain* dom, const double* r, double* z, void* stream);

/* out[k] = sum_i V[k * ld + i] * w[i] for k < m (i < n_dof): the inner products of the FGMRES
 * orthogonalisation (Sec. III.B), FP64, as a deterministic two-pass reduction (fixed per-block
 * partial sums, then one ordered sum per output): bitwise reproducible. V, w, out are device
 * pointers (out: m doubles); ld >= n_dof. Uses the domain's workspace (allocated on first use). */
dg_status dg_dot(struct dg_domain* dom, int32_t m, const double* V, int64_t ld, const double* w, double* out,
                 void* stream);

/* Allocation-free variant of dg_dot for callers that cannot allocate device memory when they
 * need it: code running during CUDA stream capture, serving loops whose memory is fixed up front,
 * plugins whose host owns every allocation. The paper has no counterpart; it is a deployment
 * convenience. Same result as dg_dot (bitwise: same kernels, same reduction order) for n values
 * per vector, without a domain: the per-block partial sums live in a fixed device array of
 * 304 * DG_NOALLOC_MAX_VECTORS doubles (152 KiB) that every GPU loading the library keeps until
 * the process exits. m above DG_NOALLOC_MAX_VECTORS is rejected with DG_ERR_INVALID_ARG; the
 * message is available from dg_last_error(NULL). The call allocates nothing and calls no
 * allocating routine. The first call on a device (with that device current) looks up the array's
 * device address, so make that first call before any stream capture; the address is kept until the
 * process exits, so the device must not be reset (cudaDeviceReset) after it. All calls share the one
 * array: calls that overlap on the GPU (concurrent streams) race and must be serialised by the
 * caller. V, w, out are device pointers; stream as elsewhere (NULL: legacy default stream). */
enum { DG_NOALLOC_MAX_VECTORS = 64 };
dg_status dg_dot_noalloc(int64_t n, int32_t m, const double* V, int64_t ld, const double* w, double* out,
                         void* stream);

/* Debug builds only (the library compiled with index bounds checks: libdg_elliptic_debug.so, from
 * `python paper_2111_06767_gb300/build.py --debug`): the indices the kernels take from set-up
 * tables (subdomain point maps, orientation and column maps) are checked before use, an index out
 * of range is skipped instead of used, and the first offending kernel source line is recorded. The
 * call synchronises the current device, returns that line (0: no index was out of range since the
 * last call) and clears it; -1 in a release build, which has no checks. Not in the paper. */
int32_t dg_debug_bounds_check(void);

/* PUNCTURE: r = b - A(u) with A(u) = A u + M S(u), S(u) = -beta (1 + alpha (1 + u))^-7. */
dg_status dg_nonlinear_residual(struct dg_domain* dom, const double* u, const double* b, double* r, void* stream);
/* PUNCTURE: linearize at u (Eq. linearized): dg_apply then applies A + M diag(S'(u)). NULL clears. */
dg_status dg_set_linearization(struct dg_domain* dom, const double* u, void* stream);
/* PUNCTURE: how the finest level's Schwarz subdomain problems (A_S + D_S) du_S = r_S of the
 * linearized operator are solved by dg_schwarz_smooth and the V-cycle (Sec. III.E): solver 0 by
 * `iterations` GMRES iterations (0..16; 0 applies the Poisson inverse alone) right-preconditioned
 * by the Poisson class inverse; solver 1 by the explicit inverse of every subdomain's own A_S + D_S.
 * Those inverses (E n_S^2 values in the smoother's precision; DG_ERR_OOM if they do not fit) are
 * built by dg_set_linearization, or by this call when a linearization is already set.
 * elliptic_solve sets the same state from its options. Default: solver 0, 3 iterations. */
dg_status dg_set_subdomain_solver(struct dg_domain* dom, int32_t solver, int32_t iterations, void* stream);
/* PUNCTURE: copy the library-computed alpha and beta at the nodes into caller-owned device buffers. */
dg_status dg_puncture_fields(const struct dg_domain* dom, double* alpha, double* beta, void* stream);

/* Solve A u = b (or A(u) = b for PUNCTURE) to ||b - A u||_2 <= tol * reference. u holds the
 * initial guess on entry and the solution on exit. Linear: FGMRES + multigrid-Schwarz.
 * Nonlinear: Newton-Raphson with line search, each step a FGMRES solve to opts->linear_tol.
 * opts and report may be NULL. Synchronous on the domain's stream. Returns DG_OK when the
 * FP64 residual recomputed at exit meets the tolerance. */
dg_status elliptic_solve(struct dg_domain* dom, const double* b, double* u, double tol, const dg_solve_opts* opts,
                         dg_solve_report* report);
/* The same solve with HOST buffers, for callers that keep their data in host memory: f_host holds
 * the nodal source f (n_dof values; POISSON: b = M f, Eq. dg_op_primal; PUNCTURE: ignored, may be
 * NULL), u_host the initial guess on entry and the solution on exit. The call copies f and u to
 * library-owned device buffers of the domain (allocated on the first call), solves as
 * elliptic_solve does and copies u back, all on the domain's stream; it returns when u_host holds
 * the result. Page-locked host buffers (cudaHostAlloc, cudaHostRegister) make the copies
 * asynchronous DMA transfers; pageable ones are staged by the driver. */
dg_status elliptic_solve_host(struct dg_domain* dom, const double* f_host, double* u_host, double tol,
                              const dg_solve_opts* opts, dg_solve_report* report);

/* elliptic_solve runs a linear FGMRES solve with the multigrid preconditioner (opts->precondition 2,
 * per-phase profiling off) as ONE CUDA graph from the second solve on a domain with the same
 * tolerance and kernels: the Hessenberg column, its Givens rotations and the stopping test of
 * Sec. III.B are computed on the device, and the Arnoldi loop is a conditional WHILE node, so an
 * iteration needs no host round trip (the first such solve runs host-driven and tunes the launch
 * shapes). A captured solve holds at most 40 Arnoldi columns; a solve that needs more continues
 * host-driven from the graph's iterate (a restart). Setting DG_SOLVE_GRAPH=0 in the environment
 * keeps every solve host-driven. */

/* Many independent linear solves (POISSON problems on distinct domains) as one CUDA graph: each
 * solve is one branch of the graph (b and u copied in, FGMRES with the multigrid preconditioner as
 * above, u copied out), so one launch runs them all concurrently on the device. create captures
 * the graph (it first runs every kernel shape of each domain once, untimed, on the domain's
 * stream, and synchronises); run launches it on `stream` and waits for it, filling count
 * reports. b[i] and u[i] are device pointers of domain i's n_dof values, fixed for the life of the
 * batch (u[i] holds the initial guess before each run and the solution after it); the domains
 * must outlive every run of the batch and must not be used by other calls while a run is in flight
 * (destroying the batch does not touch them, so it may come after them). opts as for
 * elliptic_solve with krylov 0 and precondition 2 (NULL: defaults). Errors of create and run are
 * described by dg_last_error(NULL). Not in the paper, whose solves run one at a time. */
typedef struct dg_batch dg_batch;
dg_status elliptic_batch_create(struct dg_domain* const* domains, const double* const* b, double* const* u,
                                int32_t count, double tol, const dg_solve_opts* opts, struct dg_batch** out);
dg_status elliptic_batch_run(struct dg_batch* batch, void* stream, dg_solve_report* reports);
void elliptic_batch_destroy(struct dg_batch* batch);

/* ---------------------------------------------------------------------------------------------
 * Per-phase kernel timing: CUDA events around every launch of a phase on the stream it runs on.
 * Bytes and flops are the algorithmic minimum of each launch (the data it must read and write
 * once, the arithmetic of its contraction), accumulated over launches, so bytes / time is the
 * achieved bandwidth against the roofline.
 * ------------------------------------------------------------------------------------------- */
enum dg_phase {
  DG_PHASE_APPLY_FP64 = 0,  /* DG operator, FP64 (read u [+ b, diag], write A u) */
  DG_PHASE_APPLY_FP32 = 1,  /* DG operator, FP32 */
  DG_PHASE_GATHER = 2,      /* r_S = R_S r */
  DG_PHASE_SUBDOMAIN_GEMM = 3, /* du_S = A_S^-1 r_S: read every class inverse once, r_S, write du_S */
  DG_PHASE_SCATTER = 4,     /* u += sum_S R_S^T w_S du_S */
  DG_PHASE_TRANSFER = 5,    /* restriction and prolongation */
  DG_PHASE_KRYLOV = 6,      /* FGMRES vector kernels and precision conversions */
  DG_PHASE_COARSE_SMOOTH = 7, /* fused Schwarz smoothing on a coarse level (residual, subdomain
                                 solves and scatter of all steps in one launch) */
  DG_PHASE_SUBDOMAIN_BUILD = 8, /* per-subdomain linearized matrices A_S + D_S and their inversion */
  DG_PHASE_COUNT = 9
};

typedef struct dg_phase_stats {
  int64_t launches;
  double milliseconds;  /* summed CUDA-event durations */
  double bytes;         /* summed algorithmic bytes */
  double flops;         /* summed algorithmic flops */
} dg_phase_stats;

/* Number of CUDA kernels this library has launched in the process so far (all domains). */
int64_t dg_kernel_launches(void);
/* Start (enable != 0, accumulators cleared) or stop timing launches on this domain. */
dg_status dg_profile_enable(struct dg_domain* dom, int32_t enable);
/* Synchronise the domain's streams and return the accumulated per-phase statistics. */
dg_status dg_profile_read(struct dg_domain* dom, dg_phase_stats out[DG_PHASE_COUNT]);

/* ---------------------------------------------------------------------------------------------
 * Serving: a continuous-batching request loop. Requests (a domain descriptor plus a nodal source
 * on the host) are admitted while their device footprint fits the server's memory budget and a
 * slot is free; admitted solves run concurrently on the server's streams, and completed results
 * are returned through poll. Requests that arrive while others run join as capacity frees up.
 * ------------------------------------------------------------------------------------------- */
typedef struct dg_serve_desc {
  size_t memory_budget_bytes; /* device bytes the server may hold for admitted requests (0: 80% of free) */
  int32_t max_active;         /* concurrently running solves (>= 1) */
  int32_t queue_capacity;     /* waiting requests before submit answers DG_ERR_BUSY */
  int32_t n_streams;          /* CUDA streams the workers use (>= 1) */
} dg_serve_desc;

typedef struct dg_request {
  dg_domain_desc domain;
  const double* f_host;       /* host nodal source values (n_dof, element-major); copied by submit.
                                 NULL for PUNCTURE (b = 0) */
  double tol;                 /* residual tolerance relative to ||b|| */
  dg_solve_opts opts;
} dg_request;

typedef struct dg_result {
  dg_solve_report report;
  double* u_host;             /* caller buffer of n_dof doubles, or NULL to skip the solution copy */
  int64_t n_dof;
  double submit_time;         /* server clock (s) at submit, admission and completion */
  double admit_time;
  double finish_time;
} dg_result;

dg_status elliptic_serve_create(const dg_serve_desc* desc, struct dg_server** out);
/* Copy the request into library memory and return at once with a ticket. DG_ERR_BUSY if the
 * waiting queue is full, DG_ERR_INVALID_ARG if the request can never fit the memory budget. */
dg_status elliptic_serve_submit(struct dg_server* srv, const dg_request* req, uint64_t* ticket);
/* DG_PENDING while the request waits or runs; its final status (DG_OK or an error) once done,
 * with the report, times and (if out->u_host is set) the solution copied out. A finished ticket
 * is released by the poll that returns it. */
dg_status elliptic_serve_poll(struct dg_server* srv, uint64_t ticket, dg_result* out);
/* Cancel a request: one still waiting leaves the queue; one running stops at its next Krylov
 * iteration (the solve checks between iterations, never inside a kernel). Its poll then returns
 * DG_ERR_CANCELLED. A request that has already finished keeps its result. DG_ERR_NOT_FOUND for an
 * unknown or already released ticket. */
dg_status elliptic_serve_cancel(struct dg_server* srv, uint64_t ticket);
/* Seconds on the server's clock (for latency bookkeeping). */
double elliptic_serve_clock(const struct dg_server* srv);
/* Stop accepting, finish what is admitted, join the workers and free everything. NULL-safe. */
void elliptic_serve_destroy(struct dg_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* DG_ELLIPTIC_H */
