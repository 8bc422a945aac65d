// Solver orchestration on one stream: Schwarz smoothing (Sec. III.D.5), the multigrid V-cycle
// (Sec. III.C.3), flexible GMRES (Sec. III.B, Saad Alg. 9.6) and Newton-Raphson with a line
// search (Sec. III.A). All vector work runs in the library's kernels; the host only keeps the
// (k+1) x k Hessenberg matrix and its Givens rotations, read back once per Krylov iteration.
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <type_traits>

#include "domain.h"

namespace dg {

namespace {
// algorithmic work of one DG apply: read u (+ b, diag), write the result; 12N + 12 flops per point
// for the six sum-factorised contractions plus the face terms amortised per point
double apply_bytes(int64_t ndof, size_t sz, bool b, bool diag) { return (double)ndof * sz * (2 + b + diag); }
double apply_flops(int64_t ndof, int N) { return (double)ndof * (12.0 * N + 12.0); }
}  // namespace

namespace {
// Launch shape of the DG apply for this level, precision and output: tuned on the first call (the
// timed launches compute the same result into the same output, so the call stays correct).
template <typename T>
int apply_variant(dg_domain* dom, Level& L, bool fused, const std::function<void(int)>& run, cudaStream_t s) {
  int& v = L.apply_variant[sizeof(T) == 4][fused];
  if (v < 0) {
    // launch shapes of the line kernel; the plane kernel for plain FP32 applies at N = 4
    std::vector<int> cand{0, 1, 2, 3};
    if (!fused && dom->N == 4 && sizeof(T) == 4) {  // the slice kernel and the element kernel
      cand.push_back(4);
      cand.push_back(7);
    }
    if (dom->N >= 4 && sizeof(T) == 4) {  // the block-of-lines kernel, two launch shapes
      cand.push_back(5);
      cand.push_back(6);
    }
    // DG_APPLY_VARIANT=v pins one candidate (tests of each launch shape)
    static const int forced = [] {
      const char* e = std::getenv("DG_APPLY_VARIANT");
      return e ? std::atoi(e) : -1;
    }();
    if (forced >= 0 && std::find(cand.begin(), cand.end(), forced) != cand.end()) {
      v = forced;
      return v;
    }
    const int pick = autotune({1, dom->N, (int64_t)sizeof(T), L.n[0], L.n[1], L.n[2], fused}, cand, run, s);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    DG_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone) return pick;  // not tuned while capturing: ask again later
    v = pick;
  }
  return v;
}
}  // namespace

namespace {
// Curved elements: out = A u (or b - A u); into the subdomain vectors through the level's residual
// buffer and a gather.
template <typename T>
void curved_apply(dg_domain* dom, Level& L, const T* u, T* out, const T* b, cudaStream_t s, const SubdomainOut* so,
                  const T* geo, const T* sig, T* trace, const T* D, const T* w, T* r_scratch) {
  CurvedArgs<T> a{};
  for (int i = 0; i < 3; ++i) a.n[i] = L.n[i];
  a.neumann = dom->desc.neumann_faces;
  a.ndof = L.ndof;
  a.geo = geo;
  a.sigma = sig;
  a.D = D;
  a.w = w;
  a.u = u;
  a.b = b;
  a.trace = trace;
  a.out = so ? r_scratch : out;
  DG_REQUIRE(a.out != nullptr, "curved residual needs the level's work vectors");
  launch_curved_apply<T>(dom->N, a, L.E, s);
  if (so)
    launch_gather_tab<T>(L.sw.geom, a.out, L.sw.elem_of_col.get(), L.sw.xform_of_elem.get(), dom->orient_map.get(),
                         static_cast<T*>(so->rS), s);
}
}  // namespace

void apply_level(dg_domain* dom, int level, const double* u, double* out, const double* b, bool with_lin,
                 cudaStream_t s, const SubdomainOut* so) {
  Level& L = dom->levels[level];
  if (dom->curved) {
    PhaseScope ps(dom->prof, DG_PHASE_APPLY_FP64, s, (double)L.ndof * 8 * (b ? 3 : 2) + 80.0 * L.ndof, 0.0);
    curved_apply<double>(dom, L, u, out, b, s, so, L.geo64.get(), L.sig64.get(), L.trace64.get(), dom->D64.get(),
                         dom->w64.get(), L.w64.r.get());
    return;
  }
  const double* diag = (with_lin && level == 0 && dom->lin_set) ? dom->lin64.get() : nullptr;
  PhaseScope ps(dom->prof, DG_PHASE_APPLY_FP64, s, apply_bytes(L.ndof, 8, b, diag), apply_flops(L.ndof, dom->N));
  auto run = [&](int v) {
    launch_apply<double>(dom->N, L.g64, dom->D64.get(), dom->w64.get(), u, diag, b, out, s, so, v,
                         dom->err_flag.get());
  };
  run(apply_variant<double>(dom, L, so != nullptr, run, s));
}

void apply_level_f32(dg_domain* dom, int level, const float* u, float* out, const float* b, bool with_lin,
                     cudaStream_t s, const SubdomainOut* so) {
  Level& L = dom->levels[level];
  if (dom->curved) {
    PhaseScope ps(dom->prof, DG_PHASE_APPLY_FP32, s, (double)L.ndof * 4 * (b ? 3 : 2) + 40.0 * L.ndof, 0.0);
    curved_apply<float>(dom, L, u, out, b, s, so, L.geo32.get(), L.sig32.get(), L.trace32.get(), dom->D32.get(),
                        dom->w32.get(), L.w32.r.get());
    return;
  }
  const float* diag = (with_lin && level == 0 && dom->lin_set && dom->lin32.get()) ? dom->lin32.get() : nullptr;
  PhaseScope ps(dom->prof, DG_PHASE_APPLY_FP32, s, apply_bytes(L.ndof, 4, b, diag), apply_flops(L.ndof, dom->N));
  auto run = [&](int v) {
    launch_apply<float>(dom->N, L.g32, dom->D32.get(), dom->w32.get(), u, diag, b, out, s, so, v,
                        dom->err_flag.get());
  };
  run(apply_variant<float>(dom, L, so != nullptr, run, s));
}

namespace {

template <typename T>
LevelWork<T>& work(Level& L);
template <>
LevelWork<double>& work<double>(Level& L) { return L.w64; }
template <>
LevelWork<float>& work<float>(Level& L) { return L.w32; }

template <typename T>
const T* inverses(const SchwarzLevel& sw);
template <>
const double* inverses<double>(const SchwarzLevel& sw) { return sw.inv64.get(); }
template <>
const float* inverses<float>(const SchwarzLevel& sw) { return sw.inv32.get(); }

template <typename T>
const T* shares(const dg_domain* dom);
template <>
const double* shares<double>(const dg_domain* dom) { return dom->shares64.get(); }
template <>
const float* shares<float>(const dg_domain* dom) { return dom->shares32.get(); }

template <typename T>
const T* lin_diag(const dg_domain* dom);
template <>
const double* lin_diag<double>(const dg_domain* dom) { return dom->lin64.get(); }
template <>
const float* lin_diag<float>(const dg_domain* dom) { return dom->lin32.get(); }

// The finest level of a linearized problem smooths with the linearized subdomain problems
// A_S + D_S (per-subdomain inverses, or GMRES with the Poisson inverse as preconditioner).
template <typename T>
bool linearized_smoother(const dg_domain* dom, int level) {
  return level == 0 && dom->lin_set && dom->desc.problem == DG_PROBLEM_PUNCTURE && lin_diag<T>(dom) != nullptr &&
         (dom->subdomain_solver == 1 || dom->subdomain_iterations > 0);
}

template <typename T>
void apply_T(dg_domain* dom, int level, const T* u, T* out, const T* b, cudaStream_t s,
             const SubdomainOut* so = nullptr);
template <>
void apply_T<double>(dg_domain* dom, int level, const double* u, double* out, const double* b, cudaStream_t s,
                     const SubdomainOut* so) {
  apply_level(dom, level, u, out, b, true, s, so);
}
template <>
void apply_T<float>(dg_domain* dom, int level, const float* u, float* out, const float* b, cudaStream_t s,
                    const SubdomainOut* so) {
  apply_level_f32(dom, level, u, out, b, true, s, so);
}

template <typename T>
const T* Ilo(dg_domain* dom);
template <>
const double* Ilo<double>(dg_domain* dom) { return dom->Ilo64.get(); }
template <>
const float* Ilo<float>(dg_domain* dom) { return dom->Ilo32.get(); }
template <typename T>
const T* Ihi(dg_domain* dom);
template <>
const double* Ihi<double>(dg_domain* dom) { return dom->Ihi64.get(); }
template <>
const float* Ihi<float>(dg_domain* dom) { return dom->Ihi32.get(); }

}  // namespace

template <typename T>
void launch_class_gemm_tiles(const T* inv, const T* X, T* Y, int ld, const int4* d_tiles, int n_tiles,
                             const int* d_kchunks, T alpha, cudaStream_t s, int split);

namespace {
// The CUDA-core class GEMM with its K split tuned per level and precision on first use (0, the
// heuristic, then 1, 2, 4, 8); DG_GEMM_SPLIT pins it as for the tensor-core GEMM.
template <typename T>
void simt_class_gemm(Level& L, const T* inv, const T* X, T* Y, T alpha, cudaStream_t s) {
  const SchwarzLevel& sw = L.sw;
  int& pick = L.simt_split[sizeof(T) == 8];
  auto run = [&](int split) {
    launch_class_gemm_tiles<T>(inv, X, Y, sw.ld, sw.tiles.get(), sw.n_tiles, sw.kchunks16.get(), alpha, s, split);
  };
  if (pick < 0) {
    std::vector<int> cand{0};
    const int nk = (sw.ld + 15) / 16;
    for (int sp = 1; sp <= 8; sp *= 2)
      if (nk / sp >= 4) cand.push_back(sp);
    const char* e = std::getenv("DG_GEMM_SPLIT");
    const int forced = e ? std::atoi(e) : -1;
    if (forced >= 0 && std::find(cand.begin(), cand.end(), forced) != cand.end()) {
      pick = forced;
    } else {
      const int p = autotune({4, (int64_t)sizeof(T), sw.n_classes, sw.ld, sw.n_tiles, L.E}, cand, run, s);
      cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
      DG_CUDA(cudaStreamIsCapturing(s, &cap));
      if (cap != cudaStreamCaptureStatusNone) {
        run(p);
        return;
      }
      pick = p;
    }
  }
  run(pick);
}
}  // namespace

namespace {
// du_S = A_S^-1 r_S for every subdomain of every class
template <typename T>
void class_gemm(dg_domain* dom, Level& L, const T* X, T* Y, cudaStream_t s);
template <>
void class_gemm<double>(dg_domain* dom, Level& L, const double* X, double* Y, cudaStream_t s) {
  const SchwarzLevel& sw = L.sw;
  if (dom->curved) {  // one inverse per subdomain
    launch_lin_gemv<double>(sw.inv64.get(), X, sw.nS, sw.ld, L.E, Y, s);
    return;
  }
  simt_class_gemm<double>(L, sw.inv64.get(), X, Y, sw.inv_scale, s);
}
template <>
void class_gemm<float>(dg_domain* dom, Level& L, const float* X, float* Y, cudaStream_t s) {
  const SchwarzLevel& sw = L.sw;
  if (dom->curved) {  // one inverse per subdomain
    if (sw.inv16.get())
      launch_lin_gemv_half(sw.inv16.get(), sw.inv16_scale.get(), X, sw.nS, sw.ld, L.E, Y, s);
    else
      launch_lin_gemv<float>(sw.inv32.get(), X, sw.nS, sw.ld, L.E, Y, s);
    return;
  }
  if (dom->use_tc) {
    // launch shape: split-K factor (low 4 bits; 0 = chosen from the tile count) and tile width
    // (kWide: 256 columns, kMid: 128, else 64)
    constexpr int kWide = 16, kMid = 32;
    auto run = [&](int shape) {
      const int bn = (shape & kWide) ? 256 : ((shape & kMid) ? 128 : 64);
      const int4* t = bn == 256 ? sw.tiles_tc256.get() : (bn == 128 ? sw.tiles_tc128.get() : sw.tiles_tc.get());
      const int nt = bn == 256 ? sw.n_tiles_tc256 : (bn == 128 ? sw.n_tiles_tc128 : sw.n_tiles_tc);
      launch_class_gemm_tc(sw.inv32.get(), sw.n_classes, X, Y, sw.ld, L.E, t, nt, sw.kchunks32.get(),
                           dom->err_flag.get(), (float)sw.inv_scale, s, shape & 15, bn);
    };
    if (L.gemm_split < 0) {
      // the default (0) first, then every split the shape allows, at every tile width
      std::vector<int> cand{0};
      for (int sp : tc_gemm_splits(sw.ld)) cand.push_back(sp);
      for (int w : {kMid, kWide}) {
        cand.push_back(w);
        for (int sp : tc_gemm_splits(sw.ld)) cand.push_back(w | sp);
      }
      // DG_GEMM_SPLIT=k pins one candidate (tests and measurements of each launch shape); read
      // when a level first runs its GEMM, so a process can set it per domain
      const char* e = std::getenv("DG_GEMM_SPLIT");
      const int forced = e ? std::atoi(e) : -1;
      if (forced >= 0 && std::find(cand.begin(), cand.end(), forced) != cand.end()) {
        L.gemm_split = forced;
        run(forced);
        return;
      }
      const int pick = autotune({3, sw.n_classes, sw.ld, sw.n_tiles_tc, sw.n_tiles_tc128, sw.n_tiles_tc256, L.E}, cand,
                                run, s);
      cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
      DG_CUDA(cudaStreamIsCapturing(s, &cap));
      if (cap != cudaStreamCaptureStatusNone) {
        run(pick);
        return;
      }
      L.gemm_split = pick;
    }
    run(L.gemm_split);
  } else
    simt_class_gemm<float>(L, sw.inv32.get(), X, Y, (float)sw.inv_scale, s);
}
}  // namespace

// Levels with at most this many elements are smoothed by the fused cooperative kernel (MIXED).
constexpr int kCoarseFusedElems = 64;

template <typename T>
void schwarz_smooth(dg_domain* dom, int level, const T* b, T* u, int iterations, bool u_is_zero, cudaStream_t s) {
  // FP32 coarse levels: each kernel is a short latency chain, so the next one's launch and set-up
  // overlap it (programmatic dependent launch); the fine level and FP64 keep plain stream order
  const PdlScope pdl(sizeof(T) == 4 && pdl_vcycle_mode() >= (level > 0 ? 1 : 2));
  ensure_schwarz(dom, level);
  Level& L = dom->levels[level];
  LevelWork<T>& W = work<T>(L);
  SchwarzLevel& sw = L.sw;
  DG_REQUIRE((inverses<T>(sw) != nullptr || (sizeof(T) == 4 && sw.inv16.get())) && shares<T>(dom) != nullptr,
             "Schwarz data of this precision are not built for this domain");
  if (iterations <= 0) return;
  const bool linearized_level = linearized_smoother<T>(dom, level);
  DG_REQUIRE(!linearized_level || dom->subdomain_solver != 1 || dom->linv_current,
             "per-subdomain linearized inverses are not built for the current linearization");
  if constexpr (std::is_same<T, float>::value) {
    if (dom->coarse_fused && L.E <= kCoarseFusedElems && !linearized_level && coarse_smooth_available(dom->N)) {
      // all steps of this call in one cooperative launch
      CoarseArgs a{};
      const float* diag = (level == 0 && dom->lin_set && dom->lin32.get()) ? dom->lin32.get() : nullptr;
      a.ap = ApplyArgs<float>{L.g32, dom->D32.get(), dom->w32.get(), u, diag, b, nullptr, L.E, W.rS.get(), sw.ld,
                              dom->desc.overlap, sw.col_of_elem.get(), sw.xform_of_elem.get(), dom->orient_inv.get()};
      a.sg = sw.geom;
      a.elem_of_col = sw.elem_of_col.get();
      a.map = dom->orient_map.get();
      a.shares = dom->shares32.get();
      a.duS = W.duS.get();
      a.invm = sw.inv32.get();
      a.alpha = (float)sw.inv_scale;
      a.units = sw.units.get();
      a.n_units = sw.n_units;
      a.bar = sw.bar.get();
      a.err = dom->err_flag.get();
      a.iterations = iterations;
      a.u_zero = u_is_zero ? 1 : 0;
      a.stall = dom->barrier_stall;
      const double vec = (double)L.E * sw.nS * 4.0, nS = sw.nS;
      PhaseScope ps(dom->prof, DG_PHASE_COARSE_SMOOTH, s,
                    iterations * ((double)sw.n_classes * nS * nS * 4.0 + 2 * vec + 4.0 * 4.0 * L.ndof),
                    iterations * (2.0 * nS * nS * L.E + (12.0 * dom->N + 12.0) * L.ndof));
      launch_coarse_smooth(dom->N, a, s);
      return;
    }
  }
  SubdomainOut so;
  so.rS = W.rS.get();
  so.ld = sw.ld;
  so.ov = dom->desc.overlap;
  so.col_of_elem = sw.col_of_elem.get();
  so.orient = sw.xform_of_elem.get();
  so.inv = dom->orient_inv.get();
  for (int it = 0; it < iterations; ++it) {
    const double sz = sizeof(T), vec = (double)L.E * sw.nS * sz;
    const int ld = sw.ld;
    if (it == 0 && u_is_zero) {
      // with u = 0 the residual is b itself: gather it into the subdomain vectors
      PhaseScope ps(dom->prof, DG_PHASE_GATHER, s, L.ndof * sz + vec, 0.0);
      launch_gather_tab<T>(sw.geom, b, sw.elem_of_col.get(), sw.xform_of_elem.get(), dom->orient_map.get(), W.rS.get(),
                           s);
    } else {
      apply_T<T>(dom, level, u, nullptr, b, s, &so);  // r = b - A u, written straight into r_S
    }
    const bool linearized = linearized_level;
    auto gemm = [&](const T* X, T* Y) {
      const double isz = (sizeof(T) == 4 && sw.inv16.get()) ? 2.0 : sz;  // FP16-stored inverses
      // algorithmic: each class's inverse and vectors at its real subdomain size (slots present)
      PhaseScope ps(dom->prof, DG_PHASE_SUBDOMAIN_GEMM, s, sw.alg_inv * isz + 2.0 * sw.alg_vec * sz,
                    2.0 * sw.alg_mac);
      class_gemm<T>(dom, L, X, Y, s);
    };
    if (!linearized) {
      gemm(W.rS.get(), W.duS.get());
    } else if (dom->subdomain_solver == 1) {
      // du_S = (A_S + D_S)^-1 r_S with every subdomain's own inverse (built at the linearization)
      PhaseScope ps(dom->prof, DG_PHASE_SUBDOMAIN_GEMM, s, (double)L.E * sw.nS * sw.nS * sz + 2 * vec,
                    2.0 * sw.nS * (double)sw.nS * L.E);
      launch_lin_gemv<T>(W.linv.get(), W.rS.get(), sw.nS, ld, L.E, W.duS.get(), s);
    } else {
      // GMRES on (A_S + D_S), right-preconditioned by the Poisson inverse A_S^-1 (Sec. III.E)
      const int m = dom->subdomain_iterations;
      const size_t blk = (size_t)L.E * ld;
      if (W.gV.count < (m + 1) * blk) {
        W.gV.alloc((m + 1) * blk);
        W.gZ.alloc(m * blk);
        W.gD.alloc(blk);
        W.gH.alloc((size_t)L.E * ((m + 1) * m + 1));
      }
      T* beta = W.gH.get() + (size_t)L.E * (m + 1) * m;
      launch_gather_tab<T>(sw.geom, lin_diag<T>(dom), sw.elem_of_col.get(), sw.xform_of_elem.get(),
                           dom->orient_map.get(), W.gD.get(), s);
      // the per-subdomain vector kernels count as Krylov work, the preconditioner GEMMs as GEMM
      {
        PhaseScope ps(dom->prof, DG_PHASE_KRYLOV, s, 2.0 * blk * sz, 2.0 * blk);
        launch_sub_normalize<T>(L.E, ld, W.rS.get(), W.gV.get(), beta, s);
      }
      for (int j = 0; j < m; ++j) {
        gemm(W.gV.get() + j * blk, W.gZ.get() + j * blk);
        // read V_j, D, Z_j and V_0..V_j, write V_{j+1}
        PhaseScope ps(dom->prof, DG_PHASE_KRYLOV, s, (double)blk * sz * (j + 5.0), 4.0 * blk * (j + 2.0));
        launch_sub_arnoldi<T>(L.E, ld, j, m, W.gD.get(), W.gV.get(), W.gZ.get(), W.gH.get(), s);
      }
      {
        PhaseScope ps(dom->prof, DG_PHASE_KRYLOV, s, (double)blk * sz * (m + 1.0), 2.0 * blk * m);
        launch_sub_lsq_combine<T>(L.E, ld, m, beta, W.gH.get(), W.gZ.get(), W.duS.get(), s);
      }
    }
    {
      // mode 3: the fine level's scatter also overlaps the GEMM before it
      const PdlScope pdl_scatter(sizeof(T) == 4 && level == 0 && pdl_vcycle_mode() == 3);
      PhaseScope ps(dom->prof, DG_PHASE_SCATTER, s, vec + 2.0 * L.ndof * sz, 0.0);
      launch_scatter_tab<T, T>(sw.geom, W.duS.get(), sw.col_of_elem.get(), sw.xform_of_elem.get(),
                               dom->orient_inv.get(), shares<T>(dom), u, s);
    }
  }
}

template void schwarz_smooth<double>(dg_domain*, int, const double*, double*, int, bool, cudaStream_t);
template void schwarz_smooth<float>(dg_domain*, int, const float*, float*, int, bool, cudaStream_t);

// One V-cycle from a zero initial guess: z ~= A^-1 r.
template <typename T>
void vcycle(dg_domain* dom, const T* r, T* z, cudaStream_t s) {
  const int nl = (int)dom->levels.size();
  const int pre = dom->desc.presmooth, post = dom->desc.postsmooth;
  const int N = dom->N;
  // level 0 works directly in (r, z)
  for (int l = 0; l < nl; ++l) ensure_schwarz(dom, l);
  auto B = [&](int l) -> const T* { return l == 0 ? r : work<T>(dom->levels[l]).b.get(); };
  auto U = [&](int l) -> T* { return l == 0 ? z : work<T>(dom->levels[l]).u.get(); };
  for (int l = 0; l < nl; ++l) DG_CUDA(cudaMemsetAsync(U(l), 0, sizeof(T) * dom->levels[l].ndof, s));
  const PdlScope pdl(sizeof(T) == 4 && pdl_vcycle_mode() >= 2);  // transfers and residuals
  for (int l = 0; l < nl - 1; ++l) {
    Level& L = dom->levels[l];
    schwarz_smooth<T>(dom, l, B(l), U(l), pre, true, s);
    apply_T<T>(dom, l, U(l), work<T>(L).r.get(), B(l), s);  // Eq. mg_res
    PhaseScope ps(dom->prof, DG_PHASE_TRANSFER, s, (double)(L.ndof + dom->levels[l + 1].ndof) * sizeof(T),
                  6.0 * N * L.ndof);
    launch_restrict<T>(N, L.n, dom->levels[l + 1].n, Ilo<T>(dom), Ihi<T>(dom), work<T>(L).r.get(),
                       work<T>(dom->levels[l + 1]).b.get(), s);
  }
  schwarz_smooth<T>(dom, nl - 1, B(nl - 1), U(nl - 1), pre, true, s);
  schwarz_smooth<T>(dom, nl - 1, B(nl - 1), U(nl - 1), post, pre == 0, s);
  for (int l = nl - 2; l >= 0; --l) {
    Level& L = dom->levels[l];
    {
      PhaseScope ps(dom->prof, DG_PHASE_TRANSFER, s, (double)(2 * L.ndof + dom->levels[l + 1].ndof) * sizeof(T),
                    6.0 * N * L.ndof);
      launch_prolongate_add<T>(N, L.n, dom->levels[l + 1].n, Ilo<T>(dom), Ihi<T>(dom), U(l + 1), U(l), s);
    }
    schwarz_smooth<T>(dom, l, B(l), U(l), post, false, s);
  }
}

template void vcycle<double>(dg_domain*, const double*, double*, cudaStream_t);
template void vcycle<float>(dg_domain*, const float*, float*, cudaStream_t);

namespace {

// Run the V-cycle on the domain's fixed buffers (FP32 vin32 -> vin32 + n in MIXED, vin64 -> vout64
// in FP64), replaying a captured CUDA graph when possible: the ~100 launches of a V-cycle become
// one graph launch. The graph is captured on the second call (the first one allocates lazily and
// sets kernel attributes) and re-captured when the linearization state changes.
void vcycle_fixed(dg_domain* dom, cudaStream_t s) {
  const int64_t n = dom->levels[0].ndof;
  auto run = [&](cudaStream_t st) {
    if (dom->mixed) vcycle<float>(dom, dom->vin32.get(), dom->vin32.get() + n, st);
    else vcycle<double>(dom, dom->vin64.get(), dom->vout64.get(), st);
  };
  const bool lin = dom->lin_set;
  const int m = dom->subdomain_iterations;
  const int sub = dom->subdomain_solver;
  const bool prof = dom->prof.on;
  if (dom->vgraph && (dom->vgraph_lin != lin || dom->vgraph_m != m || dom->vgraph_sub != sub ||
                      dom->vgraph_prof != prof || dom->vgraph_stall != dom->barrier_stall)) {
    // different kernels: drop the graph and run once uncaptured (it may allocate) before re-capturing
    cudaGraphExecDestroy(dom->vgraph);
    dom->vgraph = nullptr;
    dom->prof.drop_graph_records();
    dom->vcycle_calls = 0;
  }
  const bool use_graph = dom->graphs && dom->vcycle_calls > 0;
  dom->vcycle_calls++;
  if (!use_graph) {
    run(s);
    return;
  }
  // capture and replay on a private stream (the caller's may be the legacy default stream, which
  // cannot be captured), ordered after and before the caller's stream with events
  if (!dom->gstream) {
    DG_CUDA(cudaStreamCreateWithFlags(&dom->gstream, cudaStreamNonBlocking));
    DG_CUDA(cudaEventCreateWithFlags(&dom->gev_in, cudaEventDisableTiming));
    DG_CUDA(cudaEventCreateWithFlags(&dom->gev_out, cudaEventDisableTiming));
  }
  cudaStream_t gs = dom->gstream;
  DG_CUDA(cudaEventRecord(dom->gev_in, s));
  DG_CUDA(cudaStreamWaitEvent(gs, dom->gev_in, 0));
  if (!dom->vgraph) {
    cudaGraph_t g = nullptr;
    // with profiling on, the phase events become event-record nodes of the graph
    dom->prof.capturing = prof;
    const int64_t k0 = launches_total();
    DG_CUDA(cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
    try {
      run(gs);
    } catch (...) {
      dom->prof.capturing = false;
      cudaStreamEndCapture(gs, &g);
      if (g) cudaGraphDestroy(g);
      (void)cudaGetLastError();
      throw;
    }
    dom->prof.capturing = false;
    dom->vgraph_kernels = launches_total() - k0;
    count_launches(-dom->vgraph_kernels);  // captured, not launched: counted at each replay
    DG_CUDA(cudaStreamEndCapture(gs, &g));
    cudaError_t e = cudaGraphInstantiate(&dom->vgraph, g, 0);
    cudaGraphDestroy(g);
    DG_CUDA(e);
    dom->vgraph_lin = lin;
    dom->vgraph_m = m;
    dom->vgraph_sub = sub;
    dom->vgraph_prof = prof;
    dom->vgraph_stall = dom->barrier_stall;
  }
  DG_CUDA(cudaGraphLaunch(dom->vgraph, gs));
  count_launches(dom->vgraph_kernels);
  DG_CUDA(cudaEventRecord(dom->gev_out, gs));
  DG_CUDA(cudaStreamWaitEvent(s, dom->gev_out, 0));
  if (prof) {
    // read this replay's event nodes before the next replay records them again
    DG_CUDA(cudaStreamSynchronize(gs));
    dom->prof.add_graph_replay();
  }
}

}  // namespace

// z = M^-1 v in FP64 vectors; mode 0 identity, 1 Schwarz only, 2 V-cycle.
void precondition(dg_domain* dom, int mode, const double* v, double* z, cudaStream_t s) {
  const int64_t n = dom->levels[0].ndof;
  if (mode == 0) {
    DG_CUDA(cudaMemcpyAsync(z, v, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    return;
  }
  const int steps = dom->desc.presmooth + dom->desc.postsmooth;
  if (!dom->mixed) {
    if (mode == 1) {
      DG_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * n, s));
      schwarz_smooth<double>(dom, 0, v, z, steps, true, s);
    } else {
      if (!dom->vin64.get()) {
        dom->vin64.alloc(n);
        dom->vout64.alloc(n);
      }
      DG_CUDA(cudaMemcpyAsync(dom->vin64.get(), v, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      vcycle_fixed(dom, s);
      DG_CUDA(cudaMemcpyAsync(z, dom->vout64.get(), sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    }
    return;
  }
  // mixed: the whole preconditioner in FP32
  if (!dom->vin32.get()) dom->vin32.alloc(2 * n);
  float* v32 = dom->vin32.get();
  float* z32 = v32 + n;
  launch_convert_d2f(n, v, v32, s);
  if (mode == 1) {
    DG_CUDA(cudaMemsetAsync(z32, 0, sizeof(float) * n, s));
    schwarz_smooth<float>(dom, 0, v32, z32, steps, true, s);
  } else {
    vcycle_fixed(dom, s);
  }
  launch_convert_f2d(n, z32, z, s);
}

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Krylov workspace for k iterations: V (k + 1 vectors) and Z (k vectors), grown on demand
// (doubling, contents kept) so that short solves do not hold a basis sized for the iteration cap.
void ensure_workspace(dg_domain* dom, int k) {
  const int64_t n = dom->levels[0].ndof;
  if (!dom->w.get()) {
    dom->w.alloc(n);
    dom->r.alloc(n);
    dom->du.alloc(n);
    dom->ut.alloc(n);
    dom->rt.alloc(n);
    dom->tmp.alloc(n);
  }
  if (dom->kcap >= k) return;
  const int cap = std::max(k, std::min(2 * std::max(dom->kcap, 8), 400));
  DevBuf<double> V((size_t)(cap + 1) * n), Z((size_t)cap * n);
  if (dom->kcap > 0) {
    DG_CUDA(cudaMemcpyAsync(V.get(), dom->V.get(), dom->V.bytes(), cudaMemcpyDeviceToDevice, dom->stream));
    DG_CUDA(cudaMemcpyAsync(Z.get(), dom->Zb.get(), dom->Zb.bytes(), cudaMemcpyDeviceToDevice, dom->stream));
    DG_CUDA(cudaStreamSynchronize(dom->stream));
  }
  dom->V = std::move(V);
  dom->Zb = std::move(Z);
  dom->partial.alloc((size_t)multidot_partial_blocks() * (cap + 2));
  dom->dots.alloc(3 * (size_t)(cap + 2));
  dom->kcap = cap;
}

double norm2(dg_domain* dom, const double* x, cudaStream_t s) {
  const int64_t n = dom->levels[0].ndof;
  launch_multidot(n, 1, x, n, x, dom->partial.get(), dom->dots.get(), s);
  double h;
  DG_CUDA(cudaMemcpyAsync(&h, dom->dots.get(), sizeof(double), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  return std::sqrt(h);
}

struct LinearResult {
  int iterations = 0;
  double r0 = 0, final_res = 0;
  double ref = 0;  // the norm the tolerance is relative to: ||b|| or ||b - A x0||
  dg_status status = DG_OK;
};

// FGMRES on the current operator (dg_apply semantics, linearization included), x updated in place.
// Converged when the Givens estimate reaches tol * ref; the true residual is recomputed at exit.
LinearResult fgmres(dg_domain* dom, const double* b, double* x, double tol, double ref_b_norm, int max_it, int pmode,
                    bool rel_to_b) {
  cudaStream_t s = dom->stream;
  const int64_t n = dom->levels[0].ndof;
  ensure_workspace(dom, std::min(max_it, 16));
  LinearResult R;
  double* w = dom->w.get();
  apply_level(dom, 0, x, dom->r.get(), b, true, s);  // r = b - A x
  const double beta = norm2(dom, dom->r.get(), s);
  R.r0 = beta;
  const double ref = rel_to_b ? ref_b_norm : beta;
  R.ref = ref;
  if (!std::isfinite(beta)) { R.status = DG_ERR_BREAKDOWN; return R; }
  if (beta <= tol * ref || beta == 0.0) { R.final_res = beta; return R; }
  launch_axpby<double>(n, 1.0 / beta, dom->r.get(), 0.0, dom->V.get(), s);
  std::vector<double> H((size_t)(max_it + 1) * max_it, 0.0), cs(max_it), sn(max_it), g(max_it + 1, 0.0);
  g[0] = beta;
  int k = 0;
  std::vector<double> hh(2 * (max_it + 2) + 1);
  for (int j = 0; j < max_it; ++j) {
    if (dom->cancel && dom->cancel->load(std::memory_order_relaxed)) { R.status = DG_ERR_CANCELLED; break; }
    ensure_workspace(dom, j + 1);  // may move V and Z (contents kept)
    double* V = dom->V.get();
    double* Z = dom->Zb.get();
    double* dh = dom->dots.get();  // [h1 (max_it+2) | h2 (max_it+2) | norm]
    if ((int64_t)dom->dots.count < 2 * (max_it + 2) + 1) {
      dom->dots.alloc(2 * (size_t)(max_it + 2) + 1);
      dh = dom->dots.get();
    }
    precondition(dom, pmode, V + (size_t)j * n, Z + (size_t)j * n, s);
    apply_level(dom, 0, Z + (size_t)j * n, w, nullptr, true, s);
    // classical Gram-Schmidt, twice
    PhaseScope ps(dom->prof, DG_PHASE_KRYLOV, s, 8.0 * n * (4.0 * (j + 1) + 5.0), 8.0 * n * (j + 1) + 2.0 * n);
    launch_multidot(n, j + 1, V, n, w, dom->partial.get(), dh, s);
    launch_subtract_combination(n, j + 1, V, n, dh, w, s);
    launch_multidot(n, j + 1, V, n, w, dom->partial.get(), dh + (max_it + 2), s);
    launch_subtract_combination(n, j + 1, V, n, dh + (max_it + 2), w, s);
    launch_multidot(n, 1, w, n, w, dom->partial.get(), dh + 2 * (max_it + 2), s);
    DG_CUDA(cudaMemcpyAsync(hh.data(), dh, sizeof(double) * hh.size(), cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaStreamSynchronize(s));
    double* col = &H[(size_t)j * (max_it + 1)];
    for (int i = 0; i <= j; ++i) col[i] = hh[i] + hh[(max_it + 2) + i];
    const double hn = std::sqrt(std::max(0.0, hh[2 * (max_it + 2)]));
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {  // previous rotations
      const double a = col[i], c = col[i + 1];
      col[i] = cs[i] * a + sn[i] * c;
      col[i + 1] = -sn[i] * a + cs[i] * c;
    }
    const double den = std::hypot(col[j], col[j + 1]);
    if (den == 0.0 || !std::isfinite(den)) { R.status = DG_ERR_BREAKDOWN; break; }
    cs[j] = col[j] / den;
    sn[j] = col[j + 1] / den;
    col[j] = den;
    col[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    k = j + 1;
    const double est = std::fabs(g[j + 1]);
    if (!std::isfinite(est)) { R.status = DG_ERR_BREAKDOWN; break; }
    if (est <= tol * ref || hn == 0.0) break;
    launch_axpby<double>(n, 1.0 / hn, w, 0.0, V + (size_t)(j + 1) * n, s);
  }
  if (k > 0) {
    double* Z = dom->Zb.get();
    double* dh = dom->dots.get();
    std::vector<double> y(k);
    for (int i = k - 1; i >= 0; --i) {
      double acc = g[i];
      for (int l = i + 1; l < k; ++l) acc -= H[(size_t)l * (max_it + 1) + i] * y[l];
      y[i] = acc / H[(size_t)i * (max_it + 1) + i];
    }
    DG_CUDA(cudaMemcpyAsync(dh, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s));
    launch_add_combination(n, k, Z, n, dh, x, s);
  }
  R.iterations = k;
  apply_level(dom, 0, x, dom->r.get(), b, true, s);
  R.final_res = norm2(dom, dom->r.get(), s);
  if (R.status == DG_OK) {
    if (!std::isfinite(R.final_res)) R.status = DG_ERR_BREAKDOWN;
    else if (R.final_res > tol * ref * (1.0 + 1e-6)) R.status = DG_ERR_NOT_CONVERGED;
  }
  return R;
}

// ------------------------------------------------------------------ FGMRES as one CUDA graph
//
// The same method as fgmres() above with the Hessenberg column, the Givens rotations and the
// stopping test on the device (krylov_dev.cu). A solve is one graph launch: prologue (r = b - A x,
// norms, g_0, V_0), a conditional WHILE node whose body is one Arnoldi iteration (V_j into the
// V-cycle's input, the V-cycle itself, Z_j, A Z_j, two classical Gram-Schmidt passes, the rotation
// kernel that sets the loop condition, V_{j+1}), and the epilogue (y = R^-1 g, x += Z y, the true
// residual). The graph works on fixed buffers (b and x are copied in and out around the launch),
// and holds at most kGraphCap Arnoldi columns: a solve that needs more continues host-driven from
// the graph's iterate (a restart).
constexpr int kGraphCap = 40;

// The captured solve's small device arrays, carved from one buffer.
struct KrylovLayout {
  int ldh;
  double *H, *cs, *sn, *g, *y, *h1, *h2, *nrm;  // nrm: [0] ||r||^2 or ||w||^2, [1] ||b||^2, [2] final ||b - A x||^2
  static size_t size(int cap) { return (size_t)(cap + 1) * cap + 3 * (size_t)cap + 3 * (size_t)(cap + 1) + 4; }
  KrylovLayout(double* base, int cap) : ldh(cap + 1) {
    H = base;
    cs = H + (size_t)ldh * cap;
    sn = cs + cap;
    g = sn + cap;
    y = g + cap + 1;
    h1 = y + cap;
    h2 = h1 + cap + 1;
    nrm = h2 + cap + 1;
  }
};

// what the captured kernels depend on besides the buffers' contents
std::vector<int64_t> solve_graph_key(dg_domain* dom, int cap, double tol, bool rel_to_b) {
  int64_t tb = 0;
  std::memcpy(&tb, &tol, sizeof(tb));
  return {cap, tb, rel_to_b ? 1 : 0, dom->mixed ? 1 : 0, dom->lin_set ? 1 : 0, dom->subdomain_iterations,
          dom->subdomain_solver, dom->barrier_stall, (int64_t)(uintptr_t)dom->V.get(),
          (int64_t)(uintptr_t)dom->Zb.get(), dom->desc.presmooth, dom->desc.postsmooth, dom->coarse_fused ? 1 : 0};
}

bool solve_graph_wanted(dg_domain* dom, int pmode) {
  const char* e = std::getenv("DG_SOLVE_GRAPH");
  if (e && std::strcmp(e, "0") == 0) return false;
  return dom->graphs && pmode == 2 && !dom->prof.on;
}

// Arnoldi columns a captured solve holds (DG_SOLVE_GRAPH_CAP overrides, for tests of the restart)
int solve_graph_cap(int max_it) {
  const char* e = std::getenv("DG_SOLVE_GRAPH_CAP");
  const int v = e ? std::atoi(e) : 0;
  return std::min(max_it, v > 0 ? std::min(v, kGraphCap) : kGraphCap);
}

// Buffers, streams and the mapped cancel flag of a captured solve (allocated before any capture).
void prepare_solve_graph(dg_domain* dom, int cap) {
  const int64_t n = dom->levels[0].ndof;
  ensure_workspace(dom, cap);
  if (!dom->gstream) {
    DG_CUDA(cudaStreamCreateWithFlags(&dom->gstream, cudaStreamNonBlocking));
    DG_CUDA(cudaEventCreateWithFlags(&dom->gev_in, cudaEventDisableTiming));
    DG_CUDA(cudaEventCreateWithFlags(&dom->gev_out, cudaEventDisableTiming));
  }
  if (!dom->gstream2) DG_CUDA(cudaStreamCreateWithFlags(&dom->gstream2, cudaStreamNonBlocking));
  if (!dom->cancel_host) {
    DG_CUDA(cudaHostAlloc((void**)&dom->cancel_host, sizeof(int), cudaHostAllocMapped));
    *dom->cancel_host = 0;
    DG_CUDA(cudaHostGetDevicePointer((void**)&dom->cancel_dev, dom->cancel_host, 0));
  }
  if (dom->kr_cap != cap || !dom->kst.get()) {
    dom->kst.alloc(1);
    dom->kbuf.alloc(KrylovLayout::size(cap) + 8);  // + the 8-double report
    dom->kr_cap = cap;
  }
  if (!dom->kb.get()) {
    dom->kb.alloc(n);
    dom->kx.alloc(n);
    dom->zfix.alloc(n);
  }
  if (dom->mixed) {
    if (!dom->vin32.get()) dom->vin32.alloc(2 * n);
  } else if (!dom->vin64.get()) {
    dom->vin64.alloc(n);
    dom->vout64.alloc(n);
  }
}

// Run every kernel shape a captured solve uses once, uncaptured, so that launch shapes are tuned
// and lazily built data exist before the capture (nothing may allocate or tune while capturing).
void warm_solve_kernels(dg_domain* dom) {
  cudaStream_t s = dom->stream;
  const int64_t n = dom->levels[0].ndof;
  DG_CUDA(cudaMemsetAsync(dom->kx.get(), 0, sizeof(double) * n, s));
  DG_CUDA(cudaMemsetAsync(dom->kb.get(), 0, sizeof(double) * n, s));
  apply_level(dom, 0, dom->kx.get(), dom->r.get(), dom->kb.get(), true, s);
  apply_level(dom, 0, dom->kx.get(), dom->w.get(), nullptr, true, s);
  if (dom->mixed) {
    DG_CUDA(cudaMemsetAsync(dom->vin32.get(), 0, sizeof(float) * n, s));
    vcycle<float>(dom, dom->vin32.get(), dom->vin32.get() + n, s);
  } else {
    DG_CUDA(cudaMemsetAsync(dom->vin64.get(), 0, sizeof(double) * n, s));
    vcycle<double>(dom, dom->vin64.get(), dom->vout64.get(), s);
  }
  DG_CUDA(cudaStreamSynchronize(s));
}

// Capture one whole FGMRES solve of `dom` into `graph` as an independent branch: the copies of the
// caller's b and x in (when given), the prologue, the Arnoldi loop as a conditional WHILE node, the
// epilogue, x copied out and the 8-double report written (when given). Counts the branch's kernels
// outside the loop and per loop body into the domain.
void capture_solve_branch(dg_domain* dom, cudaGraph_t graph, int cap, double tol, bool rel_to_b, const double* b_in,
                          double* x_io, double* report) {
  const int64_t n = dom->levels[0].ndof;
  const KrylovLayout kl(dom->kbuf.get(), cap);
  const int ldh = kl.ldh;
  double *H = kl.H, *cs = kl.cs, *sn = kl.sn, *g = kl.g, *y = kl.y, *h1 = kl.h1, *h2 = kl.h2, *nrm = kl.nrm;
  KrylovState* st = dom->kst.get();
  double* V = dom->V.get();
  double* Z = dom->Zb.get();
  double* w = dom->w.get();
  double* r = dom->r.get();
  double* part = dom->partial.get();
  double* kb = dom->kb.get();
  double* kx = dom->kx.get();
  cudaStream_t gs = dom->gstream, bs = dom->gstream2;
  const int64_t k0 = launches_total();
  cudaGraphConditionalHandle loop;
  bool capturing = false;
  try {
    DG_CUDA(cudaGraphConditionalHandleCreate(&loop, graph, 0, cudaGraphCondAssignDefault));
    DG_CUDA(cudaStreamBeginCaptureToGraph(gs, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    capturing = true;
    if (b_in) DG_CUDA(cudaMemcpyAsync(kb, b_in, sizeof(double) * n, cudaMemcpyDeviceToDevice, gs));
    if (x_io) DG_CUDA(cudaMemcpyAsync(kx, x_io, sizeof(double) * n, cudaMemcpyDeviceToDevice, gs));
    apply_level(dom, 0, kx, r, kb, true, gs);  // r = b - A x
    launch_multidot(n, 1, r, n, r, part, nrm, gs);
    if (rel_to_b) launch_multidot(n, 1, kb, n, kb, part, nrm + 1, gs);
    launch_kr_start(st, tol, cap, rel_to_b, nrm, g, loop, gs);
    launch_kr_scale_into_v(n, r, st, V, n, gs);
    // the Arnoldi loop: a conditional WHILE node after the prologue
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    DG_CUDA(cudaStreamGetCaptureInfo(gs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps));
    DG_REQUIRE(cst == cudaStreamCaptureStatusActive, "solve capture was invalidated before the Arnoldi loop");
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = loop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    DG_CUDA(cudaGraphAddNode(&cnode, graph, deps, nullptr, ndeps, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    DG_CUDA(cudaStreamUpdateCaptureDependencies(gs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    DG_CUDA(cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const int64_t kb0 = launches_total();
    try {
      if (dom->mixed) {
        float* v32 = dom->vin32.get();
        launch_kr_load_v<float>(n, V, n, st, v32, bs);
        vcycle<float>(dom, v32, v32 + n, bs);
        launch_kr_store_z<float>(n, v32 + n, st, Z, n, dom->zfix.get(), bs);
      } else {
        launch_kr_load_v<double>(n, V, n, st, dom->vin64.get(), bs);
        vcycle<double>(dom, dom->vin64.get(), dom->vout64.get(), bs);
        launch_kr_store_z<double>(n, dom->vout64.get(), st, Z, n, dom->zfix.get(), bs);
      }
      apply_level(dom, 0, dom->zfix.get(), w, nullptr, true, bs);
      launch_kr_multidot(n, cap, V, n, w, st, part, h1, bs);  // classical Gram-Schmidt, twice
      launch_kr_sub_comb(n, V, n, h1, st, w, bs);
      launch_kr_multidot(n, cap, V, n, w, st, part, h2, bs);
      launch_kr_sub_comb(n, V, n, h2, st, w, bs);
      launch_multidot(n, 1, w, n, w, part, nrm, bs);
      launch_kr_givens(st, H, ldh, cs, sn, g, h1, h2, nrm, dom->cancel_dev, loop, bs);
      launch_kr_scale_into_v(n, w, st, V, n, bs);
    } catch (...) {
      cudaGraph_t t = nullptr;
      cudaStreamEndCapture(bs, &t);
      throw;
    }
    dom->sgraph_body_kernels = launches_total() - kb0;
    cudaStreamCaptureStatus bst = cudaStreamCaptureStatusNone;
    DG_CUDA(cudaStreamIsCapturing(bs, &bst));
    cudaGraph_t t = nullptr;
    DG_CUDA(cudaStreamEndCapture(bs, &t));
    DG_REQUIRE(bst == cudaStreamCaptureStatusActive, "capture of the Arnoldi loop body was invalidated");
    // epilogue
    launch_kr_trisolve(st, H, ldh, g, y, gs);
    launch_kr_add_comb(n, Z, n, y, st, kx, gs);
    apply_level(dom, 0, kx, r, kb, true, gs);
    launch_multidot(n, 1, r, n, r, part, nrm + 2, gs);
    if (x_io) DG_CUDA(cudaMemcpyAsync(x_io, kx, sizeof(double) * n, cudaMemcpyDeviceToDevice, gs));
    if (report) launch_kr_report(st, nrm, report, gs);
    capturing = false;
    DG_CUDA(cudaStreamEndCapture(gs, &t));
  } catch (...) {
    if (capturing) {
      cudaGraph_t t = nullptr;
      cudaStreamEndCapture(gs, &t);
    }
    (void)cudaGetLastError();
    count_launches(-(launches_total() - k0));
    throw;
  }
  dom->sgraph_fixed_kernels = launches_total() - k0 - dom->sgraph_body_kernels;
  count_launches(-(launches_total() - k0));  // captured, not launched: counted per execution
}

void build_solve_graph(dg_domain* dom, int cap, double tol, bool rel_to_b) {
  prepare_solve_graph(dom, cap);
  warm_solve_kernels(dom);
  if (tune_log())
    std::fprintf(stderr, "dg solve graph: capturing (n_dof %lld, %d columns, %s)\n", (long long)dom->levels[0].ndof,
                 cap, dom->mixed ? "mixed" : "fp64");
  if (dom->sgraph) {
    cudaGraphExecDestroy(dom->sgraph);
    dom->sgraph = nullptr;
  }
  cudaGraph_t graph = nullptr;
  DG_CUDA(cudaGraphCreate(&graph, 0));
  try {
    capture_solve_branch(dom, graph, cap, tol, rel_to_b, nullptr, nullptr,
                         dom->kbuf.get() + KrylovLayout::size(cap));
    DG_CUDA(cudaGraphInstantiate(&dom->sgraph, graph, 0));
  } catch (const Error& e) {
    if (tune_log()) std::fprintf(stderr, "dg solve graph: capture failed: %s\n", e.message.c_str());
    cudaGraphDestroy(graph);
    throw;
  }
  cudaGraphDestroy(graph);
  if (tune_log())
    std::fprintf(stderr, "dg solve graph: built (%lld kernels outside the loop, %lld per iteration)\n",
                 (long long)dom->sgraph_fixed_kernels, (long long)dom->sgraph_body_kernels);
}

// A solve's result from its 8-double report (see launch_kr_report).
LinearResult result_from_report(const double* rp) {
  LinearResult R;
  R.iterations = (int)rp[0];
  R.r0 = rp[3];
  R.ref = rp[4];
  R.final_res = rp[5];
  const int status = (int)rp[1];
  R.status = DG_OK;
  if (status == KR_BREAKDOWN) R.status = DG_ERR_BREAKDOWN;
  else if (status == KR_CANCELLED) R.status = DG_ERR_CANCELLED;
  else if (!std::isfinite(R.final_res)) R.status = DG_ERR_BREAKDOWN;
  else if (R.final_res > rp[6] * (1.0 + 1e-6)) R.status = DG_ERR_NOT_CONVERGED;
  return R;
}

// One linear solve through the captured graph; returns false (nothing done) where the graph path
// does not apply, so that the caller runs the host-driven solver instead.
bool fgmres_graph(dg_domain* dom, const double* b, double* x, double tol, int max_it, int pmode, bool rel_to_b,
                  LinearResult& R) {
  if (!solve_graph_wanted(dom, pmode)) return false;
  const int cap = solve_graph_cap(max_it);
  if (cap < 1) return false;
  cudaStream_t s = dom->stream;
  const int64_t n = dom->levels[0].ndof;
  ensure_workspace(dom, cap);
  const std::vector<int64_t> key = solve_graph_key(dom, cap, tol, rel_to_b);
  if (!dom->sgraph || dom->sgraph_key != key) {
    if (dom->skey_seen != key) {  // first solve with these kernels: host-driven (tunes and allocates)
      dom->skey_seen = key;
      return false;
    }
    try {
      build_solve_graph(dom, cap, tol, rel_to_b);
    } catch (const Error&) {
      // the capture did not work out: this domain solves host-driven from now on
      (void)cudaGetLastError();
      DG_CUDA(cudaStreamSynchronize(s));
      dom->graphs = false;
      return false;
    }
    dom->sgraph_key = key;
  }
  *reinterpret_cast<volatile int*>(dom->cancel_host) = 0;
  DG_CUDA(cudaMemcpyAsync(dom->kb.get(), b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  DG_CUDA(cudaMemcpyAsync(dom->kx.get(), x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  DG_CUDA(cudaGraphLaunch(dom->sgraph, s));
  DG_CUDA(cudaMemcpyAsync(x, dom->kx.get(), sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  if (dom->cancel) {
    // keep a cancel request visible to the rotation kernel while the solve runs
    DG_CUDA(cudaEventRecord(dom->gev_out, s));
    for (;;) {
      const cudaError_t q = cudaEventQuery(dom->gev_out);
      if (q == cudaSuccess) break;
      if (q != cudaErrorNotReady) DG_CUDA(q);
      if (dom->cancel->load(std::memory_order_relaxed)) *reinterpret_cast<volatile int*>(dom->cancel_host) = 1;
      std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
  }
  double rp[8];
  DG_CUDA(cudaMemcpyAsync(rp, dom->kbuf.get() + KrylovLayout::size(cap), sizeof(rp), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  count_launches(dom->sgraph_fixed_kernels + (int64_t)rp[2] * dom->sgraph_body_kernels);
  R = result_from_report(rp);
  if ((int)rp[1] == KR_CAP && max_it > cap) {
    // more columns than the graph holds: continue host-driven from this iterate (a restart)
    const double r0 = R.r0, ref = R.ref;
    LinearResult more = fgmres(dom, b, x, rp[6] / std::max(ref, 1e-300), ref, max_it - cap, pmode, true);
    R = more;
    R.iterations += cap;
    R.r0 = r0;
    R.ref = ref;
  }
  return true;
}

}  // namespace
}  // namespace dg

// ------------------------------------------------------------------ many solves in one graph launch

struct dg_batch {
  std::vector<dg_domain*> doms;
  cudaGraphExec_t exec = nullptr;
  dg::DevBuf<double> reports;  // 8 doubles per solve
  std::vector<int64_t> fixed, body;
  int cap = 0;
  ~dg_batch() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

namespace dg {

dg_batch* batch_create(dg_domain* const* doms, const double* const* b, double* const* u, int count, double tol,
                       const dg_solve_opts& o) {
  DG_REQUIRE(count >= 1, "batch needs at least one solve");
  const int max_it = o.max_iterations > 0 ? o.max_iterations : 200;
  DG_REQUIRE(o.krylov == 0 && o.precondition == 2, "a batch runs FGMRES with the multigrid preconditioner");
  DG_REQUIRE(tol > 0 && std::isfinite(tol), "tol must be positive");
  std::unique_ptr<dg_batch> bt(new dg_batch());
  bt->cap = std::min(max_it, kGraphCap);
  bt->reports.alloc(8 * (size_t)count);
  for (int i = 0; i < count; ++i) {
    dg_domain* dom = doms[i];
    DG_REQUIRE(dom && b[i] && u[i], "null domain or vector in the batch");
    DG_REQUIRE(dom->desc.problem == DG_PROBLEM_POISSON, "a batch holds Poisson problems");
    for (int j = 0; j < i; ++j) DG_REQUIRE(doms[j] != dom, "a domain appears twice in the batch");
    dom->lin_set = false;
    dom->barrier_stall = 0;
    prepare_solve_graph(dom, bt->cap);
    warm_solve_kernels(dom);
  }
  cudaGraph_t graph = nullptr;
  DG_CUDA(cudaGraphCreate(&graph, 0));
  try {
    for (int i = 0; i < count; ++i) {
      capture_solve_branch(doms[i], graph, bt->cap, tol, o.relative_to_b != 0, b[i], u[i],
                           bt->reports.get() + 8 * (size_t)i);
      bt->fixed.push_back(doms[i]->sgraph_fixed_kernels);
      bt->body.push_back(doms[i]->sgraph_body_kernels);
    }
    DG_CUDA(cudaGraphInstantiate(&bt->exec, graph, 0));
  } catch (...) {
    cudaGraphDestroy(graph);
    throw;
  }
  cudaGraphDestroy(graph);
  bt->doms.assign(doms, doms + count);
  return bt.release();
}

void batch_run(dg_batch* bt, cudaStream_t s, dg_solve_report* reps) {
  const size_t count = bt->doms.size();
  for (dg_domain* d : bt->doms) *reinterpret_cast<volatile int*>(d->cancel_host) = 0;
  DG_CUDA(cudaGraphLaunch(bt->exec, s));
  std::vector<double> rp(8 * count);
  DG_CUDA(cudaMemcpyAsync(rp.data(), bt->reports.get(), sizeof(double) * rp.size(), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  int64_t k = 0;
  for (size_t i = 0; i < count; ++i) {
    k += bt->fixed[i] + (int64_t)rp[8 * i + 2] * bt->body[i];
    if (!reps) continue;
    const LinearResult L = result_from_report(&rp[8 * i]);
    dg_solve_report R{};
    R.iterations = L.iterations;
    R.initial_residual = L.r0;
    R.final_residual = L.final_res;
    R.relative_residual = L.ref > 0 ? L.final_res / L.ref : 0.0;
    R.status = L.status;
    reps[i] = R;
  }
  count_launches(k);
}

void batch_destroy(dg_batch* bt) {
  // every run waited for its launch, so nothing of the graph is in flight; the domains are not
  // touched (they may already be gone)
  delete bt;
}

namespace {

// Flexible conjugate gradients (the SPD alternative to FGMRES): one search direction, made
// A-orthogonal to the previous one after every (possibly non-symmetric) V-cycle. Three host reads
// per iteration: z.A p_old, (p.r, p.A p), ||r||. Vectors r and q = A p sit next to each other in
// the Krylov buffer so that p.r and p.q are one two-vector reduction.
LinearResult fcg(dg_domain* dom, const double* b, double* x, double tol, double ref_b_norm, int max_it, int pmode,
                 bool rel_to_b) {
  cudaStream_t s = dom->stream;
  const int64_t n = dom->levels[0].ndof;
  ensure_workspace(dom, 4);
  LinearResult R;
  double* r = dom->V.get();
  double* q = r + n;
  double* z = r + 2 * n;
  double* p = r + 3 * n;
  double* dh = dom->dots.get();
  auto read = [&](int cnt, double* out) {
    DG_CUDA(cudaMemcpyAsync(out, dh, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaStreamSynchronize(s));
  };
  apply_level(dom, 0, x, r, b, true, s);  // r = b - A x
  const double beta = norm2(dom, r, s);
  R.r0 = beta;
  const double ref = rel_to_b ? ref_b_norm : beta;
  R.ref = ref;
  if (!std::isfinite(beta)) { R.status = DG_ERR_BREAKDOWN; return R; }
  double res = beta, pq_old = 0.0;
  for (int k = 0; k < max_it && res > tol * ref && res > 0.0; ++k) {
    if (dom->cancel && dom->cancel->load(std::memory_order_relaxed)) { R.status = DG_ERR_CANCELLED; break; }
    precondition(dom, pmode, r, z, s);
    if (k == 0) {
      DG_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    } else {
      launch_multidot(n, 1, q, n, z, dom->partial.get(), dh, s);  // z . A p_old
      double zq;
      read(1, &zq);
      launch_axpby<double>(n, 1.0, z, -zq / pq_old, p, s);  // p = z - (z.q_old / p_old.q_old) p_old
    }
    apply_level(dom, 0, p, q, nullptr, true, s);  // q = A p
    double pr_pq[2];
    {
      PhaseScope ps(dom->prof, DG_PHASE_KRYLOV, s, 8.0 * n * 7.0, 8.0 * n * 4.0);
      launch_multidot(n, 2, r, n, p, dom->partial.get(), dh, s);  // [p.r, p.q]
      read(2, pr_pq);
    }
    if (!(pr_pq[1] > 0.0) || !std::isfinite(pr_pq[0])) { R.status = DG_ERR_BREAKDOWN; break; }
    const double alpha = pr_pq[0] / pr_pq[1];
    launch_axpby<double>(n, alpha, p, 1.0, x, s);
    launch_axpby<double>(n, -alpha, q, 1.0, r, s);
    pq_old = pr_pq[1];
    res = norm2(dom, r, s);
    R.iterations = k + 1;
    if (!std::isfinite(res)) { R.status = DG_ERR_BREAKDOWN; break; }
  }
  apply_level(dom, 0, x, dom->r.get(), b, true, s);
  R.final_res = norm2(dom, dom->r.get(), s);
  if (R.status == DG_OK) {
    if (!std::isfinite(R.final_res)) R.status = DG_ERR_BREAKDOWN;
    else if (R.final_res > tol * ref * (1.0 + 1e-6)) R.status = DG_ERR_NOT_CONVERGED;
  }
  return R;
}

// Inverses of A_S + D_S for every finest-level subdomain at the current linearization: the class
// matrices A_S at the actual element widths (built once), d_S = R_S (M S'(u)) gathered into the
// subdomain columns, M_c = A_S + diag(d_S) per column, then batched in-place Gauss-Jordan.
template <typename T>
void build_linearized_inverses(dg_domain* dom, cudaStream_t s) {
  ensure_schwarz(dom, 0);
  Level& L = dom->levels[0];
  SchwarzLevel& sw = L.sw;
  LevelWork<T>& W = work<T>(L);
  const int nS = sw.nS, ld = sw.ld, E = L.E, nc = sw.n_classes, N = dom->N;
  const size_t n2 = (size_t)nS * nS;
  const T* Dt;
  const T* wt;
  if constexpr (std::is_same<T, float>::value) { Dt = dom->D32.get(); wt = dom->w32.get(); }
  else { Dt = dom->D64.get(); wt = dom->w64.get(); }
  if (!W.linA.get()) {
    DevBuf<int> d_patch(sw.patch.size());
    DG_CUDA(cudaMemcpyAsync(d_patch.get(), sw.patch.data(), sizeof(int) * sw.patch.size(), cudaMemcpyHostToDevice, s));
    const OpGeom<T> g = make_geom<T>(L.n, L.h, N, dom->desc.penalty, dom->lgl);
    W.linA.alloc((size_t)nc * n2);
    launch_build_subdomain_matrices<T>(N, dom->desc.overlap, g, Dt, wt, d_patch.get(), nc, nS, W.linA.get(), s);
    DG_CUDA(cudaStreamSynchronize(s));
  }
  if (W.linv.count < (size_t)E * n2) W.linv.alloc((size_t)E * n2);
  if (W.gD.count < (size_t)E * ld) W.gD.alloc((size_t)E * ld);
  const double sz = sizeof(T);
  PhaseScope ps(dom->prof, DG_PHASE_SUBDOMAIN_BUILD, s, 3.0 * E * n2 * sz, 2.0 * E * (double)n2 * nS);
  launch_gather_tab<T>(sw.geom, lin_diag<T>(dom), sw.elem_of_col.get(), sw.xform_of_elem.get(), dom->orient_map.get(),
                       W.gD.get(), s);
  launch_lin_assemble<T>(W.linA.get(), sw.class_of_col.get(), W.gD.get(), nS, ld, E, W.linv.get(), s);
  constexpr int kMaxBatch = 65535;  // grid z limit of the Gauss-Jordan update kernel
  for (int c0 = 0; c0 < E; c0 += kMaxBatch)
    launch_invert_spd_batched<T>(W.linv.get() + (size_t)c0 * n2, nS, std::min(kMaxBatch, E - c0), s);
}

void build_linearized(dg_domain* dom, cudaStream_t s) {
  dom->linv_current = false;
  if (dom->mixed) build_linearized_inverses<float>(dom, s);
  else build_linearized_inverses<double>(dom, s);
  dom->linv_current = true;
}

void set_linearization(dg_domain* dom, const double* u, cudaStream_t s) {
  launch_puncture_linearization(dom->levels[0].ndof, u, dom->mass.get(), dom->alpha.get(), dom->beta.get(),
                                dom->lin64.get(), dom->lin32.get(), s);
  dom->lin_set = true;
  dom->linv_current = false;
  if (dom->subdomain_solver == 1) build_linearized(dom, s);
}

// r = b - A(u)
void nonlinear_residual(dg_domain* dom, const double* u, const double* b, double* r, cudaStream_t s) {
  const bool was = dom->lin_set;
  dom->lin_set = false;
  apply_level(dom, 0, u, dom->tmp.get(), nullptr, false, s);
  dom->lin_set = was;
  launch_puncture_residual(dom->levels[0].ndof, dom->tmp.get(), u, b, dom->mass.get(), dom->alpha.get(),
                           dom->beta.get(), r, s);
}

}  // namespace

void puncture_residual_api(dg_domain* dom, const double* u, const double* b, double* r, cudaStream_t s) {
  ensure_workspace(dom, 1);
  nonlinear_residual(dom, u, b, r, s);
}
void puncture_linearize_api(dg_domain* dom, const double* u, cudaStream_t s) {
  if (!u) { dom->lin_set = false; dom->linv_current = false; return; }
  set_linearization(dom, u, s);
}
void subdomain_solver_api(dg_domain* dom, int solver, int iterations, cudaStream_t s) {
  DG_REQUIRE(solver == 0 || solver == 1, "subdomain solver must be 0 (GMRES) or 1 (per-subdomain inverses)");
  DG_REQUIRE(iterations >= 0 && iterations <= 16, "subdomain_iterations must be in [0, 16]");
  dom->subdomain_solver = solver;
  dom->subdomain_iterations = iterations;
  if (solver == 1 && dom->lin_set && !dom->linv_current) build_linearized(dom, s);
}

dg_status solve(dg_domain* dom, const double* b, double* u, double tol, const dg_solve_opts& o, dg_solve_report* rep) {
  const double t0 = now_s();
  cudaStream_t s = dom->stream;
  const int64_t n = dom->levels[0].ndof;
  const int max_it = o.max_iterations > 0 ? o.max_iterations : 200;
  const int pmode = o.precondition;
  DG_REQUIRE(pmode >= 0 && pmode <= 2, "precondition must be 0, 1 or 2");
  DG_REQUIRE(o.krylov == 0 || o.krylov == 1, "krylov must be 0 (FGMRES) or 1 (flexible CG)");
  DG_REQUIRE(!dom->mapped || o.krylov == 0, "flexible CG needs a symmetric operator; curved elements are not");
  DG_REQUIRE(tol > 0 && std::isfinite(tol), "tol must be positive");
  {
    const char* e = std::getenv("DG_TEST_BARRIER_STALL");
    dom->barrier_stall = (e && std::strcmp(e, "1") == 0) ? 1 : 0;
  }
  ensure_workspace(dom, std::min(max_it, 16));
  dg_solve_report R{};
  if (dom->desc.problem == DG_PROBLEM_POISSON) {
    dom->lin_set = false;
    LinearResult L;
    if (o.krylov == 1 || !fgmres_graph(dom, b, u, tol, max_it, pmode, o.relative_to_b != 0, L)) {
      const double bn = o.relative_to_b ? norm2(dom, b, s) : 0.0;
      L = o.krylov == 1 ? fcg(dom, b, u, tol, bn, max_it, pmode, o.relative_to_b != 0)
                        : fgmres(dom, b, u, tol, bn, max_it, pmode, o.relative_to_b != 0);
    }
    R.iterations = L.iterations;
    R.initial_residual = L.r0;
    R.final_residual = L.final_res;
    R.relative_residual = L.ref > 0 ? L.final_res / L.ref : 0.0;
    R.status = L.status;
  } else {
    // Newton-Raphson with line search (sufficient decrease c = 1e-4, quadratic backtracking)
    const double c = 1e-4;
    const double lin_tol = o.linear_tol > 0 ? o.linear_tol : 1e-4;
    const int max_steps = o.max_newton_steps > 0 ? o.max_newton_steps : 20;
    DG_REQUIRE(o.subdomain_solver == 0 || o.subdomain_solver == 1, "subdomain_solver must be 0 or 1");
    dom->subdomain_iterations = o.subdomain_iterations >= 0 ? o.subdomain_iterations : 3;
    DG_REQUIRE(dom->subdomain_iterations <= 16, "subdomain_iterations must be at most 16");
    dom->subdomain_solver = o.subdomain_solver;
    double* r = dom->rt.get();
    nonlinear_residual(dom, u, b, r, s);
    double rn = norm2(dom, r, s);
    const double r0 = rn;
    const double ref = (o.relative_to_b && b) ? norm2(dom, b, s) : r0;
    R.initial_residual = r0;
    R.status = DG_OK;
    if (!std::isfinite(rn)) R.status = DG_ERR_BREAKDOWN;
    int step = 0;
    while (R.status == DG_OK && rn > tol * ref && rn > 0.0) {
      if (step >= max_steps) { R.status = DG_ERR_NOT_CONVERGED; break; }
      set_linearization(dom, u, s);
      DG_CUDA(cudaMemsetAsync(dom->du.get(), 0, sizeof(double) * n, s));
      // the linear right-hand side is r (copied: the Krylov solver overwrites dom->r)
      DG_CUDA(cudaMemcpyAsync(dom->ut.get(), r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      LinearResult L;
      if (o.krylov == 1 || !fgmres_graph(dom, dom->ut.get(), dom->du.get(), lin_tol, max_it, pmode, false, L))
        L = o.krylov == 1 ? fcg(dom, dom->ut.get(), dom->du.get(), lin_tol, 0.0, max_it, pmode, false)
                          : fgmres(dom, dom->ut.get(), dom->du.get(), lin_tol, 0.0, max_it, pmode, false);
      R.iterations += L.iterations;
      if (L.status == DG_ERR_BREAKDOWN || L.status == DG_ERR_CANCELLED) { R.status = L.status; break; }
      double lam = 1.0, rn_new = 0.0;
      for (int bt = 0; bt <= 10; ++bt) {
        DG_CUDA(cudaMemcpyAsync(dom->ut.get(), u, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        launch_axpby<double>(n, lam, dom->du.get(), 1.0, dom->ut.get(), s);
        nonlinear_residual(dom, dom->ut.get(), b, r, s);
        rn_new = norm2(dom, r, s);
        if (std::isfinite(rn_new) && rn_new <= (1.0 - c * lam) * rn) break;
        const double g0 = 0.5 * rn * rn, g1 = 0.5 * rn_new * rn_new, dg0 = -rn * rn;
        double lq = std::isfinite(g1) ? -dg0 * lam * lam / (2.0 * (g1 - g0 - dg0 * lam)) : 0.1 * lam;
        lam = std::min(std::max(lq, 0.1 * lam), 0.5 * lam);
        R.line_search_steps++;
      }
      DG_CUDA(cudaMemcpyAsync(u, dom->ut.get(), sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      rn = rn_new;
      ++step;
      if (!std::isfinite(rn)) R.status = DG_ERR_BREAKDOWN;
    }
    dom->lin_set = false;
    dom->linv_current = false;
    R.newton_steps = step;
    R.final_residual = rn;
    R.relative_residual = ref > 0 ? rn / ref : 0.0;
  }
  int flag = 0;
  DG_CUDA(cudaMemcpyAsync(&flag, dom->err_flag.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  if (flag) {
    DG_CUDA(cudaMemsetAsync(dom->err_flag.get(), 0, sizeof(int), s));
    R.status = DG_ERR_TIMEOUT;
  }
  R.seconds = now_s() - t0;
  if (rep) *rep = R;
  return (dg_status)R.status;
}

}  // namespace dg

namespace dg {

cudaEvent_t Profiler::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  DG_CUDA(cudaEventCreate(&e));
  return e;
}

void Profiler::clear() {
  for (auto& r : pending) {
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  pending.clear();
  for (auto& a : acc) a = dg_phase_stats{};
}

void Profiler::drop_graph_records() {
  for (auto& r : graph_recs) {
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  graph_recs.clear();
  for (auto& a : graph_acc) a = dg_phase_stats{};
}

void Profiler::add_graph_replay() {
  for (auto& r : graph_recs) {
    float ms = 0;
    DG_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    acc[r.phase].milliseconds += ms;
  }
  for (int i = 0; i < DG_PHASE_COUNT; ++i) {
    acc[i].launches += graph_acc[i].launches;
    acc[i].bytes += graph_acc[i].bytes;
    acc[i].flops += graph_acc[i].flops;
  }
}

Profiler::~Profiler() {
  for (auto* v : {&pending, &graph_recs})
    for (auto& r : *v) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
  for (auto e : pool) cudaEventDestroy(e);
}

PhaseScope::PhaseScope(Profiler& p, int phase, cudaStream_t s, double bytes, double flops)
    : p_(p), phase_(phase), s_(s) {
  if (!p_.on) return;
  dg_phase_stats& st = p_.capturing ? p_.graph_acc[phase] : p_.acc[phase];
  st.launches++;
  st.bytes += bytes;
  st.flops += flops;
  a_ = p_.get();
  // inside stream capture only an "external" record becomes an event-record node of the graph
  if (p_.capturing) DG_CUDA(cudaEventRecordWithFlags(a_, s_, cudaEventRecordExternal));
  else DG_CUDA(cudaEventRecord(a_, s_));
}

PhaseScope::~PhaseScope() {
  if (!a_) return;
  cudaEvent_t b = nullptr;
  if (!p_.pool.empty()) {
    b = p_.pool.back();
    p_.pool.pop_back();
  } else if (cudaEventCreate(&b) != cudaSuccess) {
    (void)cudaGetLastError();
    p_.pool.push_back(a_);  // drop this record rather than throw from a destructor
    return;
  }
  const cudaError_t e =
      p_.capturing ? cudaEventRecordWithFlags(b, s_, cudaEventRecordExternal) : cudaEventRecord(b, s_);
  if (e != cudaSuccess) (void)cudaGetLastError();
  (p_.capturing ? p_.graph_recs : p_.pending).push_back({a_, b, phase_});
}

void profile_read(dg_domain* dom, dg_phase_stats* out) {
  Profiler& p = dom->prof;
  for (auto& r : p.pending) {
    DG_CUDA(cudaEventSynchronize(r.b));
    float ms = 0;
    DG_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    p.acc[r.phase].milliseconds += ms;
    p.pool.push_back(r.a);
    p.pool.push_back(r.b);
  }
  p.pending.clear();
  for (int i = 0; i < DG_PHASE_COUNT; ++i) out[i] = p.acc[i];
}

}  // namespace dg
