// extern "C" entry points: argument checks, stream selection, and translation of exceptions
// thrown by the setup/orchestration code into dg_status codes with a per-handle message.
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "domain.h"

namespace dg {

void fail(dg_status st, const std::string& msg) { throw Error{st, msg}; }

void cuda_check(cudaError_t e, const char* what, const char* file, int line) {
  if (e == cudaSuccess) return;
  (void)cudaGetLastError();
  fail(DG_ERR_CUDA, std::string(what) + " failed at " + file + ":" + std::to_string(line) + ": " +
                        cudaGetErrorString(e));
}

namespace {
std::atomic<int64_t> g_launches{0};
}
void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
int64_t launches_total() { return g_launches.load(std::memory_order_relaxed); }

void puncture_residual_api(dg_domain* dom, const double* u, const double* b, double* r, cudaStream_t s);
void puncture_linearize_api(dg_domain* dom, const double* u, cudaStream_t s);
void subdomain_solver_api(dg_domain* dom, int solver, int iterations, cudaStream_t s);

namespace {
// The last error of a call that has no domain handle to hold it (a failed dg_domain_create, any
// dg_dot_noalloc call), per thread: every such call overwrites it, so dg_last_error(NULL) always
// describes the latest of them.
thread_local std::string g_null_handle_error;
}  // namespace

void set_null_handle_error(const std::string& msg) { g_null_handle_error = msg; }
const char* null_handle_error() { return g_null_handle_error.c_str(); }

}  // namespace dg

namespace {

template <typename F>
dg_status guarded(dg_domain* dom, F&& f) {
  try {
    dg::AllocStreamScope scope(dom ? dom->stream : nullptr);
    f();
    if (dom) dom->err.clear();
    return DG_OK;
  } catch (const dg::Error& e) {
    if (dom) dom->err = e.message;
    return e.status;
  } catch (const std::bad_alloc&) {
    if (dom) dom->err = "host allocation failed";
    return DG_ERR_OOM;
  } catch (const std::exception& e) {
    if (dom) dom->err = e.what();
    return DG_ERR_INVALID_ARG;
  }
}

cudaStream_t pick(dg_domain* dom, void* stream) { return stream ? (cudaStream_t)stream : dom->stream; }

void check_level(const dg_domain* dom, int level) {
  DG_REQUIRE(level >= 0 && level < (int)dom->levels.size(), "level out of range");
}

}  // namespace

namespace dg {
// readers of the per-module bounds-check words (debug builds; see bounds.cuh)
std::vector<int (*)()>& oob_readers() {
  static std::vector<int (*)()> r;
  return r;
}
int register_oob_reader(int (*reader)()) {
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  oob_readers().push_back(reader);
  return (int)oob_readers().size();
}
}  // namespace dg

extern "C" {

dg_status dg_domain_create(const dg_domain_desc* desc, void* cuda_stream, dg_domain** out) {
  if (!desc || !out) {
    dg::set_null_handle_error("dg_domain_create: null descriptor or output pointer");
    return DG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  dg::set_null_handle_error("");
  dg_domain* dom = nullptr;
  try {
    dom = new dg_domain();
  } catch (...) {
    dg::set_null_handle_error("dg_domain_create: host allocation failed");
    return DG_ERR_OOM;
  }
  dom->desc = *desc;
  // NULL selects the legacy default stream (the one torch and most callers use by default)
  dom->stream = (cudaStream_t)cuda_stream;
  dg_status st = guarded(dom, [&] {
    dg::domain_setup(dom);
    dom->bytes = dg::domain_device_bytes(dom);
  });
  if (st != DG_OK) {
    dg::set_null_handle_error(dom->err);
    dg_domain_destroy(dom);
    return st;
  }
  *out = dom;
  return DG_OK;
}

void dg_domain_destroy(dg_domain* dom) {
  if (!dom) return;
  // buffers are released in the order of the domain's stream, after its work and that of its
  // private graph stream
  if (dom->gstream) cudaStreamSynchronize(dom->gstream);
  cudaStreamSynchronize(dom->stream);
  cudaStream_t s = dom->own_stream ? dom->stream : nullptr;
  delete dom;
  if (s) cudaStreamDestroy(s);
}

int32_t dg_debug_bounds_check(void) {
#ifdef DG_BOUNDS_CHECK
  if (cudaDeviceSynchronize() != cudaSuccess) return 0;
  int first = 0;
  for (auto reader : dg::oob_readers()) {
    const int line = reader();
    if (line && !first) first = line;
  }
  return first;
#else
  return -1;
#endif
}

const char* dg_last_error(const dg_domain* dom) {
  if (!dom) return dg::null_handle_error();
  return dom->err.c_str();
}

dg_status dg_domain_layout(const dg_domain* dom, dg_layout* out) {
  if (!dom || !out) return DG_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  const auto& L0 = dom->levels[0];
  out->n_dof = L0.ndof;
  out->n_elements = L0.E;
  out->N = dom->N;
  for (int i = 0; i < 3; ++i) out->n[i] = L0.n[i];
  out->mg_levels = (int32_t)dom->levels.size();
  for (size_t l = 0; l < dom->levels.size(); ++l) {
    for (int i = 0; i < 3; ++i) out->level_n[l][i] = dom->levels[l].n[i];
    out->n_classes[l] = dom->levels[l].sw.n_classes;
  }
  out->subdomain_size = L0.sw.nS;
  out->x = dom->X.get();
  out->y = dom->Y.get();
  out->z = dom->Z.get();
  out->device_bytes = dg::domain_device_bytes(dom);
  return DG_OK;
}

dg_status dg_apply(dg_domain* dom, const double* u, double* Au, void* stream) {
  if (!dom) return DG_ERR_INVALID_ARG;
  return guarded(dom, [&] {
    DG_REQUIRE(u && Au && u != Au, "u and Au must be distinct device pointers");
    dg::apply_level(dom, 0, u, Au, nullptr, true, pick(dom, stream));
  });
}

dg_status dg_apply_level(dg_domain* dom, int32_t level, const double* u, double* Au, void* stream) {
  if (!dom) return DG_ERR_INVALID_ARG;
  return guarded(dom, [&] {
    check_level(dom, level);
    DG_REQUIRE(u && Au && u != Au, "u and Au must be distinct device pointers");
    dg::apply_level(dom, level, u, Au, nullptr, true, pick(dom, stream));
  });
}

dg_status dg_apply_f32(dg_domain* dom, int32_t level, const float* u, float* Au, void* stream) {
  if (!dom) return DG_ERR_INVALID_ARG;
  return guarded(dom, [&] {
    check_level(dom, level);
    DG_REQUIRE(u && Au && u != Au, "u and Au must be distinct device pointers");
    DG_REQUIRE(!(level == 0 && dom->lin_set && !dom->lin32.get()),
               "the FP32 linearized operator needs a MIXED domain");
    dg::apply_level_f32(dom, level, u, Au, nullptr, true, pick(dom, stream));
  });
}

dg_status dg_rhs(dg_domain* dom, const double* f, double* b, void* stream) {
  if (!dom) return DG_ERR_INVALID_ARG;
  return guarded(dom, [&] {
    DG_REQUIRE(f && b, "null pointer");
    dg::launch_scale_mul(dom->levels[0].ndof, dom->mass.get(), f, b, pick(dom, stream));
  });
}

dg_status dg_mg_restrict(dg_domain* dom, int32_t level, const double* r_fine, double* b_coarse, void* stream) {
  if (!dom) return DG_ERR_INVALID_ARG;
  return guarded(dom, [&] {
    DG_REQUIRE(level >= 0 && level + 1 < (int)dom->levels.size(), "level out of range");
    DG_REQUIRE(r_fine && b_coarse, "null pointer");
    dg::launch_restrict<double>(dom->N, dom->levels[level].n, dom->levels[level + 1].n, dom->Ilo64.get(),
                                dom->Ihi64.get(), r_fine, b_coarse, pick(dom, stream));
  });
}

dg_status dg_mg_prolongate_add(dg_domain* dom, int32_t level, const double* u_coarse, double* u_fine, void* stream) {
  if (!dom) return DG_ERR_INVALID_ARG;
  return guarded(dom, [&] {
    DG_REQUIRE(level >= 0 && level + 1 < (int)dom->levels.size(), "level out of range");
    DG_REQUIRE(u_coarse && u_fine, "null pointer");
    dg::launch_prolongate_add<double>(dom->N, dom->levels[level].n, dom->levels[level + 1].n, dom->Ilo64.get(),
                                      dom->Ihi64.get(), u_coarse, u_fine, pick(dom, stream));
  });
}

dg_status dg_schwarz_smooth(dg_domain* dom, int32_t level, const double* b, double* u, int32_t iterations,
                            void* stream) {
  if (!dom) return DG_ERR_INVALID_ARG;
  return guarded(dom, [&] {
    check_level(dom, level);
    DG_REQUIRE(b && u && iterations >= 0, "bad arguments");
    cudaStream_t s = pick(dom, stream);
    if (!dom->mixed) {
      dg::schwarz_smooth<double>(dom, level, b, u, iterations, false, s);
      return;
    }
    const int64_t n = dom->levels[level].ndof;
    dg::DevBuf<float> tmp(2 * n);
    dg::launch_convert_d2f(n, b, tmp.get(), s);
    dg::launch_convert_d2f(n, u, tmp.get() + n, s);
    dg::schwarz_smooth<float>(dom, level, tmp.get(), tmp.get() + n, iterations, false, s);
    dg::launch_convert_f2d(n, tmp.get() + n, u, s);
    DG_CUDA(cudaStreamSynchronize(s));
  });
}

dg_status dg_vcycle(dg_domain* dom, const double* r, double* z, void* stream) {
  if (!dom) return DG_ERR_INVALID_ARG;
  return guarded(dom, [&] {
    DG_REQUIRE(r && z && r != z, "r and z must be distinct device pointers");
    cudaStream_t s = pick(dom, stream);
    dg::precondition(dom, 2, r, z, s);
  });
}

dg_status dg_dot(dg_domain* dom, int32_t m, const double* V, int64_t ld, const double* w, double* out, void* stream) {
  if (!dom) return DG_ERR_INVALID_ARG;
  return guarded(dom, [&] {
    const int64_t n = dom->levels[0].ndof;
    DG_REQUIRE(V && w && out && m >= 1 && ld >= n, "bad arguments");
    if ((int64_t)dom->partial.count < (int64_t)dg::multidot_partial_blocks() * m)
      dom->partial.alloc((size_t)dg::multidot_partial_blocks() * m);
    dg::launch_multidot(n, m, V, ld, w, dom->partial.get(), out, pick(dom, stream));
  });
}

dg_status dg_nonlinear_residual(dg_domain* dom, const double* u, const double* b, double* r, void* stream) {
  if (!dom) return DG_ERR_INVALID_ARG;
  return guarded(dom, [&] {
    DG_REQUIRE(dom->desc.problem == DG_PROBLEM_PUNCTURE, "not a PUNCTURE domain");
    DG_REQUIRE(u && r, "null pointer");
    dg::puncture_residual_api(dom, u, b, r, pick(dom, stream));
  });
}

dg_status dg_set_linearization(dg_domain* dom, const double* u, void* stream) {
  if (!dom) return DG_ERR_INVALID_ARG;
  return guarded(dom, [&] {
    DG_REQUIRE(dom->desc.problem == DG_PROBLEM_PUNCTURE, "not a PUNCTURE domain");
    dg::puncture_linearize_api(dom, u, pick(dom, stream));
  });
}

dg_status dg_set_subdomain_solver(dg_domain* dom, int32_t solver, int32_t iterations, void* stream) {
  if (!dom) return DG_ERR_INVALID_ARG;
  return guarded(dom, [&] {
    DG_REQUIRE(dom->desc.problem == DG_PROBLEM_PUNCTURE, "not a PUNCTURE domain");
    dg::subdomain_solver_api(dom, solver, iterations, pick(dom, stream));
  });
}

dg_status dg_puncture_fields(const dg_domain* dom, double* alpha, double* beta, void* stream) {
  if (!dom || !alpha || !beta) return DG_ERR_INVALID_ARG;
  if (dom->desc.problem != DG_PROBLEM_PUNCTURE) return DG_ERR_INVALID_ARG;
  dg_domain* d = const_cast<dg_domain*>(dom);
  return guarded(d, [&] {
    const size_t nb = sizeof(double) * dom->levels[0].ndof;
    cudaStream_t s = pick(d, stream);
    DG_CUDA(cudaMemcpyAsync(alpha, dom->alpha.get(), nb, cudaMemcpyDeviceToDevice, s));
    DG_CUDA(cudaMemcpyAsync(beta, dom->beta.get(), nb, cudaMemcpyDeviceToDevice, s));
  });
}

dg_status dg_layout_coordinates_host(const dg_domain_desc* d, double* x, double* y, double* z) {
  if (!d || !x || !y || !z) return DG_ERR_INVALID_ARG;
  if (d->N < 2 || d->N > DG_MAX_N || d->n[0] < 1 || d->n[1] < 1 || d->n[2] < 1) return DG_ERR_INVALID_ARG;
  try {
    const dg::LglTables t = dg::make_lgl(d->N);
    const int N = d->N, N3 = N * N * N;
    double h[3];
    for (int i = 0; i < 3; ++i) h[i] = (d->upper[i] - d->lower[i]) / d->n[i];
    const int64_t E = (int64_t)d->n[0] * d->n[1] * d->n[2];
    for (int64_t e = 0; e < E; ++e) {
      const int ex = (int)(e % d->n[0]), ey = (int)((e / d->n[0]) % d->n[1]), ez = (int)(e / ((int64_t)d->n[0] * d->n[1]));
      for (int p = 0; p < N3; ++p) {
        const int i = p % N, j = (p / N) % N, k = p / (N * N);
        const int64_t q = e * N3 + p;
        x[q] = d->lower[0] + h[0] * (ex + 0.5 * (t.x[i] + 1.0));
        y[q] = d->lower[1] + h[1] * (ey + 0.5 * (t.x[j] + 1.0));
        z[q] = d->lower[2] + h[2] * (ez + 0.5 * (t.x[k] + 1.0));
      }
    }
  } catch (...) {
    return DG_ERR_INVALID_ARG;
  }
  return DG_OK;
}

dg_status dg_copy_coordinates(const dg_domain* dom, double* x, double* y, double* z, void* stream) {
  if (!dom || !x || !y || !z) return DG_ERR_INVALID_ARG;
  dg_domain* d = const_cast<dg_domain*>(dom);
  return guarded(d, [&] {
    const size_t nb = sizeof(double) * dom->levels[0].ndof;
    cudaStream_t s = pick(d, stream);
    DG_CUDA(cudaMemcpyAsync(x, dom->X.get(), nb, cudaMemcpyDeviceToDevice, s));
    DG_CUDA(cudaMemcpyAsync(y, dom->Y.get(), nb, cudaMemcpyDeviceToDevice, s));
    DG_CUDA(cudaMemcpyAsync(z, dom->Z.get(), nb, cudaMemcpyDeviceToDevice, s));
  });
}

dg_status elliptic_solve(dg_domain* dom, const double* b, double* u, double tol, const dg_solve_opts* opts,
                         dg_solve_report* report) {
  if (!dom) return DG_ERR_INVALID_ARG;
  dg_solve_opts o{};
  o.max_iterations = 200;
  o.precondition = 2;
  o.linear_tol = 1e-4;
  o.max_newton_steps = 20;
  o.subdomain_iterations = 3;
  if (opts) o = *opts;
  dg_status result = DG_OK;
  dg_status st = guarded(dom, [&] {
    DG_REQUIRE(u != nullptr, "u must be a device pointer");
    DG_REQUIRE(b != nullptr || dom->desc.problem == DG_PROBLEM_PUNCTURE, "b must be a device pointer");
    result = dg::solve(dom, b, u, tol, o, report);
  });
  if (st != DG_OK) {
    if (report) report->status = st;
    return st;
  }
  if (result != DG_OK) dom->err = "solve ended with status " + std::to_string((int)result);
  return result;
}

dg_status elliptic_solve_host(dg_domain* dom, const double* f_host, double* u_host, double tol,
                              const dg_solve_opts* opts, dg_solve_report* report) {
  if (!dom) return DG_ERR_INVALID_ARG;
  dg_status st = guarded(dom, [&] {
    DG_REQUIRE(u_host != nullptr, "u_host must be a host pointer");
    DG_REQUIRE(f_host != nullptr || dom->desc.problem == DG_PROBLEM_PUNCTURE, "f_host must be a host pointer");
    const int64_t n = dom->levels[0].ndof;
    if (!dom->host_f.get()) {
      dom->host_f.alloc(n);
      dom->host_b.alloc(n);
      dom->host_u.alloc(n);
    }
    cudaStream_t s = dom->stream;
    DG_CUDA(cudaMemcpyAsync(dom->host_u.get(), u_host, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    if (f_host) {
      DG_CUDA(cudaMemcpyAsync(dom->host_f.get(), f_host, sizeof(double) * n, cudaMemcpyHostToDevice, s));
      dg::launch_scale_mul(n, dom->mass.get(), dom->host_f.get(), dom->host_b.get(), s);
    }
  });
  if (st != DG_OK) {
    if (report) report->status = st;
    return st;
  }
  const dg_status result = elliptic_solve(dom, f_host ? dom->host_b.get() : nullptr, dom->host_u.get(), tol, opts,
                                          report);
  st = guarded(dom, [&] {
    DG_CUDA(cudaMemcpyAsync(u_host, dom->host_u.get(), sizeof(double) * dom->levels[0].ndof, cudaMemcpyDeviceToHost,
                            dom->stream));
    DG_CUDA(cudaStreamSynchronize(dom->stream));
  });
  if (st != DG_OK) return st;
  if (result != DG_OK) dom->err = "solve ended with status " + std::to_string((int)result);
  return result;
}

dg_status elliptic_batch_create(dg_domain* const* domains, const double* const* b, double* const* u, int32_t count,
                                double tol, const dg_solve_opts* opts, dg_batch** out) {
  if (!domains || !b || !u || !out || count < 1) {
    dg::set_null_handle_error("elliptic_batch_create: null argument or count < 1");
    return DG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  dg_solve_opts o{};
  o.max_iterations = 200;
  o.precondition = 2;
  o.linear_tol = 1e-4;
  o.max_newton_steps = 20;
  o.subdomain_iterations = 3;
  if (opts) o = *opts;
  try {
    dg::AllocStreamScope scope(domains[0] ? domains[0]->stream : nullptr);
    *out = dg::batch_create(domains, b, u, count, tol, o);
    dg::set_null_handle_error("");
    return DG_OK;
  } catch (const dg::Error& e) {
    dg::set_null_handle_error(e.message);
    return e.status;
  } catch (const std::bad_alloc&) {
    dg::set_null_handle_error("host allocation failed");
    return DG_ERR_OOM;
  } catch (const std::exception& e) {
    dg::set_null_handle_error(e.what());
    return DG_ERR_INVALID_ARG;
  }
}

dg_status elliptic_batch_run(dg_batch* batch, void* stream, dg_solve_report* reports) {
  if (!batch) return DG_ERR_INVALID_ARG;
  try {
    dg::batch_run(batch, (cudaStream_t)stream, reports);
    dg::set_null_handle_error("");
    return DG_OK;
  } catch (const dg::Error& e) {
    dg::set_null_handle_error(e.message);
    return e.status;
  }
}

void elliptic_batch_destroy(dg_batch* batch) { dg::batch_destroy(batch); }

int64_t dg_kernel_launches(void) { return dg::launches_total(); }

dg_status dg_profile_enable(dg_domain* dom, int32_t enable) {
  if (!dom) return DG_ERR_INVALID_ARG;
  return guarded(dom, [&] {
    DG_CUDA(cudaStreamSynchronize(dom->stream));
    dom->prof.clear();
    dom->prof.on = enable != 0;
    // events for graph capture come from this pool (no event creation while capturing)
    while (dom->prof.on && dom->prof.pool.size() < 1024) {
      cudaEvent_t e;
      DG_CUDA(cudaEventCreate(&e));
      dom->prof.pool.push_back(e);
    }
  });
}

dg_status dg_profile_read(dg_domain* dom, dg_phase_stats out[DG_PHASE_COUNT]) {
  if (!dom || !out) return DG_ERR_INVALID_ARG;
  return guarded(dom, [&] { dg::profile_read(dom, out); });
}

}  // extern "C"
