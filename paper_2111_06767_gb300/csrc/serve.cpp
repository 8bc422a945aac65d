// Continuous-batching request loop for elliptic solves.
//
// submit() copies a request into library memory and queues it. Worker threads (one per
// concurrently running solve, each with its own CUDA stream) admit the oldest waiting request
// whose estimated device footprint fits the remaining memory budget, take a domain for it, solve
// it and publish the result; admission happens whenever a worker and enough budget free up, so
// requests that arrive while others run join the device work as capacity allows. poll() hands a
// finished result back exactly once.
//
// Domains stay on the device between requests: a finished request's domain (its multigrid
// hierarchy, explicit subdomain inverses, Krylov and multigrid work vectors and captured graphs)
// is kept in an idle pool keyed by its descriptor, and the next request with the same descriptor
// reuses it instead of building a new one (the paper's amortisation of the explicit inverses over
// many solves, Sec. III.E). Idle domains count against the memory budget and are released, least
// recently used first, when a request that needs new memory would not fit otherwise. Requests with
// per-node geometry or coefficients are not pooled.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "domain.h"

namespace {

double clock_now() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Job {
  uint64_t ticket = 0;
  dg_request req{};
  std::vector<double> f;
  std::vector<double> xyz, coef;  // copies of per-node geometry / coefficient (curved domains)
  std::atomic<bool> cancel{false};
  size_t bytes = 0;
  double submit_time = 0, admit_time = 0, finish_time = 0;
  dg_status status = DG_PENDING;
  dg_solve_report report{};
  std::vector<double> u;
};

}  // namespace

namespace dg {

// Upper bound of a domain's device footprint (bytes) before it is built.
size_t estimate_domain_bytes(const dg_domain_desc& d, int max_iterations, bool linearized_inverses) {
  const int N = d.N, ov = d.overlap;
  const size_t nS = (size_t)N * N * N + 6 * (size_t)ov * N * N;
  const size_t ld = (nS + 31) / 32 * 32;
  const bool mixed = d.precision == DG_PRECISION_MIXED;
  const size_t fb = mixed ? 4 : 8;
  size_t total = (size_t)48 * (nS + 7 * N * N * N) * 4 + (size_t)64 * N * N * N * 7 * fb;  // point maps, shares
  int n[3] = {d.n[0], d.n[1], d.n[2]};
  size_t build_peak = 0;
  for (int l = 0; l < DG_MAX_LEVELS; ++l) {
    const size_t E = (size_t)n[0] * n[1] * n[2];
    const size_t ndof = E * N * N * N;
    // classes up to symmetry: 1, 2 or 3 boundary categories per dimension (n = 1-2, 3-4, >= 5);
    // dimensions of equal element width count as a multiset
    const double hw[3] = {(d.upper[0] - d.lower[0]) / n[0], (d.upper[1] - d.lower[1]) / n[1],
                          (d.upper[2] - d.lower[2]) / n[2]};
    const int cats[3] = {n[0] <= 2 ? 1 : (n[0] <= 4 ? 2 : 3), n[1] <= 2 ? 1 : (n[1] <= 4 ? 2 : 3),
                         n[2] <= 2 ? 1 : (n[2] <= 4 ? 2 : 3)};
    size_t classes = (size_t)cats[0] * cats[1] * cats[2];
    if (hw[0] == hw[1] && hw[1] == hw[2] && cats[0] == cats[1] && cats[1] == cats[2])
      classes = (size_t)cats[0] * (cats[0] + 1) * (cats[0] + 2) / 6;
    if (d.neumann_faces) {
      // the two sides of a dimension may differ: up to 5 positions per dimension, no symmetry
      classes = (size_t)std::min(n[0], 5) * std::min(n[1], 5) * std::min(n[2], 5);
    }
    classes = std::min(classes, E);
    if (d.node_xyz || d.coef) {
      // every subdomain has its own inverse, compact; MIXED keeps FP16 copies (FP32 with "simt"),
      // built in the smoother's precision; plus the nodal metric, face-node penalty and traces
      const size_t store = mixed ? (d.subdomain_gemm == DG_GEMM_SIMT ? 4 : 2) : 8;
      build_peak = std::max(build_peak, E * nS * nS * (mixed ? 4 : 8));
      total += E * nS * nS * store + ndof * (11 * 12 + 8) + E * 6 * N * N * 24;
    } else {
      build_peak = std::max(build_peak, classes * nS * nS * 8);  // FP64 build, freed after inversion
      total += classes * ld * ld * fb;                            // stored inverses
    }
    total += 2 * E * ld * fb + 3 * ndof * fb + 4 * E * 4;       // r_S, du_S, b, u, r, tables
    if ((d.mg_levels && l + 1 == d.mg_levels) || (n[0] % 2 && n[1] % 2 && n[2] % 2)) break;
    for (int i = 0; i < 3; ++i)
      if (n[i] % 2 == 0) n[i] /= 2;
  }
  const size_t ndof0 = (size_t)d.n[0] * d.n[1] * d.n[2] * N * N * N;
  if (linearized_inverses && d.problem == DG_PROBLEM_PUNCTURE) {
    // per-subdomain inverses of the finest level plus its class matrices (at most one per element)
    total += 2 * (size_t)d.n[0] * d.n[1] * d.n[2] * nS * nS * fb;
  }
  // Krylov basis: grown on demand; admission counts up to 64 iterations
  total += ndof0 * 8 * (2 * (size_t)std::min(max_iterations, 64) + 16);
  return total + build_peak + (8u << 20);
}

}  // namespace dg

struct PooledDomain {
  dg_domain* dom = nullptr;
  size_t bytes = 0;
  uint64_t last_use = 0;
};

struct dg_server {
  dg_serve_desc desc{};
  std::mutex mu;
  std::unordered_map<std::string, std::vector<PooledDomain>> idle;  // key: descriptor bytes
  size_t idle_bytes = 0;
  uint64_t use_clock = 0;
  std::condition_variable cv_work, cv_done;
  std::deque<Job*> waiting;
  std::unordered_map<uint64_t, Job*> jobs;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  size_t budget = 0, in_use = 0;
  uint64_t next_ticket = 1;
  bool stopping = false;
  double t0 = clock_now();

  void run(int wid);
  // With mu held: an idle domain for this key (removed from the pool), or nullptr.
  dg_domain* take_idle(const std::string& key, size_t* bytes);
  // With mu held: move least recently used idle domains into `out` until `need` more bytes fit.
  void evict_for(size_t need, std::vector<dg_domain*>& out);
};

namespace {
// Pool key: the descriptor's bytes, or "" (not pooled) for per-node geometry or coefficients.
std::string pool_key(const dg_domain_desc& d) {
  if (d.node_xyz || d.coef) return std::string();
  dg_domain_desc k = d;
  k.node_xyz = nullptr;
  k.coef = nullptr;
  return std::string(reinterpret_cast<const char*>(&k), sizeof(k));
}
}  // namespace

dg_domain* dg_server::take_idle(const std::string& key, size_t* bytes) {
  if (key.empty()) return nullptr;
  auto it = idle.find(key);
  if (it == idle.end() || it->second.empty()) return nullptr;
  PooledDomain p = it->second.back();
  it->second.pop_back();
  idle_bytes -= p.bytes;
  *bytes = p.bytes;
  return p.dom;
}

void dg_server::evict_for(size_t need, std::vector<dg_domain*>& out) {
  while (in_use + idle_bytes + need > budget && idle_bytes > 0) {
    std::vector<PooledDomain>* oldest = nullptr;
    size_t pos = 0;
    for (auto& kv : idle)
      for (size_t i = 0; i < kv.second.size(); ++i)
        if (!oldest || kv.second[i].last_use < (*oldest)[pos].last_use) {
          oldest = &kv.second;
          pos = i;
        }
    if (!oldest) break;
    idle_bytes -= (*oldest)[pos].bytes;
    out.push_back((*oldest)[pos].dom);
    oldest->erase(oldest->begin() + pos);
  }
}

void dg_server::run(int wid) {
  cudaStream_t s = streams[wid % streams.size()];
  for (;;) {
    Job* job = nullptr;
    dg_domain* dom = nullptr;
    std::string key;
    std::vector<dg_domain*> evicted;
    {
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        if (stopping && waiting.empty()) return;
        for (auto it = waiting.begin(); it != waiting.end(); ++it) {
          const std::string k = pool_key((*it)->req.domain);
          size_t pooled = 0;
          dg_domain* d = take_idle(k, &pooled);
          if (d) {  // an idle domain of this shape: no new memory
            job = *it;
            dom = d;
            key = k;
            job->bytes = pooled;
            waiting.erase(it);
            break;
          }
          if (in_use + (*it)->bytes > budget) continue;
          evict_for((*it)->bytes, evicted);
          if (in_use + idle_bytes + (*it)->bytes <= budget) {
            job = *it;
            key = k;
            waiting.erase(it);
            break;
          }
        }
        if (job) break;
        cv_work.wait(lk);
      }
      in_use += job->bytes;
      job->admit_time = clock_now() - t0;
    }
    for (dg_domain* d : evicted) dg_domain_destroy(d);
    dg_status st = DG_OK;
    if (dom) {
      dom->stream = s;  // idle: all of its earlier work is complete
    } else {
      st = dg_domain_create(&job->req.domain, s, &dom);
    }
    if (st == DG_OK) {
      dg_layout lay;
      dg_domain_layout(dom, &lay);
      try {
        job->u.assign(lay.n_dof, 0.0);
      } catch (...) {
        st = DG_ERR_OOM;
      }
      if (st == DG_OK) {
        dg_solve_opts o = job->req.opts;
        o.relative_to_b = job->req.domain.problem == DG_PROBLEM_POISSON ? 1 : 0;
        dom->cancel = &job->cancel;
        st = elliptic_solve_host(dom, job->req.domain.problem == DG_PROBLEM_POISSON ? job->f.data() : nullptr,
                                 job->u.data(), job->req.tol, &o, &job->report);
        dom->cancel = nullptr;
      }
      if (cudaStreamSynchronize(s) != cudaSuccess) {
        (void)cudaGetLastError();
        if (st == DG_OK) st = DG_ERR_CUDA;
      }
    }
    const bool keep = dom && !key.empty() && (st == DG_OK || st == DG_ERR_NOT_CONVERGED || st == DG_ERR_CANCELLED);
    if (dom && !keep) {
      dg_domain_destroy(dom);
      dom = nullptr;
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      in_use -= job->bytes;
      if (keep) {
        idle[key].push_back(PooledDomain{dom, job->bytes, ++use_clock});
        idle_bytes += job->bytes;
      }
      job->status = st;
      job->report.status = st;
      job->finish_time = clock_now() - t0;
    }
    cv_work.notify_all();
    cv_done.notify_all();
  }
}

extern "C" {

dg_status elliptic_serve_create(const dg_serve_desc* desc, dg_server** out) {
  if (!desc || !out) return DG_ERR_INVALID_ARG;
  *out = nullptr;
  if (desc->max_active < 1 || desc->queue_capacity < 1 || desc->n_streams < 1) return DG_ERR_INVALID_ARG;
  dg_server* srv = new (std::nothrow) dg_server();
  if (!srv) return DG_ERR_OOM;
  srv->desc = *desc;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    (void)cudaGetLastError();
    delete srv;
    return DG_ERR_CUDA;
  }
  srv->budget = desc->memory_budget_bytes ? desc->memory_budget_bytes : (size_t)(0.8 * (double)free_b);
  for (int i = 0; i < desc->n_streams; ++i) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      (void)cudaGetLastError();
      for (auto x : srv->streams) cudaStreamDestroy(x);
      delete srv;
      return DG_ERR_CUDA;
    }
    srv->streams.push_back(s);
  }
  for (int i = 0; i < desc->max_active; ++i) srv->workers.emplace_back([srv, i] { srv->run(i); });
  *out = srv;
  return DG_OK;
}

dg_status elliptic_serve_submit(dg_server* srv, const dg_request* req, uint64_t* ticket) {
  if (!srv || !req || !ticket) return DG_ERR_INVALID_ARG;
  const dg_domain_desc& d = req->domain;
  if (d.N < 2 || d.N > DG_MAX_N || d.n[0] < 1 || d.n[1] < 1 || d.n[2] < 1) return DG_ERR_INVALID_ARG;
  if (d.problem == DG_PROBLEM_POISSON && !req->f_host) return DG_ERR_INVALID_ARG;
  const int max_it = req->opts.max_iterations > 0 ? req->opts.max_iterations : 200;
  if (req->opts.subdomain_solver != 0 && req->opts.subdomain_solver != 1) return DG_ERR_INVALID_ARG;
  const size_t bytes = dg::estimate_domain_bytes(d, max_it, req->opts.subdomain_solver == 1);
  Job* job = new (std::nothrow) Job();
  if (!job) return DG_ERR_OOM;
  job->req = *req;
  job->bytes = bytes;
  if (d.problem == DG_PROBLEM_POISSON) {
    const size_t ndof = (size_t)d.n[0] * d.n[1] * d.n[2] * d.N * d.N * d.N;
    try {
      job->f.assign(req->f_host, req->f_host + ndof);
    } catch (...) {
      delete job;
      return DG_ERR_OOM;
    }
  }
  job->req.f_host = nullptr;
  if (d.node_xyz || d.coef) {
    // per-node geometry and coefficient are copied as the source is; the queued descriptor points at
    // the copies, which live as long as the job
    const size_t ndof = (size_t)d.n[0] * d.n[1] * d.n[2] * d.N * d.N * d.N;
    try {
      if (d.node_xyz) job->xyz.assign(d.node_xyz, d.node_xyz + 3 * ndof);
      if (d.coef) job->coef.assign(d.coef, d.coef + ndof);
    } catch (...) {
      delete job;
      return DG_ERR_OOM;
    }
    job->req.domain.node_xyz = d.node_xyz ? job->xyz.data() : nullptr;
    job->req.domain.coef = d.coef ? job->coef.data() : nullptr;
  }
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stopping || bytes > srv->budget) {
      delete job;
      return DG_ERR_INVALID_ARG;
    }
    if ((int)srv->waiting.size() >= srv->desc.queue_capacity) {
      delete job;
      return DG_ERR_BUSY;
    }
    job->ticket = srv->next_ticket++;
    job->submit_time = clock_now() - srv->t0;
    srv->jobs[job->ticket] = job;
    srv->waiting.push_back(job);
    *ticket = job->ticket;
  }
  srv->cv_work.notify_all();
  return DG_OK;
}

dg_status elliptic_serve_poll(dg_server* srv, uint64_t ticket, dg_result* out) {
  if (!srv) return DG_ERR_INVALID_ARG;
  Job* job = nullptr;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(ticket);
    if (it == srv->jobs.end()) return DG_ERR_NOT_FOUND;
    if (it->second->status == DG_PENDING) return DG_PENDING;
    job = it->second;
    srv->jobs.erase(it);
  }
  const dg_status st = job->status;
  if (out) {
    out->report = job->report;
    out->n_dof = (int64_t)job->u.size();
    out->submit_time = job->submit_time;
    out->admit_time = job->admit_time;
    out->finish_time = job->finish_time;
    if (out->u_host && !job->u.empty()) std::memcpy(out->u_host, job->u.data(), sizeof(double) * job->u.size());
  }
  delete job;
  return st;
}

dg_status elliptic_serve_cancel(dg_server* srv, uint64_t ticket) {
  if (!srv) return DG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->jobs.find(ticket);
  if (it == srv->jobs.end()) return DG_ERR_NOT_FOUND;
  Job* job = it->second;
  if (job->status != DG_PENDING) return DG_OK;  // finished: the result stands
  job->cancel.store(true);
  for (auto w = srv->waiting.begin(); w != srv->waiting.end(); ++w) {
    if (*w != job) continue;
    // never admitted: leave the queue now
    srv->waiting.erase(w);
    job->status = DG_ERR_CANCELLED;
    job->report.status = DG_ERR_CANCELLED;
    job->finish_time = clock_now() - srv->t0;
    break;
  }
  return DG_OK;
}

double elliptic_serve_clock(const dg_server* srv) { return srv ? clock_now() - srv->t0 : 0.0; }

void elliptic_serve_destroy(dg_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stopping = true;
  }
  srv->cv_work.notify_all();
  for (auto& t : srv->workers) t.join();
  for (auto& kv : srv->idle)
    for (auto& p : kv.second) dg_domain_destroy(p.dom);
  for (auto& kv : srv->jobs) delete kv.second;
  for (auto s : srv->streams) cudaStreamDestroy(s);
  delete srv;
}

}  // extern "C"
