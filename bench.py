"""Benchmark: multigrid-Schwarz preconditioned FGMRES solves of the 3-D Poisson problem with a
16-Gaussian source on [-1,1]^3, 8^3 elements, 8 LGL points per dimension (262,144 points),
3-level h-multigrid, Schwarz overlap 2, penalty C = 1.5, relative residual 1e-10.

One step = one complete solve from u = 0 (every kernel of the hot path: DG operator, Schwarz
gather / subdomain-inverse GEMM / weighted scatter on every level, restriction, prolongation,
FGMRES orthogonalisation). The headline value is solves/s with the FP32 preconditioner under
FP64 FGMRES; the plain FP64 solver, the DG-apply rate and the per-phase roofline are reported
beside it. Multi-GPU: independent replicas (one solve stream per GPU, no collective).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--impl reference` times the FP64 CPU oracle (test infrastructure) on a bounded sample of the
same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DG-apply GDOF/s; solves/s & p99 latency at 1e-10 residual, mixed vs FP64"
WORKLOAD = ("poisson-gauss16-8x8x8-N8: 3-D Poisson on [-1,1]^3, 8^3 elements, N=8 LGL points/dim "
            "(262,144 DOF), 16 seeded Gaussians (widths U[0.1,0.4]), 3-level h-MG V-cycle, Schwarz overlap 2, "
            "3+3 smoothing, C=1.5, FGMRES to 1e-10 relative residual from u=0")
N_CFG, n_CFG, LEVELS = 8, (8, 8, 8), 3
FP64_PEAK_TFLOPS = 1.199  # FP64 FMA rate probed on this machine's GB300 (152 SMs)
FP32_PEAK_TFLOPS = 72.7   # FP32 FMA rate probed on this machine's GB300 (152 SMs at 1987 MHz)
TOL = 1e-10

# CPU baseline: the oracle (FP64 numpy) on the same 8^3, N = 8 problem, 3-level V-cycle. One solve
# takes minutes on the host, so the bounded sample is a few of its FGMRES iterations, timed one by one
# after the first (which also builds the subdomain matrices and is left out); the rate per solve is
# the mean iteration time times the oracle's own iteration count for this problem at 1e-10 (10, the
# same as the GPU solve's).
# the oracle's FGMRES iterations to 1e-10 on each workload the sample can run (the headline Gaussian
# problem, and the 2^3-element sine problem that CPU tests of this script use)
ORACLE_ITERATIONS = {"gauss": 10, "sine": 4}

_SAMPLE_SCRIPT = r"""
import json, os, sys, time
sys.path.insert(0, sys.argv[1])
import numpy as np
import workloads
from oracle import dg, krylov, solve
iters, budget, which = int(sys.argv[2]), float(sys.argv[3]), sys.argv[4]
cfg = workloads.GAUSS_8x8x8 if which == "gauss" else workloads.SINE_2x2x2
t_start = time.perf_counter()
grid = dg.BoxGrid(cfg.lower, cfg.upper, cfg.n, cfg.N, cfg.penalty)
pr = solve.Problem(grid, mg_levels=cfg.mg_levels, overlap=cfg.overlap, presmooth=cfg.presmooth,
                   postsmooth=cfg.postsmooth)
x, y, z = grid.coordinates()
src = workloads.gaussian_source(cfg.seed) if which == "gauss" else workloads.sine_source_3d
b = dg.rhs(pr.graphs[0], src(x, y, z))
setup = time.perf_counter() - t_start
stamps = [time.perf_counter()]
class Done(Exception):
    pass
def cb(j, res):
    stamps.append(time.perf_counter())
    print(json.dumps({"iteration": j, "seconds": stamps[-1] - stamps[-2], "estimate": res}), flush=True)
    if j >= iters + 1 or (j >= 2 and stamps[-1] - t_start > budget):
        raise Done()
try:
    krylov.fgmres(pr.apply, b, None, pr.vcycle, 1e-10, 200, callback=cb)
except Done:
    pass
print(json.dumps({"setup_s": setup, "first_iteration_s": stamps[1] - stamps[0],
                  "iteration_s": [stamps[i + 1] - stamps[i] for i in range(1, len(stamps) - 1)],
                  "dof": int(b.size)}), flush=True)
"""


def oracle_threads():
    """Host cores the oracle's BLAS may use."""
    return os.cpu_count() or 1


def start_cpu_sample(iters: int, budget_s: float, threads: int, which: str = "gauss"):
    """Start the oracle sample in its own interpreter (BLAS limited to `threads`)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    proc = subprocess.Popen([sys.executable, "-c", _SAMPLE_SCRIPT, ROOT, str(iters), str(budget_s), which],
                            stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
    proc.which = which
    return proc


def finish_cpu_sample(proc, threads: int):
    out, err = proc.communicate()
    if proc.returncode != 0:
        return None
    res = json.loads(out.strip().splitlines()[-1])
    its = res["iteration_s"]
    if not its:
        return None
    per_iter = sum(its) / len(its)
    n_it = ORACLE_ITERATIONS[proc.which]
    value = 1.0 / (per_iter * n_it)
    what = ("the same problem (8^3 elements, N=8" if proc.which == "gauss" else "the 2^3-element sine problem (N=6")
    sample = (f"oracle (numpy FP64) MG-Schwarz FGMRES on {what}, {res['dof']} DOF): {len(its)} FGMRES "
              f"iteration(s) timed one by one ({per_iter:.2f} s each) after the first (set-up {res['setup_s']:.1f} s, "
              f"first iteration incl. subdomain-matrix build {res['first_iteration_s']:.1f} s, both untimed); "
              f"solves/s = 1 / (mean iteration time x {n_it} iterations, the oracle's count at 1e-10)")
    return {"value": value, "unit": "solves/s", "cores": threads, "kind": "oracle", "sample": sample,
            "iteration_seconds": its, "setup_seconds": res["setup_s"] + res["first_iteration_s"]}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    threads = oracle_threads()
    iters = max(1, min(args.steps, 3))
    cpu = finish_cpu_sample(start_cpu_sample(iters, 600.0, threads, args.oracle_workload), threads)
    if cpu is None:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle sample failed"}), flush=True)
        return
    its = cpu["iteration_seconds"]
    value = cpu["value"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": len(its), "warmup": 1,
            "ms_per_step": 1e3 * sum(its) / len(its) * ORACLE_ITERATIONS[args.oracle_workload],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.oracle_workload == "gauss" else "poisson-sine-2x2x2-N6",
                       "step": "one FGMRES iteration of the solve"},
            "cpu_baseline": {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self._stop = threading.Event()
        self._t = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                for line in out.stdout.strip().splitlines():
                    self.rows.append([c.strip() for c in line.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9 for i in range(4) if r[5 + i] == "Active"})
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def max_over_ranks(x: float, device=None) -> float:
    """The largest x over all ranks of the default process group (x itself without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, max_seconds: float) -> float:
    """Units processed by all ranks divided by the slowest rank's time (weak scaling)."""
    return world * units_per_rank / max_seconds


def build_requests(dgg, workloads, items, precision="mixed"):
    """(desc, f) for (kind, n, N, seed) items: Poisson on [-1,1]^3 with a seeded 16-Gaussian source,
    puncture on [-20,20]^3 with the binary punctures; n is per dimension (int or 3-tuple)."""
    out = []
    for kind, n, N, seed in items:
        nn = (n,) * 3 if isinstance(n, int) else tuple(n)
        if kind == "poisson":
            desc = dgg.make_desc((-1.0,) * 3, (1.0,) * 3, nn, N, precision=precision, overlap=2)
            x, y, z = dgg.host_coordinates(desc)
            f = workloads.gaussian_source(seed)(x, y, z)
        else:
            desc = dgg.make_desc((-20.0,) * 3, (20.0,) * 3, nn, N, precision=precision, overlap=2, problem="puncture",
                                 punctures=workloads.BINARY_PUNCTURES)
            f = None
        out.append((desc, f))
    return out


def served_run(dgg, workloads, duration, rate=200.0, seed=5, max_active=8, precision="mixed", warm=True):
    """Poisson-process arrivals of Poisson / puncture requests (n ~ U{2..12} cubic, N ~ U{4..8}) into the
    continuous-batching server; latency = completion - scheduled arrival. With `warm`, one request of
    every shape the stream uses is served first (outside the timed window): the server keeps finished
    domains with their explicit inverses on the device and reuses them for later requests of the same
    shape (the paper's amortised set-up, Sec. III.E), so the window measures the steady state."""
    import time as _t

    arr = workloads.poisson_arrivals(seed, rate, duration)
    reqs = build_requests(dgg, workloads, [(k, n, N, rs) for _, k, n, N, rs in arr], precision=precision)
    srv = dgg.Server(max_active=max_active, n_streams=max_active, queue_capacity=1 << 20)
    warm_s = 0.0
    if warm:
        seen, first = set(), []
        for (_, k, n, N, _), rq in zip(arr, reqs):
            if (k, n, N) not in seen:
                seen.add((k, n, N))
                first.append(rq)
        t0 = srv.clock()
        for _ in range(2):  # a second pass also captures each shape's whole-solve graph
            tks = [srv.submit(d, f, tol=1e-10) for d, f in first]
            for tk in tks:
                while srv.poll(tk)[0] == 1:
                    _t.sleep(0.0005)
        warm_s = srv.clock() - t0
    pending, done, i = {}, {}, 0
    start = srv.clock()
    while len(done) < len(reqs):
        now = srv.clock() - start
        while i < len(reqs) and arr[i][0] <= now:
            tk = srv.submit(reqs[i][0], reqs[i][1], tol=1e-10)
            pending[tk] = arr[i][0]
            i += 1
        for tk in list(pending):
            st, res = srv.poll(tk)
            if st != 1:
                done[tk] = (st, res.finish_time - start - pending.pop(tk), res.report.relative_residual)
        _t.sleep(0.0002)
    total = srv.clock() - start
    srv.close()
    lat = sorted(v[1] for v in done.values())
    pick = lambda q: 1e3 * lat[min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1)]
    return {"requests": len(reqs), "arrival_rate_per_s": rate, "arrival_window_s": duration,
            "warm_up_s": warm_s, "solves_per_s": len(reqs) / total, "p50_latency_ms": pick(0.5), "p99_latency_ms": pick(0.99),
            "ok": sum(1 for v in done.values() if v[0] == 0), "max_relative_residual": max(v[2] for v in done.values()),
            "max_active": max_active,
            "precision": "mixed (TF32 subdomain GEMM, FP64 FGMRES)" if precision == "mixed" else "fp64"}


def served_capacity(dgg, workloads, count=400, seed=5, max_active=8):
    """Service capacity of the server on the served stream's mix: the first `count` requests of the
    arrival stream submitted at once (every shape warmed first, as in served_run), solves/s until the
    last one completes. The timed window of served_run cannot exceed its arrival rate; this is the
    rate the server would sustain under a heavier stream."""
    import time as _t

    arr = workloads.poisson_arrivals(seed, 200.0, 20.0)[:count]
    reqs = build_requests(dgg, workloads, [(k, n, N, rs) for _, k, n, N, rs in arr])
    srv = dgg.Server(max_active=max_active, n_streams=max_active, queue_capacity=1 << 20)
    seen, first = set(), []
    for (_, k, n, N, _), rq in zip(arr, reqs):
        if (k, n, N) not in seen:
            seen.add((k, n, N))
            first.append(rq)
    for _ in range(2):
        tks = [srv.submit(d, f, tol=TOL) for d, f in first]
        for tk in tks:
            while srv.poll(tk)[0] == 1:
                _t.sleep(0.0005)
    t0 = srv.clock()
    tks = [srv.submit(d, f, tol=TOL) for d, f in reqs]
    ok = 0
    for tk in tks:
        while True:
            st, _ = srv.poll(tk)
            if st != 1:
                ok += st == 0
                break
            _t.sleep(0.0005)
    total = srv.clock() - t0
    srv.close()
    return {"requests": count, "solves_per_s": count / total, "ok": ok, "max_active": max_active,
            "timing": "all requests submitted at once, host wall clock to the last completion"}


def served_compare(dgg, workloads, duration, prefix, streams=8):
    """The served stream in MIXED precision, and the first `prefix` seconds of arrivals in both
    precisions (the plain FP64 solver on the same requests, for the mixed/FP64 throughput ratio)."""
    out = served_run(dgg, workloads, duration, max_active=streams)
    out["capacity"] = served_capacity(dgg, workloads, max_active=streams)
    if prefix > 0:
        m = served_run(dgg, workloads, prefix, max_active=streams)
        f = served_run(dgg, workloads, prefix, precision="fp64", max_active=streams)
        out["prefix"] = {"window_s": prefix, "mixed": m, "fp64": f,
                         "mixed_over_fp64_solves_per_s": m["solves_per_s"] / f["solves_per_s"]}
    return out


def batched_run(dgg, workloads, torch, count=512, seed=4, precision="mixed", rounds=3, group=512):
    """`count` independent Poisson solves of uneven shapes (n_i ~ U{2..8}, N ~ U{4..9}, seeded Gaussian
    sources), each domain built once (set-up: hierarchy, explicit inverses, launch-shape tuning, graph
    capture; timed apart), then solved as captured multi-solve graphs (elliptic_batch_*: every solve a
    branch of one graph, `group` solves per graph, one launch per graph). The steady rate is `count`
    solves per round of launches, timed over `rounds` rounds with CUDA events; each round starts every
    solve from u = 0."""
    shapes = workloads.batched_shapes(seed, count)
    t0 = time.perf_counter()
    doms, bs, us = [], [], []
    for k, (n, N) in enumerate(shapes):
        d = dgg.Domain(n=n, N=N, precision=precision, overlap=2)
        x, y, z = d.coordinates()
        bs.append(d.rhs(workloads.gaussian_source(seed + k)(x, y, z).contiguous()))
        us.append(torch.zeros_like(bs[-1]))
        doms.append(d)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    batches = [dgg.Batch(doms[g:g + group], bs[g:g + group], us[g:g + group], tol=TOL)
               for g in range(0, count, group)]
    torch.cuda.synchronize()
    t_capture = time.perf_counter() - t0
    reps = [None] * len(batches)

    def one_round():
        for u in us:
            u.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k, bt in enumerate(batches):  # each run is one graph launch and waits for it
            reps[k] = bt.run()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3

    one_round()  # first launch of each graph uploads it
    times = [one_round() for _ in range(rounds)]
    flat = [r for rs in reps for r in rs]
    out = {"solves": count, "precision": precision, "solves_per_s": count * rounds / sum(times),
           "seconds_per_round": sum(times) / rounds, "graphs": len(batches), "solves_per_graph": group,
           "ok": sum(1 for r in flat if r.status == 0), "max_relative_residual": max(r.relative_residual for r in flat),
           "iterations_mean": sum(r.iterations for r in flat) / len(flat),
           "setup_s": {"domains": t_build, "capture": t_capture},
           "timing": "CUDA events around each round of graph launches (every solve from u = 0)"}
    for bt in batches:
        bt.close()
    for d in doms:
        d.close()
    return out


def batched_compare(dgg, workloads, torch, count, fp64_count):
    """The batched workload in MIXED precision, and its first `fp64_count` solves in both precisions
    (plain FP64 on the GPU is ~50x slower, so it runs on a prefix of the same stream)."""
    out = {"mixed": batched_run(dgg, workloads, torch, count)}
    if fp64_count > 0:
        out["prefix_mixed"] = batched_run(dgg, workloads, torch, fp64_count, group=fp64_count)
        out["prefix_fp64"] = batched_run(dgg, workloads, torch, fp64_count, precision="fp64", rounds=1,
                                         group=fp64_count)
        out["prefix_mixed_over_fp64"] = out["prefix_mixed"]["solves_per_s"] / out["prefix_fp64"]["solves_per_s"]
    return out


def concurrent_run(dgg, workloads, torch, n_streams=8, rounds=4):
    """The Gaussian solve of the headline workload on n_streams domains at once (one host thread
    and one CUDA stream each, independent right-hand sides of the same problem): the throughput of
    the GPU when independent solves share it, with the latency of each solve."""
    import threading
    import time as _t

    src = workloads.gaussian_source(2)
    doms, bs, us, streams = [], [], [], []
    for _ in range(n_streams):
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            d = dgg.Domain(n=n_CFG, N=N_CFG, penalty=1.5, precision="mixed", mg_levels=LEVELS, overlap=2, stream=s)
            x, y, z = d.coordinates()
            b = d.rhs(src(x, y, z).contiguous(), stream=s)
            u = torch.zeros_like(b)
        doms.append(d)
        bs.append(b)
        us.append(u)
        streams.append(s)
    torch.cuda.synchronize()
    lat = [[] for _ in range(n_streams)]
    worst = [0.0] * n_streams

    def worker(i, n, record):
        with torch.cuda.stream(streams[i]):
            for _ in range(n):
                us[i].zero_()
                t = _t.perf_counter()
                rep = doms[i].solve(bs[i], us[i], TOL)  # returns after the final FP64 residual check
                if record:
                    lat[i].append(_t.perf_counter() - t)
                    worst[i] = max(worst[i], rep.relative_residual)

    def run(n, record):
        ths = [threading.Thread(target=worker, args=(i, n, record)) for i in range(n_streams)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()

    run(2, False)  # graphs captured, launch shapes tuned
    torch.cuda.synchronize()
    t0 = _t.perf_counter()
    run(rounds, True)
    total = _t.perf_counter() - t0
    flat = sorted(x for l in lat for x in l)
    pick = lambda q: 1e3 * flat[min(len(flat) - 1, int(math.ceil(q * len(flat))) - 1)]
    return {"streams": n_streams, "solves": n_streams * rounds, "solves_per_s": n_streams * rounds / total,
            "p50_latency_ms": pick(0.5), "p99_latency_ms": pick(0.99), "max_relative_residual": max(worst),
            "timing": "host wall clock over all threads (each solve ends with a host read of its residual)"}


def puncture_compare(dgg, workloads, torch, stream, steps):
    """The binary-puncture workload (16^3 elements, N = 6, [-20,20]^3, 884,736 DOF, mixed precision,
    Newton to 1e-10 with linearized solves to 1e-4) with the two finest-level subdomain solvers:
    3 GMRES iterations preconditioned by the Poisson class inverses (Laplacian approximation) and
    the explicit inverse of every subdomain's linearized matrix, rebuilt at every Newton step."""
    d = dgg.Domain((-20.0,) * 3, (20.0,) * 3, (16, 16, 16), 6, precision="mixed", overlap=2, problem="puncture",
                   punctures=workloads.BINARY_PUNCTURES, stream=stream)
    u = torch.zeros(d.n_dof, dtype=torch.float64, device="cuda")
    out, sols = {}, {}
    for solver in ("gmres", "inverse"):
        opts = dgg.solve_opts(linear_tol=1e-4, subdomain_solver=solver)
        times, reps = [], []
        for i in range(1 + steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                u.zero_()
                e0.record(stream)
                rep = d.solve(None, u, TOL, opts=opts)
                e1.record(stream)
            e1.synchronize()
            if i > 0:
                times.append(e0.elapsed_time(e1))
                reps.append(rep)
        sols[solver] = u.clone()
        d.profile(True)
        with torch.cuda.stream(stream):
            u.zero_()
            d.solve(None, u, TOL, opts=opts)
        stream.synchronize()
        prof = d.profile_read()
        d.profile(False)
        ms = sum(times) / len(times)
        out[solver] = {"solves_per_s": 1e3 / ms, "ms_per_solve": ms, "newton_steps": reps[0].newton_steps,
                       "krylov_iterations": reps[0].iterations,
                       "relative_residual": max(r.relative_residual for r in reps),
                       "phases_ms": {k: round(v["ms"], 3) for k, v in prof.items() if v["launches"]}}
        if solver == "inverse":
            g = prof["subdomain_gemm"]
            out[solver]["inverse_apply_GB/s"] = g["bytes"] / max(g["ms"], 1e-12) / 1e6
    nS = d.layout.subdomain_size
    out["per_subdomain_inverse_bytes"] = 16**3 * nS * nS * 4
    out["solution_rel_diff"] = float((sols["inverse"] - sols["gmres"]).norm() / sols["gmres"].norm())
    d.close()
    return out


def warp_map(X, Y, Z):
    """Smooth warp of [-1,1]^3 that keeps the six faces planar (curved interior elements)."""
    return (X + 0.1 * (1 - X**2) * Y, Y + 0.12 * (1 - Y**2) * Z * X, Z + 0.1 * (1 - Z**2) * (X + Y))


def curved_compare(dgg, workloads, torch, stream, steps):
    """The Gaussian workload (8^3 elements, N = 8, 3 levels) on a warped mesh of curved elements:
    set-up (metric, 584 per-subdomain inverses), solves/s in mixed precision and FP64, and the
    curved DG apply rate at the workload size and at 64^3 elements, N = 4 (16.8M DOF)."""
    out = {}
    desc = dgg.make_desc((-1.0,) * 3, (1.0,) * 3, n_CFG, N_CFG)
    xyz = warp_map(*dgg.host_coordinates(desc))
    src = workloads.gaussian_source(2)
    for prec in ("mixed", "fp64"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            d = dgg.Domain(n=n_CFG, N=N_CFG, precision=prec, mg_levels=LEVELS, overlap=2, stream=stream, node_xyz=xyz)
            x, y, z = d.coordinates()
            b = d.rhs(src(x, y, z).contiguous(), stream=stream)
            u = torch.zeros_like(b)
            rep = d.solve(b, u, TOL)  # builds the per-subdomain inverses of every level
        stream.synchronize()
        setup_s = time.perf_counter() - t0
        k = steps if prec == "mixed" else 1
        times = []
        for i in range(k):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                u.zero_()
                e0.record(stream)
                rep = d.solve(b, u, TOL)
                e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = sum(times) / len(times)
        d.profile(True)
        with torch.cuda.stream(stream):
            u.zero_()
            d.solve(b, u, TOL)
        stream.synchronize()
        prof = d.profile_read()
        d.profile(False)
        gm = prof["subdomain_gemm"]
        out[prec] = {"solves_per_s": 1e3 / ms, "ms_per_solve": ms, "iterations": rep.iterations,
                     "relative_residual": rep.relative_residual, "first_solve_with_setup_s": setup_s,
                     "phases_ms": {k: round(v["ms"], 3) for k, v in prof.items() if v["launches"]},
                     "subdomain_gemm_GB/s": gm["bytes"] / max(gm["ms"], 1e-12) / 1e6}
        d.close()
    # apply rates: the operator reads u and the metric (J and 9 G entries per node) and writes A u
    def rate(dom, prec, reps):
        n = dom.n_dof
        dt = torch.float64 if prec == "fp64" else torch.float32
        uu = torch.empty(n, dtype=dt, device="cuda").uniform_(-1, 1)
        o = torch.empty_like(uu)
        fn = (lambda: dom.apply(uu, o, stream=stream)) if prec == "fp64" else (
            lambda: dom.apply_f32(uu, 0, o, stream=stream))
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
        e1.synchronize()
        return n / (e0.elapsed_time(e1) / 1e3 / reps) / 1e9
    hbm = measured_peaks().get("hbm_gbs", 6800.0)
    for name, n, N in (("config_8cubed_N8", n_CFG, N_CFG), ("roofline_size_64cubed_N4", (64, 64, 64), 4)):
        dsc = dgg.make_desc((-1.0,) * 3, (1.0,) * 3, n, N)
        with torch.cuda.stream(stream):
            dom = dgg.Domain(n=n, N=N, mg_levels=1, overlap=1, precision="mixed", stream=stream,
                             node_xyz=warp_map(*dgg.host_coordinates(dsc)))
        g64, g32 = rate(dom, "fp64", 5), rate(dom, "fp32", 10)
        out[f"apply_{name}"] = {"dof": dom.n_dof, "fp64_gdofs": g64, "fp32_gdofs": g32,
                                "fp64_hbm_frac": 96.0 * g64 / hbm, "fp32_hbm_frac": 48.0 * g32 / hbm,
                                "algorithmic_bytes_per_dof": {"fp64": 96, "fp32": 48}}
        dom.close()
    return out


TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "subdomain_gemm_traffic_poisson-gauss16-8x8x8-N8.md")
GEMM_SOURCES = ("tc_gemm.cu",)


def gemm_sources_digest():
    import hashlib

    h = hashlib.sha256()
    for name in GEMM_SOURCES:
        with open(os.path.join(ROOT, "paper_2111_06767_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def gemm_traffic_per_launch():
    """DRAM bytes (read + write) per subdomain-GEMM launch from the committed ncu summary, or None
    when the GEMM kernels have changed since those counters were taken (source digest differs)."""
    try:
        with open(TRAFFIC_PROFILE) as f:
            fields = dict(line.strip("- \n").split(": ", 1) for line in f if line.startswith("- ") and ": " in line)
        if fields.get("gemm_sources_sha256") != gemm_sources_digest():
            return None
        return float(fields["traffic_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import workloads
    import paper_2111_06767_gb300 as dgg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    cpu_proc, cpu_threads = None, 0

    stream = torch.cuda.Stream()
    src = workloads.gaussian_source(2)
    doms = {}
    for prec in ("mixed", "fp64"):
        with torch.cuda.stream(stream):
            doms[prec] = dgg.Domain(n=n_CFG, N=N_CFG, penalty=1.5, precision=prec, mg_levels=LEVELS, overlap=2,
                                    stream=stream)
    d = doms["mixed"]
    with torch.cuda.stream(stream):
        x, y, z = d.coordinates()
        f = src(x, y, z).contiguous()
        b = d.rhs(f, stream=stream)
        u = torch.zeros_like(b)
    stream.synchronize()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def timed_solves(dom, steps, warm, profile=False, opts=None):
        times, reps = [], []
        for i in range(warm + steps):
            flush.fill_(float(i))  # evict L2 between steps (outside the timed events)
            torch.cuda.synchronize()
            if profile and i == warm:
                dom.profile(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                u.zero_()
                e0.record(stream)
                rep = dom.solve(b, u, TOL, opts=opts)
                e1.record(stream)
            e1.synchronize()
            if i >= warm:
                times.append(e0.elapsed_time(e1))
                reps.append(rep)
        prof = dom.profile_read() if profile else None
        if profile:
            dom.profile(False)
        return times, reps, prof

    # ---- headline: mixed-precision solves (no instrumentation inside the timed region)
    timed_solves(d, 0, args.warmup)
    barrier()
    torch.cuda.synchronize()
    l0 = dgg.lib().dg_kernel_launches()
    torch.cuda.nvtx.range_push("timed")
    with ClockSampler(local) as clk:
        times, reps, _ = timed_solves(d, args.steps, 0)
    torch.cuda.nvtx.range_pop()
    launches = dgg.lib().dg_kernel_launches() - l0
    barrier()
    # the same K solves again with per-phase CUDA events (event nodes inside the V-cycle graph,
    # read after every replay) for the kernel roofline and the phase breakdown
    _, _, prof = timed_solves(d, args.steps, 0, profile=True)
    total_s = max_over_ranks(sum(times) / 1e3, device="cuda")
    value = whole_job_rate(args.steps, world, total_s)
    u_mixed = u.clone()

    # ---- the same mixed-precision solve with flexible CG instead of FGMRES
    fcg_opts = dgg.solve_opts(krylov="fcg")
    timed_solves(d, 0, 1, opts=fcg_opts)
    tcg, repscg, _ = timed_solves(d, args.steps, 0, opts=fcg_opts)
    fcg = {"value": len(tcg) / (sum(tcg) / 1e3), "unit": "solves/s", "iterations": repscg[0].iterations,
           "relative_residual": max(r.relative_residual for r in repscg),
           "solution_rel_diff_vs_fgmres": float((u - u_mixed).norm() / u_mixed.norm())}

    # ---- plain FP64 solver (same workload), with one profiled solve for its phases
    d64 = doms["fp64"]
    timed_solves(d64, 0, 1)
    t64, reps64, _ = timed_solves(d64, max(2, args.steps // 2), 0)
    value64 = len(t64) / (sum(t64) / 1e3)
    _, _, prof64 = timed_solves(d64, 1, 0, profile=True)
    g64 = prof64["subdomain_gemm"]
    fp64_gemm_tflops = g64["flops"] / max(g64["ms"], 1e-12) / 1e9
    sol_diff = float((u_mixed - u).norm() / u.norm())

    # ---- end to end through the C ABI with host buffers (elliptic_solve_host): the call copies the
    # page-locked host source f to the device, forms b = M f, solves from u = 0 and copies u back
    f_host = f.cpu().pin_memory()
    u_host = torch.zeros_like(f_host).pin_memory()
    e2e_times = []
    for i in range(args.warmup + args.steps):
        flush.fill_(float(i))
        u_host.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep_h = d.solve_host(f_host, u_host, TOL)
        if i >= args.warmup:
            e2e_times.append(time.perf_counter() - t0)
    assert rep_h.status == 0
    e2e_value = world * len(e2e_times) / sum(e2e_times)

    # ---- DG apply rates (config size, L2 resident) and the HBM-sized roofline sweep point
    def apply_rate(dom, prec, reps=20):
        n = dom.n_dof
        dt = torch.float64 if prec == "fp64" else torch.float32
        uu = torch.empty(n, dtype=dt, device="cuda").uniform_(-1, 1)
        out = torch.empty_like(uu)
        fn = (lambda: dom.apply(uu, out, stream=stream)) if prec == "fp64" else (
            lambda: dom.apply_f32(uu, 0, out, stream=stream))
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
        e1.synchronize()
        sec = e0.elapsed_time(e1) / 1e3 / reps
        return n / sec / 1e9, sec

    apply = {"config": {"fp64_gdofs": apply_rate(d64, "fp64")[0], "fp32_gdofs": apply_rate(d, "fp32")[0]}}
    big = dgg.Domain(n=(96, 96, 96), N=4, penalty=1.5, precision="mixed", mg_levels=1, overlap=1, stream=stream)
    g64, s64 = apply_rate(big, "fp64", 5)
    g32, s32 = apply_rate(big, "fp32", 10)
    pk = measured_peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    apply["roofline_size_N4_96cubed"] = {
        "dof": big.n_dof, "fp64_gdofs": g64, "fp32_gdofs": g32,
        "fp32_hbm_frac": 8.0 * g32 / hbm, "fp64_hbm_frac": 16.0 * g64 / hbm,
        "fp64_alu_bound_gdofs": 1.2e12 / (12 * 4 + 12) / 1e9}
    big.close()
    # the sweep over N at about the same size (u + A u far above L2): GDOF/s and the fraction of the
    # HBM copy rate counting u and A u (8 B/DOF in FP32, 16 in FP64)
    if args.apply_sweep:
        sweep = {}
        for Ns, ns in ((4, 96), (5, 77), (6, 64), (7, 55), (8, 48), (9, 43)):
            dm = dgg.Domain(n=(ns,) * 3, N=Ns, penalty=1.5, precision="mixed", mg_levels=1, overlap=1, stream=stream)
            r64, r32 = apply_rate(dm, "fp64", 3)[0], apply_rate(dm, "fp32", 5)[0]
            fl = 12 * Ns + 12  # flop per DOF of the sum-factorised operator
            roof32 = min(hbm / 8.0, FP32_PEAK_TFLOPS * 1e3 / fl)  # GDOF/s: HBM (8 B/DOF) or the FP32 pipe
            roof64 = min(hbm / 16.0, FP64_PEAK_TFLOPS * 1e3 / fl)
            sweep[f"N{Ns}_{ns}cubed"] = {
                "dof": dm.n_dof, "fp32_gdofs": r32, "fp32_hbm_frac": 8.0 * r32 / hbm,
                "fp32_pipe_frac": r32 * fl / (FP32_PEAK_TFLOPS * 1e3),
                "fp32_binding_roof": "hbm" if roof32 == hbm / 8.0 else "fp32 pipe", "fp32_roof_frac": r32 / roof32,
                "fp64_gdofs": r64, "fp64_hbm_frac": 16.0 * r64 / hbm, "fp64_flop_rate_tflops": r64 * fl / 1e3,
                "fp64_pipe_frac": r64 * fl / (FP64_PEAK_TFLOPS * 1e3), "fp64_roof_frac": r64 / roof64}
            dm.close()
        apply["sweep"] = sweep

    # ---- roofline of the dominant kernel phase of the timed solves
    dom_phase = max(prof, key=lambda k: prof[k]["ms"])
    ph = prof[dom_phase]
    achieved_gbs = ph["bytes"] / (ph["ms"] / 1e3) / 1e9
    achieved_tf = ph["flops"] / (ph["ms"] / 1e3) / 1e12
    # peaks: HBM copy bandwidth (measured); the TF32 tensor-core peak derived from the measured
    # sustained BF16 cuBLAS rate x the nominal TF32/BF16 dense ratio (1.1 / 2.25 PFLOP/s); the FP32
    # SIMT peak from the unit count (152 SMs x 128 lanes x 2 flops) x the median SM clock under load
    clk_sum = clk.summary()
    sm_mhz = clk_sum["sm_mhz"] or pk.get("sm_max_mhz", 2070.0)
    tf32_peak = pk.get("bf16_tflops_sustained", 1700.0) * (1.1 / 2.25)
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    tensor = dom_phase == "subdomain_gemm" and d.desc.subdomain_gemm != dgg.GEMM_MODES["simt"]
    peak_flops = tf32_peak if tensor else fp32_peak
    intensity = ph["flops"] / max(ph["bytes"], 1.0)
    ridge = peak_flops * 1e12 / (hbm * 1e9)
    if intensity < ridge:
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s", "frac": achieved_gbs / hbm,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    elif tensor:
        roof = {"bound": "tensor", "achieved": achieved_tf, "peak": tf32_peak, "unit": "TFLOP/s",
                "frac": achieved_tf / tf32_peak,
                "peak_source": "TF32 = measured sustained BF16 (MEASURED_PEAKS.json) x nominal 1.1/2.25"}
    else:
        roof = {"bound": "alu", "achieved": achieved_tf, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved_tf / fp32_peak, "peak_source": "FP32 SIMT: 152 SM x 128 lanes x 2 x median SM clock"}
    traffic = gemm_traffic_per_launch() if dom_phase == "subdomain_gemm" else None
    roof.update({"kernel": dom_phase, "traffic": traffic, "launches": ph["launches"],
                 "measured": "CUDA events around every launch of the phase, on the solve stream, over a second run "
                             "of the same K solves right after the timed region",
                 "avg_launch_ms": ph["ms"] / max(ph["launches"], 1), "bytes_per_launch": ph["bytes"] / max(ph["launches"], 1)})
    phases = {k: {"launches": v["launches"], "ms": round(v["ms"], 4),
                  "share": round(v["ms"] / max(sum(p["ms"] for p in prof.values()), 1e-12), 4),
                  "GB/s": round(v["bytes"] / max(v["ms"], 1e-12) / 1e6, 1)} for k, v in prof.items()}

    concurrent = concurrent_run(dgg, workloads, torch, args.concurrent) if args.concurrent > 0 and rank == 0 else None
    served = (served_compare(dgg, workloads, args.served_seconds, args.served_fp64_seconds, args.served_streams)
              if args.served_seconds > 0 and rank == 0 else None)
    batched = (batched_compare(dgg, workloads, torch, args.batched, args.batched_fp64)
               if args.batched > 0 and rank == 0 else None)
    punct = (puncture_compare(dgg, workloads, torch, stream, args.puncture_steps)
             if args.puncture_steps > 0 and rank == 0 else None)
    curv = (curved_compare(dgg, workloads, torch, stream, args.curved_steps)
            if args.curved_steps > 0 and rank == 0 else None)

    if rank == 0 and not args.no_cpu:
        # the oracle sample runs in its own interpreter after the GPU legs, on all host cores: beside
        # them its BLAS threads would compete with the server's and the host-driven solves' threads
        cpu_threads = oracle_threads()
        cpu_proc = start_cpu_sample(2, 420.0, cpu_threads)
    cpu = finish_cpu_sample(cpu_proc, cpu_threads) if cpu_proc is not None else None
    if cpu is not None:
        cpu = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}
    lat = sorted(times)
    p50 = lat[len(lat) // 2]
    p99 = lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "FP32 V-cycle (smoother, explicit subdomain inverses, "
                   "transfers) under FP64 FGMRES", "solves_per_step_per_gpu": 1, "parallelism": f"replicas x{world}",
                   "l2": "256 MB buffer written between timed steps (outside the events)"},
        "clocks": clk_sum,
        "latency_ms": {"p50": p50, "p99": p99},
        "iterations": reps[0].iterations, "relative_residual": max(r.relative_residual for r in reps),
        "fp64": {"value": value64, "unit": "solves/s", "iterations": reps64[0].iterations,
                 "relative_residual": max(r.relative_residual for r in reps64),
                 "mixed_vs_fp64_solution_rel_diff": sol_diff, "mixed_speedup": value / value64 / world,
                 "phases_ms": {k: round(v["ms"], 3) for k, v in prof64.items() if v["launches"]},
                 "subdomain_gemm_tflops": fp64_gemm_tflops,
                 "subdomain_gemm_frac_of_fp64_pipe": fp64_gemm_tflops / FP64_PEAK_TFLOPS,
                 "fp64_peak": f"{FP64_PEAK_TFLOPS} TFLOP/s, FP64 FMA rate probed on this pool's GB300"},
        "fcg": fcg,
        "dg_apply": apply,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": 2 * f.numel() * 8,
                "d2h_bytes_per_step": u.numel() * 8,
                "call": "elliptic_solve_host (C ABI): host f and u in, host u out, page-locked buffers"},
        "gpu_launches": int(launches),
        "roofline": roof,
        "phases": phases,
        "served": served,
        "batched": batched,
        "concurrent": concurrent,
        "puncture_16cubed_N6": punct,
        "curved_warped_8cubed_N8": curv,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_case(a):
    """One operation of the solver a few times on a seeded input, for kernel profiling under ncu
    (--case smooth|apply|vcycle|solve; [-1,1]^3 with --n^3 elements and --N points per dimension).
    smooth: Schwarz smoothing steps on the finest level (residual apply, gather, subdomain GEMM,
    scatter); apply: the DG operator alone (FP32 for --precision mixed, FP64 otherwise); vcycle:
    full V-cycles; solve: FGMRES solves to 1e-10 of the 16-Gaussian source (one untimed solve first,
    then --reps solves inside the NVTX range "timed", a 256 MB buffer written before each so that L2
    starts cold). --warp: curved elements (a smooth warp of the box's nodes)."""
    import torch

    import paper_2111_06767_gb300 as dgg

    xyz = None
    if a.warp:
        xyz = warp_map(*dgg.host_coordinates(dgg.make_desc((-1.0,) * 3, (1.0,) * 3, (a.n,) * 3, a.N)))
    d = dgg.Domain(n=(a.n,) * 3, N=a.N, precision=a.precision, mg_levels=a.levels, overlap=2, gemm=a.gemm,
                   node_xyz=xyz)
    g = torch.Generator(device="cuda").manual_seed(7)
    dt = torch.float32 if (a.case == "apply" and a.precision == "mixed") else torch.float64
    x = torch.empty(d.n_dof, dtype=dt, device="cuda").uniform_(-1, 1, generator=g)
    y = torch.zeros_like(x)
    if a.case == "solve":
        import workloads

        X, Y, Z = d.coordinates()
        b = d.rhs(workloads.gaussian_source(2)(X, Y, Z).contiguous())
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        d.solve(b, y, TOL)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        for i in range(a.reps):
            flush.fill_(float(i))
            y.zero_()
            d.solve(b, y, TOL)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    else:
        for _ in range(a.reps):
            if a.case == "apply":
                if dt == torch.float32:
                    d.apply_f32(x, 0, y)
                else:
                    d.apply(x, y)
            elif a.case == "smooth":
                d.schwarz_smooth(0, x, y, 1)
            else:
                d.vcycle(x, y)
        torch.cuda.synchronize()
    print(f"{a.case} done: n={a.n}^3 N={a.N} dof={d.n_dof}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--oracle-workload", choices=["gauss", "sine"], default="gauss",
                    help="problem of the oracle sample (--impl reference): the headline 8^3 Gaussian workload, "
                         "or the small 2^3 sine problem (quick CPU checks of this script)")
    ap.add_argument("--served-seconds", type=float, default=20.0, help="arrival window of the served stream (0: skip)")
    ap.add_argument("--served-streams", type=int, default=8,
                    help="solves the server runs at once (one worker thread and CUDA stream each)")
    ap.add_argument("--served-fp64-seconds", type=float, default=0.25,
                    help="arrival window replayed in both precisions for the mixed/FP64 ratio (0: skip)")
    ap.add_argument("--batched", type=int, default=512, help="also run this many batched uneven solves (0: skip)")
    ap.add_argument("--concurrent", type=int, default=8,
                    help="also solve the headline problem on this many streams at once (0: skip)")
    ap.add_argument("--batched-fp64", type=int, default=32,
                    help="prefix of the batched stream also solved in plain FP64 for the mixed/FP64 ratio")
    ap.add_argument("--puncture-steps", type=int, default=2,
                    help="timed solves of the 16^3 puncture workload per subdomain solver (0: skip)")
    ap.add_argument("--no-apply-sweep", dest="apply_sweep", action="store_false",
                    help="skip the DG-apply sweep over N = 4..9 at about 56M DOF")
    ap.add_argument("--curved-steps", type=int, default=3,
                    help="timed mixed solves of the warped-mesh workload (0: skip the curved leg)")
    ap.add_argument("--case", choices=["smooth", "apply", "vcycle", "solve"],
                    help="profiling harness: run one operation --reps times and exit (no JSON line)")
    ap.add_argument("--n", type=int, default=8, help="--case: elements per dimension")
    ap.add_argument("--N", type=int, default=8, help="--case: LGL points per dimension")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed", help="--case: precision")
    ap.add_argument("--gemm", choices=["default", "simt", "tf32"], default="default", help="--case: subdomain GEMM")
    ap.add_argument("--levels", type=int, default=1, help="--case: multigrid levels")
    ap.add_argument("--reps", type=int, default=3, help="--case: repetitions")
    ap.add_argument("--warp", action="store_true", help="--case: curved elements (a smooth warp of the box)")
    args = ap.parse_args()
    if args.case:
        run_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
