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
TOL = 1e-10

# CPU sample of the same workload for the oracle timings: the same problem family on 2^3 elements
# (4,096 DOF, 2 levels); multigrid-Schwarz iteration counts do not depend on h, so the per-solve
# work scales with the number of points and the rate is scaled by 4,096 / 262,144.
SAMPLE_N_ELEMS = (2, 2, 2)

_SAMPLE_SCRIPT = r"""
import json, os, sys, time
sys.path.insert(0, sys.argv[1])
import numpy as np
import workloads
from oracle import dg, solve
steps, warm = int(sys.argv[2]), int(sys.argv[3])
grid = dg.BoxGrid((-1.0,)*3, (1.0,)*3, (2, 2, 2), 8, 1.5)
pr = solve.Problem(grid, mg_levels=0, overlap=2)
x, y, z = grid.coordinates()
b = dg.rhs(pr.graphs[0], workloads.gaussian_source(2)(x, y, z))
times, its = [], []
for i in range(warm + steps):
    t0 = time.perf_counter()
    u, info = pr.solve_linear(b, tol=1e-10)
    dt = time.perf_counter() - t0
    if i >= warm:
        times.append(dt); its.append(info["iterations"])
print(json.dumps({"times": times, "iterations": its, "dof": int(b.size)}))
"""


def cpu_sample(steps: int, warm: int):
    """Time the oracle's multigrid-Schwarz FGMRES solve of the 2^3-element sample in a fresh
    interpreter with all host cores available to its BLAS."""
    cores = os.cpu_count() or 1
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(cores)
    out = subprocess.run([sys.executable, "-c", _SAMPLE_SCRIPT, ROOT, str(steps), str(warm)], capture_output=True,
                         text=True, env=env, check=True)
    res = json.loads(out.stdout.strip().splitlines()[-1])
    scale = res["dof"] / (n_CFG[0] * n_CFG[1] * n_CFG[2] * N_CFG**3)
    rates = [scale / t for t in res["times"]]  # config-size solves per second
    return res, rates, cores


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    res, rates, cores = cpu_sample(args.steps, min(args.warmup, 1))
    total = sum(res["times"])
    value = len(res["times"]) * (res["dof"] / (n_CFG[0] * n_CFG[1] * n_CFG[2] * N_CFG**3)) / total
    sample = (f"oracle (numpy FP64) MG-Schwarz FGMRES solve of the same problem on 2^3 elements, N=8 "
              f"({res['dof']} DOF, {res['iterations'][0]} iterations), subdomain matrices built in an untimed "
              f"warm-up solve, rate scaled by {res['dof']}/262144 DOF")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(res["times"]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample},
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


def served_run(dgg, workloads, duration, rate=200.0, seed=5, max_active=4, precision="mixed"):
    """Poisson-process arrivals of Poisson / puncture requests (n ~ U{2..12} cubic, N ~ U{4..8}) into the
    continuous-batching server; latency = completion - scheduled arrival."""
    import time as _t

    arr = workloads.poisson_arrivals(seed, rate, duration)
    reqs = build_requests(dgg, workloads, [(k, n, N, rs) for _, k, n, N, rs in arr], precision=precision)
    srv = dgg.Server(max_active=max_active, n_streams=max_active, queue_capacity=1 << 20)
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
            "solves_per_s": len(reqs) / total, "p50_latency_ms": pick(0.5), "p99_latency_ms": pick(0.99),
            "ok": sum(1 for v in done.values() if v[0] == 0), "max_relative_residual": max(v[2] for v in done.values()),
            "max_active": max_active,
            "precision": "mixed (TF32 subdomain GEMM, FP64 FGMRES)" if precision == "mixed" else "fp64"}


def served_compare(dgg, workloads, duration, prefix):
    """The served stream in MIXED precision, and the first `prefix` seconds of arrivals in both
    precisions (the plain FP64 solver on the same requests, for the mixed/FP64 throughput ratio)."""
    out = served_run(dgg, workloads, duration)
    if prefix > 0:
        m = served_run(dgg, workloads, prefix)
        f = served_run(dgg, workloads, prefix, precision="fp64")
        out["prefix"] = {"window_s": prefix, "mixed": m, "fp64": f,
                         "mixed_over_fp64_solves_per_s": m["solves_per_s"] / f["solves_per_s"]}
    return out


def batched_run(dgg, workloads, count=512, seed=4, max_active=8, precision="mixed"):
    """`count` independent Poisson solves of uneven shapes (n_i ~ U{2..8}, N ~ U{4..9}), all submitted
    at once; domains are built inside the run (explicit inverses come from the library cache after
    the first of each shape)."""
    shapes = workloads.batched_shapes(seed, count)
    reqs = build_requests(dgg, workloads, [("poisson", n, N, seed + k) for k, (n, N) in enumerate(shapes)],
                          precision=precision)
    srv = dgg.Server(max_active=max_active, n_streams=max_active, queue_capacity=1 << 20)
    start = srv.clock()
    pending = {srv.submit(d, f, tol=1e-10): k for k, (d, f) in enumerate(reqs)}
    res_ok, worst = 0, 0.0
    while pending:
        for tk in list(pending):
            st, res = srv.poll(tk)
            if st != 1:
                pending.pop(tk)
                res_ok += st == 0
                worst = max(worst, res.report.relative_residual)
    total = srv.clock() - start
    srv.close()
    return {"solves": count, "precision": precision, "solves_per_s": count / total, "seconds": total, "ok": res_ok,
            "max_relative_residual": worst, "max_active": max_active}


def batched_compare(dgg, workloads, count, fp64_count):
    """The batched stream in MIXED precision, and its first `fp64_count` solves in both precisions
    (plain FP64 on the GPU is ~50x slower, so it runs on a prefix of the same stream)."""
    out = {"mixed": batched_run(dgg, workloads, count)}
    if fp64_count > 0:
        out["prefix_mixed"] = batched_run(dgg, workloads, fp64_count)
        out["prefix_fp64"] = batched_run(dgg, workloads, fp64_count, precision="fp64")
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

    cpu = None
    if rank == 0 and not args.no_cpu:
        # before the first GPU work: the oracle runs in its own interpreter
        res, rates, cores = cpu_sample(1, 1)
        cpu = {"value": rates[0], "unit": "solves/s", "cores": cores, "kind": "oracle",
               "sample": (f"oracle (numpy FP64) MG-Schwarz FGMRES solve of the same problem on 2^3 elements, N=8 "
                          f"({res['dof']} DOF, {res['iterations'][0]} iterations, {res['times'][0]:.1f} s after an "
                          f"untimed warm-up that builds the subdomain matrices), rate scaled by "
                          f"{res['dof']}/262144 DOF")}

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

    # ---- plain FP64 solver (same workload)
    d64 = doms["fp64"]
    timed_solves(d64, 0, 1)
    t64, reps64, _ = timed_solves(d64, max(2, args.steps // 2), 0)
    value64 = len(t64) / (sum(t64) / 1e3)
    sol_diff = float((u_mixed - u).norm() / u.norm())

    # ---- end to end through the public API: pinned host f -> device, solve, solution -> host
    f_host = f.cpu().pin_memory()
    u_host = torch.empty_like(f_host).pin_memory()
    f_dev = torch.empty_like(f)
    e2e_times = []
    for i in range(args.warmup + args.steps):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            f_dev.copy_(f_host, non_blocking=True)
            d.rhs(f_dev, b, stream=stream)
            u.zero_()
            d.solve(b, u, TOL)
            u_host.copy_(u, non_blocking=True)
        stream.synchronize()
        if i >= args.warmup:
            e2e_times.append(time.perf_counter() - t0)
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
            sweep[f"N{Ns}_{ns}cubed"] = {"dof": dm.n_dof, "fp32_gdofs": r32, "fp32_hbm_frac": 8.0 * r32 / hbm,
                                         "fp64_gdofs": r64, "fp64_hbm_frac": 16.0 * r64 / hbm,
                                         "fp64_flop_rate_tflops": r64 * (12 * Ns + 12) / 1e3}
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
    served = (served_compare(dgg, workloads, args.served_seconds, args.served_fp64_seconds)
              if args.served_seconds > 0 and rank == 0 else None)
    batched = (batched_compare(dgg, workloads, args.batched, args.batched_fp64)
               if args.batched > 0 and rank == 0 else None)
    punct = (puncture_compare(dgg, workloads, torch, stream, args.puncture_steps)
             if args.puncture_steps > 0 and rank == 0 else None)
    curv = (curved_compare(dgg, workloads, torch, stream, args.curved_steps)
            if args.curved_steps > 0 and rank == 0 else None)

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
                 "mixed_vs_fp64_solution_rel_diff": sol_diff, "mixed_speedup": value / value64 / world},
        "fcg": fcg,
        "dg_apply": apply,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": f.numel() * 8,
                "d2h_bytes_per_step": u.numel() * 8},
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--served-seconds", type=float, default=2.0, help="arrival window of the served stream (0: skip)")
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
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
