"""Continuous-batching server (elliptic_serve_*): requests of different sizes, orders and problem
kinds run concurrently; every result equals the same request solved alone (FP64 domains,
deterministic kernels and reductions: agreement to 1e-12 relative), and the queue reports BUSY /
NOT_FOUND / INVALID_ARG as documented."""
import time

import numpy as np
import pytest
import torch

import workloads
from gpu_util import box, rel

pytestmark = pytest.mark.gpu

dgg = pytest.importorskip("paper_2111_06767_gb300")
from paper_2111_06767_gb300 import _native  # noqa: E402


def _request(kind, n, N, seed):
    if kind == "poisson":
        desc = dgg.make_desc((-1.0,) * 3, (1.0,) * 3, (n,) * 3, N, precision="fp64", overlap=2)
        grid = box((n,) * 3, N)
        x, y, z = grid.coordinates()
        f = workloads.gaussian_source(seed)(x, y, z).ravel()
    else:
        desc = dgg.make_desc((-20.0,) * 3, (20.0,) * 3, (n,) * 3, N, precision="fp64", overlap=2, problem="puncture",
                             punctures=workloads.BINARY_PUNCTURES)
        f = None
    return desc, f


def _alone(desc, f, tol):
    lo, hi, n = tuple(desc.lower), tuple(desc.upper), tuple(desc.n)
    kind = "puncture" if desc.problem == 1 else "poisson"
    d = dgg.Domain(lo, hi, n, desc.N, precision="fp64", overlap=2, problem=kind,
                   punctures=workloads.BINARY_PUNCTURES if kind == "puncture" else ())
    u = torch.zeros(d.n_dof, dtype=torch.float64, device="cuda")
    if kind == "poisson":
        b = d.rhs(torch.from_numpy(f).cuda())
        d.solve(b, u, tol, opts=dgg.solve_opts(relative_to_b=True))
    else:
        d.solve(None, u, tol)
    return u.cpu().numpy()


def test_results_alone_equal_results_in_the_mix():
    reqs = [("poisson", 4, 5, 11), ("puncture", 2, 4, 0), ("poisson", 2, 6, 12), ("poisson", 3, 4, 13),
            ("puncture", 4, 5, 0), ("poisson", 6, 4, 14)]
    srv = dgg.Server(max_active=3, n_streams=3)
    tickets = []
    for kind, n, N, seed in reqs:
        desc, f = _request(kind, n, N, seed)
        tickets.append((srv.submit(desc, f, tol=1e-10), desc, f))
    results = {}
    t0 = time.time()
    while len(results) < len(tickets) and time.time() - t0 < 300:
        for t, desc, f in tickets:
            if t in results:
                continue
            u = np.empty(desc.n[0] * desc.n[1] * desc.n[2] * desc.N**3)
            st, res = srv.poll(t, u)
            if st != _native.DG_PENDING:
                results[t] = (st, res.report.relative_residual, u, res.submit_time, res.admit_time,
                              res.finish_time)
        time.sleep(0.01)
    assert len(results) == len(tickets)
    # requests overlapped on the device: some admission happened before an earlier finish
    finishes = sorted(r[5] for r in results.values())
    assert min(r[4] for r in results.values()) < finishes[-1]
    for t, desc, f in tickets:
        st, relres, u, *_ = results[t]
        assert st == _native.DG_OK and relres <= 1e-10
        assert rel(u, _alone(desc, f, 1e-10)) < 1e-12
    assert srv.poll(tickets[0][0])[0] == -8  # a returned ticket is released
    srv.close()


def test_queue_errors():
    srv = dgg.Server(max_active=1, queue_capacity=1, n_streams=1, memory_budget_bytes=1 << 30)
    st, _ = srv.poll(12345)
    assert st == -8  # DG_ERR_NOT_FOUND
    big, _ = _request("poisson", 64, 8, 1)
    with pytest.raises(dgg.NativeError) as e:
        srv.submit(big, np.zeros(64**3 * 8**3), tol=1e-8)  # 134M points can never fit 1 GiB
    assert e.value.status == -1
    desc, f = _request("poisson", 6, 8, 2)
    t1 = srv.submit(desc, f, tol=1e-10)
    busy = 0
    for _ in range(5):  # the single worker holds one request; the queue holds one more
        try:
            srv.submit(desc, f, tol=1e-10)
        except dgg.NativeError as err:
            assert err.status == -7  # DG_ERR_BUSY
            busy += 1
    assert busy >= 3
    srv.close()


def test_curved_coefficient_and_neumann_requests_in_the_mix():
    """Requests with curved elements (node coordinates), a variable coefficient and Neumann faces are
    served beside plain ones; the server copies the per-node arrays at submission, and every result
    equals the same request solved alone."""
    warp = lambda X, Y, Z: (X + 0.1 * (1 - X**2) * Y, Y + 0.12 * (1 - Y**2) * Z * X, Z + 0.1 * (1 - Z**2) * (X + Y))
    specs = [dict(n=(4, 4, 4), N=4, mapping=warp), dict(n=(3, 3, 3), N=5, coef=True),
             dict(n=(4, 4, 4), N=4, neumann=(0, 1)), dict(n=(2, 2, 2), N=6),
             dict(n=(2, 3, 2), N=4, mapping=warp, coef=True, neumann=(4,))]
    srv = dgg.Server(max_active=3, n_streams=3)
    jobs = []
    for i, sp in enumerate(specs):
        grid = box(sp["n"], sp["N"])
        x, y, z = grid.coordinates()
        xyz = warp(x, y, z) if sp.get("mapping") else None
        px, py, pz = xyz if xyz else (x, y, z)
        coef = 1.0 + 0.5 * px**2 + 0.2 * np.tanh(py * pz) if sp.get("coef") else None
        kw = dict(precision="fp64", overlap=2, neumann=sp.get("neumann", ()), node_xyz=xyz, coef=coef)
        desc = dgg.make_desc((-1.0,) * 3, (1.0,) * 3, sp["n"], sp["N"], **kw)
        f = workloads.gaussian_source(20 + i)(px, py, pz).ravel()
        jobs.append((srv.submit(desc, f, tol=1e-10), sp, kw, f))
        del desc  # the server holds its own copies
    results = {}
    t0 = time.time()
    while len(results) < len(jobs) and time.time() - t0 < 300:
        for t, sp, kw, f in jobs:
            if t in results:
                continue
            u = np.empty(int(np.prod(sp["n"])) * sp["N"] ** 3)
            st, res = srv.poll(t, u)
            if st != _native.DG_PENDING:
                results[t] = (st, res.report.relative_residual, u)
        time.sleep(0.01)
    assert len(results) == len(jobs)
    for t, sp, kw, f in jobs:
        st, relres, u = results[t]
        assert st == _native.DG_OK and relres <= 1e-10, sp
        d = dgg.Domain((-1.0,) * 3, (1.0,) * 3, sp["n"], sp["N"], **kw)
        b = d.rhs(torch.from_numpy(f).cuda())
        ua = torch.zeros_like(b)
        d.solve(b, ua, 1e-10, opts=dgg.solve_opts(relative_to_b=True))
        assert rel(u, ua.cpu().numpy()) < 1e-12, sp
    srv.close()


def test_cancel_waiting_and_running_requests():
    """With one worker: a long FP64 request is cancelled while it runs (the solve stops at its next
    Krylov iteration), a queued one is cancelled before admission, and the remaining request is
    served as if alone; tickets that were never issued report NOT_FOUND."""
    srv = dgg.Server(max_active=1, n_streams=1)
    long_desc, long_f = _request("poisson", 12, 8, 30)  # FP64 12^3, N = 8: over a second with its set-up
    short_desc, short_f = _request("poisson", 2, 4, 31)
    t_long = srv.submit(long_desc, long_f, tol=1e-10)
    t_queued = srv.submit(short_desc, short_f, tol=1e-10)
    t_kept = srv.submit(short_desc, short_f, tol=1e-10)
    assert srv.cancel(t_queued) == 0
    time.sleep(0.15)  # the long request is admitted at once and runs for several hundred ms
    assert srv.cancel(t_long) == 0
    status = {}
    t0 = time.time()
    while len(status) < 3 and time.time() - t0 < 120:
        for t in (t_long, t_queued, t_kept):
            if t in status:
                continue
            u = np.empty(2**3 * 4**3) if t == t_kept else None
            st, res = srv.poll(t, u)
            if st != _native.DG_PENDING:
                status[t] = (st, u, res.report.iterations)
        time.sleep(0.01)
    assert status[t_queued][0] == _native.DG_ERR_CANCELLED
    assert status[t_long][0] == _native.DG_ERR_CANCELLED
    assert status[t_kept][0] == _native.DG_OK
    assert rel(status[t_kept][1], _alone(short_desc, short_f, 1e-10)) < 1e-12
    assert srv.cancel(10**9) == -8 and srv.poll(10**9)[0] == -8
    srv.close()
