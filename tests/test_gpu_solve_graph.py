"""Whole solves as CUDA graphs: FGMRES (Sec. III.B) with its Hessenberg column, Givens rotations and
stopping test computed on the device and the Arnoldi loop as a conditional WHILE node, so that a
solve is one graph launch with no host round trip per iteration; and many solves of different
shapes captured as one graph (elliptic_batch_*).

The captured solve runs the same kernels on the same data as the host-driven one, with the same
reduction trees for every inner product; only the rotations are computed on the device instead of
the host (hypot and the divisions may round differently), so solutions agree to rounding and the
iteration counts are equal. Every solution is also checked against the oracle's dense direct solve
where that is small enough. These small problems are solved to a 1e-11 residual: at 1e-10 their
solutions are 1.3e-10 from the direct solution (the residual bounds the error only up to the
condition number), so the tolerance is tightened until the 1e-10 solution parity holds."""
import numpy as np
import pytest
import torch

import workloads
from gpu_util import box, rel
from oracle import dg, solve

pytestmark = pytest.mark.gpu

dgg = pytest.importorskip("paper_2111_06767_gb300")
nat = dgg._native


def _gauss_rhs(d, n, N, seed=2):
    grid = box(n, N)
    x, y, z = grid.coordinates()
    f = workloads.gaussian_source(seed)(x, y, z)
    return d.rhs(torch.from_numpy(f.ravel()).cuda()), f


def _direct(n, N, f):
    grid = box(n, N)
    pr = solve.Problem(grid)
    return np.linalg.solve(dg.assemble(pr.graphs[0]), dg.rhs(pr.graphs[0], f).ravel())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("relative_to_b", [False, True])
def test_captured_solve_equals_host_driven_solve(precision, relative_to_b, monkeypatch):
    n, N = (4, 2, 2), 5
    out = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("DG_SOLVE_GRAPH", mode)
        d = dgg.Domain(n=n, N=N, precision=precision)
        b, f = _gauss_rhs(d, n, N)
        runs = []
        for _ in range(3):  # host-driven (tunes), captured and launched, launched again
            u = torch.zeros_like(b)
            k0 = nat.load().dg_kernel_launches()
            rep = d.solve(b, u, tol=1e-11, opts=dgg.solve_opts(relative_to_b=relative_to_b))
            launched = nat.load().dg_kernel_launches() - k0
            assert rep.status == 0 and rep.relative_residual <= 1e-11
            runs.append((u.cpu().numpy(), rep.iterations, launched))
        out[mode] = runs
    ud = _direct(n, N, f)
    host, graph = out["0"], out["1"]
    for (uh, ih, _), (ug, ig, lg) in zip(host, graph):
        assert ig == ih
        assert rel(ug, uh) <= 1e-12
        assert rel(ug, ud) <= 1e-10
        assert lg > 10 * ig  # the kernels of the captured solve are counted
    assert np.array_equal(graph[1][0], graph[2][0])  # a replay is bitwise reproducible


def test_captured_solve_restarts_host_driven_past_its_column_cap(monkeypatch):
    """With the captured solve limited to 3 Arnoldi columns, a solve needing more continues
    host-driven from the graph's iterate (a restart) and still reaches the direct solution."""
    n, N = (2, 2, 2), 6
    monkeypatch.setenv("DG_SOLVE_GRAPH_CAP", "3")
    d = dgg.Domain(n=n, N=N, precision="fp64")
    b, f = _gauss_rhs(d, n, N)
    ud = _direct(n, N, f)
    for _ in range(3):
        u = torch.zeros_like(b)
        rep = d.solve(b, u, tol=1e-11)
        assert rep.status == 0 and rep.relative_residual <= 1e-11 and rep.iterations > 3
        assert rel(u.cpu().numpy(), ud) <= 1e-10
    u = torch.zeros_like(b)
    rep = d.solve(b, u, tol=1e-11, opts=dgg.solve_opts(max_iterations=3), check_status=False)
    assert rep.status == -4  # DG_ERR_NOT_CONVERGED
    assert rep.iterations == 3


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_of_uneven_solves_in_one_graph(precision):
    """Six solves of different element counts and orders (prime counts: Schwarz-only levels) in one
    captured graph, run twice; each equals the same problem solved alone to rounding and the
    direct solution to 1e-10. The domains are released before the batch (allowed: destroying a batch
    does not touch its domains)."""
    shapes = [((2, 3, 2), 4), ((3, 3, 3), 5), ((4, 4, 2), 6), ((2, 2, 2), 8), ((5, 2, 3), 4), ((4, 4, 4), 4)]
    doms, bs, us, fs = [], [], [], []
    for i, (n, N) in enumerate(shapes):
        d = dgg.Domain(n=n, N=N, precision=precision)
        b, f = _gauss_rhs(d, n, N, seed=40 + i)
        doms.append(d)
        bs.append(b)
        us.append(torch.zeros_like(b))
        fs.append(f)
    batch = dgg.Batch(doms, bs, us, tol=1e-11)
    for rnd in range(2):
        for u in us:
            u.zero_()
        reps = batch.run()
        for i, ((n, N), rep) in enumerate(zip(shapes, reps)):
            assert rep.status == 0 and rep.relative_residual <= 1e-11, (rnd, i, rep)
            assert rel(us[i].cpu().numpy(), _direct(n, N, fs[i])) <= 1e-10, (rnd, i)
    for i, (n, N) in enumerate(shapes):  # alone
        u = torch.zeros_like(bs[i])
        rep = doms[i].solve(bs[i], u, tol=1e-11)
        assert rep.iterations == reps[i].iterations
        assert rel(u.cpu().numpy(), us[i].cpu().numpy()) <= 1e-12
    for d in doms:
        d.close()
    batch.close()


def test_batch_rejects_a_domain_twice_and_nonlinear_problems():
    d = dgg.Domain(n=(2, 2, 2), N=4)
    b, _ = _gauss_rhs(d, (2, 2, 2), 4)
    u = torch.zeros_like(b)
    with pytest.raises(nat.NativeError, match="twice"):
        dgg.Batch([d, d], [b, b], [u, u])
    p = dgg.Domain((-20.0,) * 3, (20.0,) * 3, (2, 2, 2), 4, problem="puncture", punctures=workloads.BINARY_PUNCTURES)
    with pytest.raises(nat.NativeError, match="Poisson"):
        dgg.Batch([p], [b], [u])
