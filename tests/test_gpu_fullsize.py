"""Parity at the full sizes of the benchmark workloads, in the configuration bench.py times.

The oracle cannot run the full multigrid solves at these sizes within a test, so the GPU
solutions are checked through properties that hold at any size: the oracle's own FP64 operator
(Sec. II) applied to the GPU solution must leave a residual at the solver's tolerance, the mixed
and FP64 solvers must agree with each other, and the Newton path must take the same steps."""
import numpy as np
import pytest
import torch

import workloads
from gpu_util import box, rel
from oracle import dg, puncture

pytestmark = pytest.mark.gpu

dgg = pytest.importorskip("paper_2111_06767_gb300")


def test_gaussian_8x8x8_N8_three_levels():
    """16 Gaussians, 8^3 elements, N = 8, 3-level V-cycle, N_overlap = 2 (262,144 DOF)."""
    n, N = (8, 8, 8), 8
    grid = box(n, N)
    x, y, z = grid.coordinates()
    f = workloads.gaussian_source(2)(x, y, z)
    graph = grid.graph()
    b_ref = dg.rhs(graph, f).ravel()
    sols = {}
    for precision in ("fp64", "mixed"):
        d = dgg.Domain(n=n, N=N, precision=precision, mg_levels=3, overlap=2)
        b = d.rhs(torch.from_numpy(f.ravel()).cuda())
        u = torch.zeros_like(b)
        rep = d.solve(b, u, tol=1e-10)
        assert rep.status == 0 and rep.relative_residual <= 1e-10
        assert rel(b.cpu().numpy(), b_ref) < 1e-14
        uh = u.cpu().numpy()
        r = b_ref - dg.apply(graph, uh.reshape(-1, N, N, N)).ravel()
        assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b_ref)
        sols[precision] = (uh, rep.iterations)
    assert rel(sols["mixed"][0], sols["fp64"][0]) < 1e-10
    assert abs(sols["mixed"][1] - sols["fp64"][1]) <= 1
    # the flexible conjugate gradient method on the same problem (mixed precision)
    d = dgg.Domain(n=n, N=N, precision="mixed", mg_levels=3, overlap=2)
    b = d.rhs(torch.from_numpy(f.ravel()).cuda())
    u = torch.zeros_like(b)
    rep = d.solve(b, u, tol=1e-10, opts=dgg.solve_opts(krylov="fcg"))
    assert rep.status == 0 and rep.relative_residual <= 1e-10
    uh = u.cpu().numpy()
    r = b_ref - dg.apply(graph, uh.reshape(-1, N, N, N)).ravel()
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b_ref)
    assert rel(uh, sols["fp64"][0]) < 1e-10


def test_puncture_16x16x16_N6_newton():
    """Binary punctures on [-20,20]^3, 16^3 elements, N = 6 (884,736 DOF), Newton-Krylov with the
    FP32 Schwarz smoother under FP64 FGMRES."""
    n, N = (16, 16, 16), 6
    grid = box(n, N, lower=(-20.0,) * 3, upper=(20.0,) * 3)
    graph = grid.graph()
    x, y, z = grid.coordinates()
    alpha, beta = puncture.alpha_beta(x, y, z, workloads.BINARY_PUNCTURES)
    mass = dg.mass_diag(graph)
    sols = {}
    for precision in ("fp64", "mixed"):
        d = dgg.Domain((-20.0,) * 3, (20.0,) * 3, n, N, precision=precision, overlap=2, problem="puncture",
                       punctures=workloads.BINARY_PUNCTURES)
        u = torch.zeros(d.n_dof, dtype=torch.float64, device="cuda")
        rep = d.solve(None, u, tol=1e-10, opts=dgg.solve_opts(linear_tol=1e-4))
        assert rep.status == 0 and rep.relative_residual <= 1e-10
        uh = u.cpu().numpy().reshape(-1, N, N, N)
        r0 = -(mass * puncture.source(np.zeros_like(uh), alpha, beta))
        r = -(dg.apply(graph, uh) + mass * puncture.source(uh, alpha, beta))
        assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(r0)
        sols[precision] = (uh, rep)
    (u64, r64), (u32, r32) = sols["fp64"], sols["mixed"]
    assert r32.newton_steps == r64.newton_steps
    assert r32.iterations <= 1.5 * r64.iterations + 3
    assert rel(u32, u64) < 1e-10


def test_puncture_16x16x16_N6_per_subdomain_inverses():
    """The same puncture workload with the explicit inverse of each of the 4096 finest-level
    subdomains' linearized matrices (648 x 648 each, 6.9 GB in FP32), rebuilt at every Newton step:
    same Newton steps, the oracle's operator confirms the residual, and the solution agrees with
    the default subdomain solver's to 1e-10."""
    n, N = (16, 16, 16), 6
    grid = box(n, N, lower=(-20.0,) * 3, upper=(20.0,) * 3)
    graph = grid.graph()
    x, y, z = grid.coordinates()
    alpha, beta = puncture.alpha_beta(x, y, z, workloads.BINARY_PUNCTURES)
    mass = dg.mass_diag(graph)
    d = dgg.Domain((-20.0,) * 3, (20.0,) * 3, n, N, precision="mixed", overlap=2, problem="puncture",
                   punctures=workloads.BINARY_PUNCTURES)
    sols = {}
    for solver in ("gmres", "inverse"):
        u = torch.zeros(d.n_dof, dtype=torch.float64, device="cuda")
        rep = d.solve(None, u, tol=1e-10, opts=dgg.solve_opts(linear_tol=1e-4, subdomain_solver=solver))
        assert rep.status == 0 and rep.relative_residual <= 1e-10, solver
        sols[solver] = (u.cpu().numpy().reshape(-1, N, N, N), rep)
    uh, rep = sols["inverse"]
    r0 = -(mass * puncture.source(np.zeros_like(uh), alpha, beta))
    r = -(dg.apply(graph, uh) + mass * puncture.source(uh, alpha, beta))
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(r0)
    assert rep.newton_steps == sols["gmres"][1].newton_steps
    assert rel(uh, sols["gmres"][0]) < 1e-10



def test_more_subdomains_than_one_launch_takes():
    """41^3 = 68,921 elements at N = 2: the per-subdomain builds (curved column kernel, linearized
    inverses, batched Gauss-Jordan) run in chunks of at most 65,535 subdomains. A warped-mesh solve
    and a puncture solve with per-subdomain linearized inverses reach 1e-10; the oracle's operator
    confirms the curved residual, and the puncture solution equals the default subdomain solver's."""
    from oracle import curved

    n, N = (41, 41, 41), 2
    box_g = dg.BoxGrid((-1.0,) * 3, (1.0,) * 3, n, N, 1.5)
    warp = lambda X, Y, Z: (X + 0.1 * (1 - X**2) * Y, Y + 0.12 * (1 - Y**2) * Z * X, Z + 0.1 * (1 - Z**2) * (X + Y))
    g = curved.MappedGrid.from_mapping(box_g, warp)
    x, y, z = g.coordinates()
    f = workloads.gaussian_source(2)(x, y, z)
    d = dgg.Domain(n=n, N=N, precision="mixed", overlap=1, node_xyz=(x, y, z))
    b = d.rhs(torch.from_numpy(f.ravel()).cuda())
    u = torch.zeros_like(b)
    rep = d.solve(b, u, tol=1e-10, opts=dgg.solve_opts(max_iterations=400))
    assert rep.status == 0 and rep.relative_residual <= 1e-10
    gr = g.graph()
    res = dg.rhs(gr, f) - dg.apply(gr, u.cpu().numpy().reshape(-1, N, N, N))
    assert np.linalg.norm(res) <= 1.01e-10 * np.linalg.norm(b.cpu().numpy())
    d.close()

    dp = dgg.Domain((-20.0,) * 3, (20.0,) * 3, n, N, precision="mixed", overlap=1, problem="puncture",
                    punctures=workloads.BINARY_PUNCTURES)
    sols = {}
    for solver in ("gmres", "inverse"):
        up = torch.zeros(dp.n_dof, dtype=torch.float64, device="cuda")
        rp = dp.solve(None, up, tol=1e-10, opts=dgg.solve_opts(linear_tol=1e-4, subdomain_solver=solver,
                                                               max_iterations=400))
        assert rp.status == 0 and rp.relative_residual <= 1e-10, solver
        sols[solver] = up.cpu().numpy()
    assert rel(sols["inverse"], sols["gmres"]) < 1e-10
