"""GPU parity of the puncture source terms, the nonlinear residual and linearization (Sec. III.A,
Eq. linearized) and the Newton-Krylov solve against the oracle."""
import numpy as np
import pytest
import torch

import workloads
from gpu_util import box, rand, rel
from oracle import dg, newton, puncture, solve

pytestmark = pytest.mark.gpu

dgg = pytest.importorskip("paper_2111_06767_gb300")

P = workloads.BINARY_PUNCTURES
BOX = dict(lower=(-20.0,) * 3, upper=(20.0,) * 3)


def _dom(n, N, precision="fp64", punctures=P, levels=0):
    return dgg.Domain(BOX["lower"], BOX["upper"], n, N, precision=precision, mg_levels=levels, overlap=2,
                      problem="puncture", punctures=punctures)


def test_puncture_fields_residual_and_linearization():
    n, N = (4, 4, 4), 5
    d = _dom(n, N)
    grid = box(n, N, **BOX)
    pr = solve.PunctureProblem(grid, P)
    a, b = (t.cpu().numpy() for t in d.puncture_fields())
    assert rel(a, pr.alpha) < 1e-13 and rel(b, pr.beta) < 1e-12
    u = 0.1 * rand(51, (grid.n_elements, N, N, N))
    ut = torch.from_numpy(u.ravel()).cuda()
    r = d.nonlinear_residual(ut).cpu().numpy()
    assert rel(r, pr.residual(u)) < 1e-12
    d.set_linearization(ut)
    v = rand(52, (grid.n_elements, N, N, N))
    lin = d.apply(torch.from_numpy(v.ravel()).cuda()).cpu().numpy()
    D = pr.mass * puncture.source_deriv(u, pr.alpha, pr.beta)
    assert rel(lin, pr.apply(v) + D * v) < 1e-12
    d.set_linearization(None)
    plain = d.apply(torch.from_numpy(v.ravel()).cuda()).cpu().numpy()
    assert rel(plain, pr.apply(v)) < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_newton_solution_matches_oracle(precision):
    n, N = (4, 4, 4), 5
    grid = box(n, N, **BOX)
    pr = solve.PunctureProblem(grid, P)
    u_ref, rep_ref = pr.solve(tol=1e-12, linear_tol=1e-6)
    assert rep_ref["converged"]
    d = _dom(n, N, precision)
    u = torch.zeros(d.n_dof, dtype=torch.float64, device="cuda")
    rep = d.solve(None, u, tol=1e-10, opts=dgg.solve_opts(linear_tol=1e-4))
    assert rep.relative_residual <= 1e-10 and rep.newton_steps >= 2
    # confirm the residual with the oracle's operator, and the solution against the oracle's
    assert np.linalg.norm(pr.residual(u.cpu().numpy().reshape(u_ref.shape))) <= 1.01e-10 * rep.initial_residual
    assert rel(u.cpu().numpy(), u_ref) < 1e-10


def test_zero_momentum_needs_no_newton_step():
    still = tuple(workloads.Puncture(p.position, p.mass, (0.0, 0.0, 0.0)) for p in P)
    d = _dom((2, 2, 2), 4, punctures=still)
    u = torch.zeros(d.n_dof, dtype=torch.float64, device="cuda")
    rep = d.solve(None, u, tol=1e-10)
    assert rep.newton_steps == 0 and float(u.abs().max()) == 0.0


@pytest.mark.parametrize("n", [8, 12])
def test_mixed_newton_tracks_fp64_on_larger_grids(n):
    """On grids where the linearization term is tiny next to the Laplacian (far from the punctures
    the FP32 Arnoldi step of the subdomain GMRES reduces to cancellation noise), the mixed solver
    must still converge like the FP64 one: same Newton steps, a linear iteration count close to
    FP64's, and the same solution to 1e-10."""
    N = 6
    res = {}
    for precision in ("fp64", "mixed"):
        d = _dom((n,) * 3, N, precision)
        u = torch.zeros(d.n_dof, dtype=torch.float64, device="cuda")
        rep = d.solve(None, u, tol=1e-10, opts=dgg.solve_opts(linear_tol=1e-4, max_iterations=100))
        assert rep.relative_residual <= 1e-10
        res[precision] = (rep, u.cpu().numpy())
    (r64, u64), (r32, u32) = res["fp64"], res["mixed"]
    assert r32.newton_steps == r64.newton_steps
    assert r32.iterations <= 1.5 * r64.iterations + 3
    assert rel(u32, u64) < 1e-10
