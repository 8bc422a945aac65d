"""GPU parity of the finest-level Schwarz smoother of a linearized puncture problem (Sec. III.E)
against the oracle, for both subdomain solvers: GMRES on A_S + D_S preconditioned by the Poisson
class inverse (the Laplacian approximation), and the explicit inverse of every subdomain's own
A_S + D_S rebuilt at each linearization. FP64 agreement 1e-10 relative (dense LU in the oracle
against Gauss-Jordan inverses here); MIXED 1e-4 with FP32 subdomain GEMMs and 3e-3 with TF32 ones
(the GMRES path's Poisson-inverse products; the per-subdomain inverses are applied in FP32)."""
import numpy as np
import pytest
import torch

import workloads
from gpu_util import box, rand, rel
from oracle import dg, puncture, schwarz, solve

pytestmark = pytest.mark.gpu

dgg = pytest.importorskip("paper_2111_06767_gb300")

P = workloads.BINARY_PUNCTURES


def _setup(n, N, ov, half_width, precision, seed=61, gemm="default"):
    lower, upper = (-half_width,) * 3, (half_width,) * 3
    d = dgg.Domain(lower, upper, n, N, precision=precision, mg_levels=1, overlap=ov, problem="puncture", punctures=P,
                   gemm=gemm)
    grid = box(n, N, lower=lower, upper=upper)
    pr = solve.PunctureProblem(grid, P, mg_levels=1, overlap=ov)
    u = 0.1 * rand(seed, (grid.n_elements, N, N, N))
    D = pr.mass * puncture.source_deriv(u, pr.alpha, pr.beta)
    return d, grid, pr, u, D


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()


@pytest.mark.parametrize("n,N,ov,hw", [((3, 2, 2), 4, 2, 4.0), ((2, 2, 2), 5, 3, 20.0), ((1, 1, 1), 6, 2, 4.0),
                                       ((4, 3, 2), 3, 1, 8.0)])
@pytest.mark.parametrize("solver", ["gmres", "inverse"])
def test_linearized_smoother_matches_oracle(n, N, ov, hw, solver):
    for precision, gemm, tol in (("fp64", "default", 1e-10), ("mixed", "simt", 1e-4), ("mixed", "tf32", 3e-3)):
        d, grid, pr, u, D = _setup(n, N, ov, hw, precision, gemm=gemm)
        lv = pr.schwarz[0]
        lin = lambda x: dg.apply(pr.graphs[0], x) + D * x
        sub = (schwarz.gmres_subdomain_solver(lv, D, 3) if solver == "gmres"
               else schwarz.inverse_subdomain_solver(lv, D))
        b = rand(62, (grid.n_elements, N, N, N))
        u0 = rand(63, (grid.n_elements, N, N, N))
        ref = lv.smooth(b, u0, 2, lin, sub)
        d.set_subdomain_solver(solver, 3)
        d.set_linearization(_dev(u))
        out = d.schwarz_smooth(0, _dev(b), _dev(u0), 2).cpu().numpy()
        assert rel(out, ref) < tol, (precision, gemm, solver)


def test_inverses_follow_the_linearization_and_the_call_order():
    """Building the inverses when the solver is chosen after the linearization gives the same smoother;
    a new linearization rebuilds them (the result changes with u and matches the oracle again)."""
    n, N, ov = (3, 2, 2), 4, 2
    d, grid, pr, u, D = _setup(n, N, ov, 4.0, "fp64")
    lv = pr.schwarz[0]
    b = rand(64, (grid.n_elements, N, N, N))
    u0 = np.zeros_like(b)
    d.set_subdomain_solver("inverse")
    d.set_linearization(_dev(u))
    first = d.schwarz_smooth(0, _dev(b), _dev(u0), 1).cpu().numpy()
    d2 = dgg.Domain((-4.0,) * 3, (4.0,) * 3, n, N, mg_levels=1, overlap=ov, problem="puncture", punctures=P)
    d2.set_linearization(_dev(u))
    d2.set_subdomain_solver("inverse")
    assert rel(d2.schwarz_smooth(0, _dev(b), _dev(u0), 1).cpu().numpy(), first) < 1e-13
    u2 = 2.0 * u
    d.set_linearization(_dev(u2))
    D2 = pr.mass * puncture.source_deriv(u2, pr.alpha, pr.beta)
    lin2 = lambda x: dg.apply(pr.graphs[0], x) + D2 * x
    ref2 = lv.smooth(b, u0, 1, lin2, schwarz.inverse_subdomain_solver(lv, D2))
    out2 = d.schwarz_smooth(0, _dev(b), _dev(u0), 1).cpu().numpy()
    assert rel(out2, ref2) < 1e-10 and rel(out2, first) > 1e-6


def test_subdomain_solver_arguments_are_checked():
    d, *_ = _setup((2, 2, 2), 3, 1, 4.0, "fp64")
    for args in (("inverse", -1), ("gmres", 17)):
        with pytest.raises(dgg.NativeError):
            d.set_subdomain_solver(*args)
    assert dgg.lib().dg_set_subdomain_solver(d.handle, 2, 3, None) != 0
    pois = dgg.Domain(n=(2, 2, 2), N=3, mg_levels=1, overlap=1)
    with pytest.raises(dgg.NativeError):
        pois.set_subdomain_solver("inverse")
    o = dgg.solve_opts()
    o.subdomain_solver = 2
    u = torch.zeros(d.n_dof, dtype=torch.float64, device="cuda")
    with pytest.raises(dgg.NativeError):
        d.solve(None, u, tol=1e-10, opts=o)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_newton_with_per_subdomain_inverses_matches_oracle(precision):
    """Binary punctures on [-20,20]^3, 4^3 elements, N = 5: Newton-Krylov with per-subdomain
    linearized inverses reaches the oracle's solution; FP64 takes as many Krylov iterations as the
    oracle with the same subdomain solver (within one per Newton step)."""
    n, N = (4, 4, 4), 5
    grid = box(n, N, lower=(-20.0,) * 3, upper=(20.0,) * 3)
    pr = solve.PunctureProblem(grid, P)
    u_ref, rep_ref = pr.solve(tol=1e-10, linear_tol=1e-4, subdomain_solver="inverse")
    assert rep_ref["converged"]
    d = dgg.Domain((-20.0,) * 3, (20.0,) * 3, n, N, precision=precision, overlap=2, problem="puncture", punctures=P)
    u = torch.zeros(d.n_dof, dtype=torch.float64, device="cuda")
    rep = d.solve(None, u, tol=1e-10, opts=dgg.solve_opts(linear_tol=1e-4, subdomain_solver="inverse"))
    assert rep.relative_residual <= 1e-10
    assert np.linalg.norm(pr.residual(u.cpu().numpy().reshape(u_ref.shape))) <= 1.01e-10 * rep.initial_residual
    u_tight, _ = pr.solve(tol=1e-13, linear_tol=1e-8)
    assert rel(u.cpu().numpy(), u_tight) < 1e-10
    if precision == "fp64":
        its = sum(info["iterations"] for info in rep_ref["linear_iterations"])
        assert rep.newton_steps == rep_ref["steps"]
        assert abs(rep.iterations - its) <= rep.newton_steps


def test_per_subdomain_inverses_that_do_not_fit_report_oom():
    """36^3 elements, N = 6, overlap 5 (n_S = 1296): the per-subdomain linearized inverses would need
    46,656 x 1296^2 x 4 B = 313 GB, more than the device holds. The linearization reports
    DG_ERR_OOM (an allocation that fails, no fault), and the domain keeps working with the default
    subdomain solver."""
    d = dgg.Domain((-20.0,) * 3, (20.0,) * 3, (36, 36, 36), 6, precision="mixed", mg_levels=1, overlap=5,
                   problem="puncture", punctures=P)
    u = torch.zeros(d.n_dof, dtype=torch.float64, device="cuda")
    d.set_subdomain_solver("inverse")
    with pytest.raises(dgg.NativeError) as info:
        d.set_linearization(u)
    assert info.value.status == -2  # DG_ERR_OOM
    d.set_subdomain_solver("gmres", 3)
    d.set_linearization(u)
    b = torch.ones_like(u)
    out = d.schwarz_smooth(0, b, torch.zeros_like(u), 1)
    assert torch.isfinite(out).all() and float(out.abs().max()) > 0
