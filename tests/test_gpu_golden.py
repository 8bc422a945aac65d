"""Solution parity: GPU solves must reach the oracle's solution to 1e-10 relative L2.

The reference solutions of the benchmark workloads are written by
tests/golden/make_reference_solutions.py, which calls only the FP64 CPU oracle (multigrid-Schwarz
FGMRES to a 1e-14 estimate for the Gaussian source, Newton to a 1e-13 nonlinear residual for the
punctures). A residual bounds the relative error only up to the condition number of A: on the
Gaussian workload a 1e-10 oracle solve is 3.6e-12 from u*, so the benchmark's 1e-10 tolerance meets
the parity with margin; where a small problem's error at a 1e-10 residual exceeds 1e-10 (measured
below), its solve is tightened until the parity holds. The small sine workload (2^3 elements,
N = 6) is compared with the oracle's dense direct solve.
"""
import json
import os

import numpy as np
import pytest
import torch

import workloads
from gpu_util import box, rel
from oracle import dg, solve

pytestmark = pytest.mark.gpu

dgg = pytest.importorskip("paper_2111_06767_gb300")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    path = os.path.join(GOLDEN, name + "_u.npy")
    with open(os.path.join(GOLDEN, name + "_u.json")) as fh:
        meta = json.load(fh)
    return np.load(path), meta


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("krylov", ["fgmres", "fcg"])
def test_sine_2x2x2_N6_matches_dense_direct_solve(precision, krylov):
    """A 1e-10 residual leaves this problem up to 1.9e-10 (FGMRES, depending on the tuned launch
    shapes) or 3.6e-10 (flexible CG with the FP32 V-cycle) from the direct solution (measured), so
    both solve to 1e-11, the tolerance at which the parity holds."""
    tol = 1e-11
    cfg = workloads.SINE_2x2x2
    grid = box(cfg.n, cfg.N, cfg.penalty)
    x, y, z = grid.coordinates()
    f = workloads.sine_source_3d(x, y, z)
    pr = solve.Problem(grid, mg_levels=cfg.mg_levels, overlap=cfg.overlap)
    ud = np.linalg.solve(dg.assemble(pr.graphs[0]), dg.rhs(pr.graphs[0], f).ravel())
    d = dgg.Domain(n=cfg.n, N=cfg.N, penalty=cfg.penalty, precision=precision, mg_levels=cfg.mg_levels,
                   overlap=cfg.overlap)
    b = d.rhs(torch.from_numpy(f.ravel()).cuda())
    u = torch.zeros_like(b)
    rep = d.solve(b, u, tol=tol, opts=dgg.solve_opts(krylov=krylov))
    assert rep.status == 0 and rep.relative_residual <= tol
    assert rel(u.cpu().numpy(), ud) <= 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gauss16_8x8x8_N8_matches_oracle_solution(precision):
    """The headline workload, in the configuration bench.py times (3-level V-cycle, overlap 2)."""
    cfg = workloads.GAUSS_8x8x8
    u_ref, meta = _golden(cfg.name)
    assert meta["true_relative_residual"] < 1e-12 and u_ref.size == cfg.n_dof
    grid = box(cfg.n, cfg.N, cfg.penalty)
    x, y, z = grid.coordinates()
    f = workloads.gaussian_source(cfg.seed)(x, y, z)
    d = dgg.Domain(n=cfg.n, N=cfg.N, penalty=cfg.penalty, precision=precision, mg_levels=cfg.mg_levels,
                   overlap=cfg.overlap)
    b = d.rhs(torch.from_numpy(f.ravel()).cuda())
    for krylov in ("fgmres", "fcg"):
        for _ in range(2):  # the first solve runs the V-cycle uncaptured, the second replays its graph
            u = torch.zeros_like(b)
            rep = d.solve(b, u, tol=1e-10, opts=dgg.solve_opts(krylov=krylov))
            assert rep.status == 0 and rep.relative_residual <= 1e-10
            assert rel(u.cpu().numpy(), u_ref) <= 1e-10, (krylov, rel(u.cpu().numpy(), u_ref))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_puncture_16cubed_N6_matches_oracle_solution(precision):
    """The binary-puncture workload: Newton-Krylov to a 1e-10 nonlinear residual (linearized solves
    to 1e-4), FP32 or FP64 Schwarz smoother under FP64 FGMRES."""
    cfg = workloads.PUNCTURE_16
    u_ref, meta = _golden(cfg.name)
    assert meta["true_relative_residual"] < 1e-12 and u_ref.size == cfg.n_dof
    d = dgg.Domain(cfg.lower, cfg.upper, cfg.n, cfg.N, penalty=cfg.penalty, precision=precision,
                   overlap=cfg.overlap, problem="puncture", punctures=workloads.BINARY_PUNCTURES)
    u = torch.zeros(d.n_dof, dtype=torch.float64, device="cuda")
    rep = d.solve(None, u, tol=1e-10, opts=dgg.solve_opts(linear_tol=1e-4))
    assert rep.status == 0 and rep.relative_residual <= 1e-10
    assert rel(u.cpu().numpy(), u_ref) <= 1e-10, rel(u.cpu().numpy(), u_ref)
