"""GPU parity of the DG operator (Sec. II) and the multigrid transfers (Sec. III.C.2) against the
FP64 oracle, through the C ABI. FP64 tolerance 1e-12 relative (rounding of the ~12N-flop
contractions); FP32 tolerance 2e-5 relative (FP32 unit roundoff 6e-8 times the same depth and
the conditioning of the face terms)."""
import numpy as np
import pytest
import torch

import workloads
from gpu_util import box, rand, rel
from oracle import dg, mg

pytestmark = pytest.mark.gpu

dgg = pytest.importorskip("paper_2111_06767_gb300")

CASES = [((1, 1, 1), 2), ((2, 1, 1), 3), ((3, 2, 1), 4), ((2, 2, 2), 5), ((2, 3, 2), 6), ((1, 2, 3), 7),
         ((2, 2, 2), 8), ((2, 1, 2), 9), ((1, 1, 2), 10), ((5, 3, 4), 4)]


@pytest.mark.parametrize("n,N", CASES)
def test_apply_fp64_and_fp32_match_oracle(n, N):
    lower, upper = (-1.0, -0.5, 0.0), (1.0, 0.7, 2.5)
    d = dgg.Domain(lower, upper, n, N, penalty=1.5, mg_levels=1, overlap=1)
    grid = box(n, N, lower=lower, upper=upper)
    u = rand(10 + N, (grid.n_elements, N, N, N))
    ref = dg.apply(grid.graph(), u)
    out = d.apply(torch.from_numpy(u.ravel()).cuda()).cpu().numpy()
    assert rel(out, ref) < 1e-12
    out32 = d.apply_f32(torch.from_numpy(u.ravel()).float().cuda()).double().cpu().numpy()
    assert rel(out32, ref) < 2e-5


def test_apply_full_size_gaussian_config():
    """8^3 elements, N = 8 (262,144 points): the workload of the Gaussian-source benchmark."""
    n, N = (8, 8, 8), 8
    d = dgg.Domain(n=n, N=N, mg_levels=1, overlap=2)
    grid = box(n, N)
    u = rand(5, (grid.n_elements, N, N, N))
    ref = dg.apply(grid.graph(), u)
    out = d.apply(torch.from_numpy(u.ravel()).cuda()).cpu().numpy()
    assert rel(out, ref) < 1e-12


def test_apply_sampled_elements_at_roofline_size():
    """N = 4 on 64^3 elements (16.8M points): oracle on sampled elements with their face neighbours."""
    n, N = (64, 64, 64), 4
    d = dgg.Domain(n=n, N=N, mg_levels=1, overlap=1)
    grid = box(n, N)
    E = grid.n_elements
    u_dev = torch.empty(E * N**3, dtype=torch.float64, device="cuda").uniform_(-1, 1, generator=torch.Generator("cuda").manual_seed(3))
    out = d.apply(u_dev).view(E, N, N, N).cpu().numpy()
    u = u_dev.view(E, N, N, N).cpu().numpy()
    full = grid.graph()
    for e in [0, 1, 63, 64 * 64 - 1, 123456, E // 2 + 17, E - 1]:
        slots = [e] + [int(q) for q in full.nbr[e] if q >= 0]
        pos = {g: s for s, g in enumerate(slots)}
        pn = np.full((len(slots), 6), dg.ZERO)
        for s, g in enumerate(slots):
            for f in range(6):
                q = full.nbr[g, f]
                pn[s, f] = dg.EXTERNAL if q == dg.EXTERNAL else pos.get(int(q), dg.ZERO)
        patch = dg.ElementGraph(N, full.penalty, full.h[slots], pn, full.h_ext[slots])
        ref = dg.apply(patch, u[slots])[0]
        assert rel(out[e], ref) < 1e-12, e


@pytest.mark.parametrize("n,N", [((2, 2, 2), 3), ((4, 2, 6), 4), ((4, 4, 4), 6), ((2, 4, 3), 5)])
def test_transfers_match_oracle(n, N):
    d = dgg.Domain(n=n, N=N, mg_levels=2, overlap=1)
    fine = box(n, N)
    coarse = mg.hierarchy(fine, 2)[1]
    assert tuple(d.layout.level_n[1]) == coarse.n
    rf = rand(21, (fine.n_elements, N, N, N))
    uc = rand(22, (coarse.n_elements, N, N, N))
    ref_b = mg.restrict(fine, coarse, rf)
    out_b = d.restrict(0, torch.from_numpy(rf.ravel()).cuda()).cpu().numpy()
    assert rel(out_b, ref_b) < 1e-13
    base = rand(23, (fine.n_elements, N, N, N))
    ref_u = base + mg.prolongate(fine, coarse, uc)
    out_u = d.prolongate_add(0, torch.from_numpy(uc.ravel()).cuda(), torch.from_numpy(base.ravel()).cuda()).cpu().numpy()
    assert rel(out_u, ref_u) < 1e-13


def test_rhs_and_coordinates():
    n, N = (3, 2, 2), 5
    lower, upper = (-1.0, 0.0, 2.0), (2.0, 1.0, 3.0)
    d = dgg.Domain(lower, upper, n, N, mg_levels=1, overlap=1)
    grid = box(n, N, lower=lower, upper=upper)
    x, y, z = grid.coordinates()
    X, Y, Z = (t.cpu().numpy() for t in d.coordinates())
    assert max(np.abs(X - x.ravel()).max(), np.abs(Y - y.ravel()).max(), np.abs(Z - z.ravel()).max()) < 1e-14
    f = rand(4, x.shape)
    b = d.rhs(torch.from_numpy(f.ravel()).cuda()).cpu().numpy()
    assert rel(b, dg.rhs(grid.graph(), f)) < 1e-14


def test_krylov_dot_products_deterministic_and_accurate():
    """FGMRES inner products (Sec. III.B): FP64 two-pass reduction, equal to an exact-sum reference
    to rounding and bitwise reproducible."""
    import math

    d = dgg.Domain(n=(4, 4, 2), N=5, mg_levels=1, overlap=1)
    n = d.n_dof
    V = rand(61, (7, n))
    w = rand(62, (n,))
    Vt = torch.from_numpy(V).cuda()
    wt = torch.from_numpy(w).cuda()
    out1 = d.dot(Vt, wt).cpu().numpy()
    out2 = d.dot(Vt, wt).cpu().numpy()
    assert np.array_equal(out1, out2)
    exact = np.array([math.fsum(V[k] * w) for k in range(7)])
    assert np.abs(out1 - exact).max() <= 1e-13 * np.abs(V).sum(axis=1).max()


_PLANE_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[2]); sys.path.insert(0, sys.argv[2] + "/tests")
import workloads, paper_2111_06767_gb300 as dgg
from gpu_util import box, rand
out = {}
cases = [((3, 2, 1), ()), ((5, 3, 4), ()), ((33, 2, 1), (1, 4)), ((7, 5, 3), (0, 2, 5)), ((1, 1, 1), ())]
lower, upper = (-1.0, -0.5, 0.0), (1.0, 0.7, 2.5)
for N in [int(x) for x in sys.argv[3].split(",")]:
    for c, (n, neu) in enumerate(cases):
        d = dgg.Domain(lower, upper, n, N, mg_levels=1, overlap=1, neumann=neu)
        u = rand(300 + c, (n[0] * n[1] * n[2], N, N, N))
        out[f"apply{N}_{c}"] = d.apply_f32(torch.from_numpy(u.ravel()).float().cuda()).double().cpu().numpy()
    d = dgg.Domain(n=(4, 4, 2), N=N, mg_levels=2, overlap=2, precision="mixed", gemm="simt")
    out[f"vcycle{N}"] = d.vcycle(torch.from_numpy(rand(41, (32, N, N, N)).ravel()).cuda()).cpu().numpy()
    dp = dgg.Domain((-20.0,) * 3, (20.0,) * 3, (4, 3, 2), N, mg_levels=1, overlap=1, problem="puncture",
                    punctures=workloads.BINARY_PUNCTURES, precision="mixed")
    dp.set_linearization(torch.from_numpy(0.1 * rand(51, (24, N, N, N)).ravel()).cuda())
    out[f"lin{N}"] = dp.apply_f32(torch.from_numpy(rand(52, (24, N, N, N)).ravel()).float().cuda()).double().cpu().numpy()
np.savez(sys.argv[1], **out)
"""


@pytest.mark.parametrize("variant,orders", [("4", (4,)), ("7", (4,)), ("1", (4, 7)),
                                            ("5", (4, 5, 6, 7, 8, 9, 10)), ("6", (4, 5, 6, 7, 8, 9, 10))])
def test_pinned_fp32_apply_kernels_match_oracle(tmp_path, variant, orders):
    """Each plain FP32 apply kernel pinned for every apply of the process (DG_APPLY_VARIANT: 4 the
    slice-per-thread kernel at N = 4, 7 the element-per-thread kernel at N = 4, 5 and 6 the two launch
    shapes of the block-of-lines kernel, 1 a line-kernel shape for comparison): the operator against the oracle on ragged element counts
    (66 elements: no launch shape divides it), Neumann faces and a single element, the V-cycle's
    residual (b - A u) and the linearized puncture operator (+ diag u), at every order offered."""
    import os
    import subprocess
    import sys

    from oracle import puncture, solve

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "plane.py"
    script.write_text(_PLANE_SCRIPT)
    f = tmp_path / "out.npz"
    subprocess.run([sys.executable, str(script), str(f), root, ",".join(str(N) for N in orders)],
                   env=dict(os.environ, DG_APPLY_VARIANT=variant), check=True, timeout=900)
    got = np.load(f)
    cases = [((3, 2, 1), ()), ((5, 3, 4), ()), ((33, 2, 1), (1, 4)), ((7, 5, 3), (0, 2, 5)), ((1, 1, 1), ())]
    lower, upper = (-1.0, -0.5, 0.0), (1.0, 0.7, 2.5)
    for N in orders:
        for c, (n, neu) in enumerate(cases):
            grid = dg.BoxGrid(lower, upper, n, N, 1.5, tuple(fc in neu for fc in range(6)))
            u = rand(300 + c, (grid.n_elements, N, N, N))
            assert rel(got[f"apply{N}_{c}"], dg.apply(grid.graph(), u)) < 2e-5, (variant, N, n)
        pr = solve.Problem(box((4, 4, 2), N), mg_levels=2)
        assert rel(got[f"vcycle{N}"], pr.vcycle(rand(41, (32, N, N, N)))) < 1e-4, (variant, N)
        gp = box((4, 3, 2), N, lower=(-20.0,) * 3, upper=(20.0,) * 3)
        pp = solve.PunctureProblem(gp, workloads.BINARY_PUNCTURES, mg_levels=1)
        ul, v = 0.1 * rand(51, (24, N, N, N)), rand(52, (24, N, N, N))
        ref = pp.apply(v) + pp.mass * puncture.source_deriv(ul, pp.alpha, pp.beta) * v
        assert rel(got[f"lin{N}"], ref) < 2e-5, (variant, N)
