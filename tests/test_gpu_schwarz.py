"""GPU parity of the Schwarz smoother (Sec. III.D) and the V-cycle (Sec. III.C.3) against the
oracle. The oracle solves each subdomain problem with a dense LU solve; the GPU applies explicit
inverses built column by column and inverted by Gauss-Jordan: FP64 agreement to ~kappa(A_S) eps,
asserted at 1e-10 relative. The MIXED smoother is held to 1e-4 relative with the FP32 CUDA-core
GEMM and to 3e-3 with the TF32 tensor-core GEMM (10 mantissa bits per input)."""
import numpy as np
import pytest
import torch

from gpu_util import box, rand, rel
from oracle import dg, mg, schwarz, solve

pytestmark = pytest.mark.gpu

dgg = pytest.importorskip("paper_2111_06767_gb300")


@pytest.mark.parametrize("n,N,ov", [((1, 1, 1), 3, 1), ((2, 2, 2), 4, 2), ((3, 2, 1), 5, 2), ((3, 3, 3), 4, 3),
                                    ((4, 3, 2), 6, 2), ((2, 2, 3), 3, 2)])
def test_schwarz_smooth_matches_oracle(n, N, ov):
    d = dgg.Domain(n=n, N=N, mg_levels=1, overlap=ov)
    grid = box(n, N)
    lv = schwarz.SchwarzLevel(grid, ov)
    b = rand(31, (grid.n_elements, N, N, N))
    u0 = rand(32, (grid.n_elements, N, N, N))
    ref = lv.smooth(b, u0, 2)
    out = d.schwarz_smooth(0, torch.from_numpy(b.ravel()).cuda(), torch.from_numpy(u0.ravel()).cuda(), 2).cpu().numpy()
    assert rel(out, ref) < 1e-10
    for gemm, tol in (("simt", 1e-4), ("tf32", 3e-3)):
        dm = dgg.Domain(n=n, N=N, mg_levels=1, overlap=ov, precision="mixed", gemm=gemm)
        out32 = dm.schwarz_smooth(0, torch.from_numpy(b.ravel()).cuda(), torch.from_numpy(u0.ravel()).cuda(),
                                  2).cpu().numpy()
        assert rel(out32, ref) < tol, gemm


def test_subdomain_class_count():
    """Per dimension an element is at the boundary, next to it, or inside (5 positions on 8 elements);
    up to reflections and exchanges of the cube's axes that leaves 10 classes on 8^3 elements, 4 on
    4^3 and 1 on 2^3; an anisotropic box keeps the unequal axis apart."""
    d = dgg.Domain(n=(8, 8, 8), N=4, mg_levels=3, overlap=2)
    assert list(d.layout.n_classes)[:3] == [10, 4, 1]
    assert d.layout.subdomain_size == 4**3 + 12 * 4**2
    d2 = dgg.Domain((0.0,) * 3, (1.0, 1.0, 2.0), (4, 4, 4), N=3, mg_levels=1, overlap=1)
    assert d2.layout.n_classes[0] == 3 * 2  # per axis {0,3} or {1,2}; x and y interchangeable, z apart


@pytest.mark.parametrize("n,N,levels", [((2, 2, 2), 4, 0), ((4, 4, 2), 3, 0), ((4, 4, 4), 4, 2)])
def test_vcycle_matches_oracle(n, N, levels):
    d = dgg.Domain(n=n, N=N, mg_levels=levels, overlap=2)
    grid = box(n, N)
    pr = solve.Problem(grid, mg_levels=levels)
    assert d.mg_levels == len(pr.levels)
    r = rand(41, (grid.n_elements, N, N, N))
    ref = pr.vcycle(r)
    out = d.vcycle(torch.from_numpy(r.ravel()).cuda()).cpu().numpy()
    assert rel(out, ref) < 1e-10
    for gemm, tol in (("simt", 1e-4), ("tf32", 3e-3)):
        dm = dgg.Domain(n=n, N=N, mg_levels=levels, overlap=2, precision="mixed", gemm=gemm)
        for _ in range(3):  # uncaptured, captured, replayed
            out32 = dm.vcycle(torch.from_numpy(r.ravel()).cuda()).cpu().numpy()
            assert rel(out32, ref) < tol, gemm
    for _ in range(2):
        assert rel(d.vcycle(torch.from_numpy(r.ravel()).cuda()).cpu().numpy(), ref) < 1e-10


@pytest.mark.parametrize("n,N,levels", [((4, 4, 4), 6, 2), ((2, 2, 2), 8, 1), ((3, 4, 2), 5, 1)])
def test_fused_coarse_smoother_matches_step_kernels(n, N, levels, monkeypatch):
    """With DG_COARSE_FUSED=1, coarse levels (at most 64 elements) of a MIXED domain are smoothed by
    one cooperative launch per smoothing call (residual, subdomain solves and scatter of every step,
    separated by grid barriers). It must agree with the per-step kernels (the default) to FP32
    rounding, for the V-cycle (first step a gather, u = 0), captured and replayed, and for
    smoothing with u != 0."""
    grid = box(n, N)
    r = torch.from_numpy(rand(91, (grid.n_elements * N**3,))).cuda()
    u0 = torch.from_numpy(rand(92, (grid.n_elements * N**3,))).cuda()
    out = {}
    for fused in ("1", "0"):
        monkeypatch.setenv("DG_COARSE_FUSED", fused)
        d = dgg.Domain(n=n, N=N, mg_levels=levels, overlap=2, precision="mixed", gemm="simt")
        vs = [d.vcycle(r).cpu().numpy() for _ in range(3)]  # uncaptured, captured, replayed
        sm = d.schwarz_smooth(0, r, u0.clone(), 3).cpu().numpy() - u0.cpu().numpy()
        out[fused] = (vs, sm)
    (v1, s1), (v0, s0) = out["1"], out["0"]
    assert np.array_equal(v1[1], v1[2])
    for a, b in zip(v1, v0):
        assert rel(a, b) < 1e-5
    assert rel(s1, s0) < 1e-5
