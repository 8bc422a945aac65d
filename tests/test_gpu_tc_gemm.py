"""The subdomain-inverse GEMM on tcgen05 tensor cores (TF32 inputs, FP32 accumulate) against the
FP32 CUDA-core GEMM, and solves that use it. TF32 keeps 10 mantissa bits of each input, so one
smoothing step agrees with the FP32 path to ~1e-3 relative; FGMRES absorbs the difference and the
solution still meets the 1e-10 residual."""
import numpy as np
import pytest
import torch

import workloads
from gpu_util import box, rand, rel

pytestmark = pytest.mark.gpu

dgg = pytest.importorskip("paper_2111_06767_gb300")


@pytest.mark.parametrize("n,N,ov", [((2, 2, 2), 4, 2), ((4, 3, 2), 5, 2), ((8, 8, 8), 8, 2), ((3, 3, 3), 6, 1)])
def test_tensor_core_smoothing_matches_simt(n, N, ov):
    grid = box(n, N)
    b = torch.from_numpy(rand(81, (grid.n_elements * N**3,))).cuda()
    u0 = torch.from_numpy(rand(82, (grid.n_elements * N**3,))).cuda()
    outs = {}
    for gemm in ("simt", "tf32"):
        d = dgg.Domain(n=n, N=N, mg_levels=1, overlap=ov, precision="mixed", gemm=gemm)
        outs[gemm] = d.schwarz_smooth(0, b, u0.clone(), 1).cpu().numpy()
    du_s = outs["simt"] - u0.cpu().numpy()
    du_t = outs["tf32"] - u0.cpu().numpy()
    assert rel(du_t, du_s) < 3e-3


def test_tensor_core_solve_meets_tolerance():
    n, N = (8, 8, 8), 8
    grid = box(n, N)
    x, y, z = grid.coordinates()
    f = torch.from_numpy(workloads.gaussian_source(2)(x, y, z).ravel()).cuda()
    sols = {}
    for prec, gemm in (("fp64", "default"), ("mixed", "tf32")):
        d = dgg.Domain(n=n, N=N, mg_levels=3, overlap=2, precision=prec, gemm=gemm)
        b = d.rhs(f)
        u = torch.zeros_like(b)
        rep = d.solve(b, u, tol=1e-10)
        assert rep.relative_residual <= 1e-10
        sols[prec] = (u.cpu().numpy(), rep.iterations)
    assert rel(sols["mixed"][0], sols["fp64"][0]) < 1e-10
    assert sols["mixed"][1] <= sols["fp64"][1] + 2


_SOLVE_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[2]); sys.path.insert(0, sys.argv[2] + "/tests")
import workloads, paper_2111_06767_gb300 as dgg
from gpu_util import box
n, N = (6, 6, 6), 6
x, y, z = box(n, N).coordinates()
d = dgg.Domain(n=n, N=N, precision="mixed", mg_levels=2, overlap=2)
b = d.rhs(torch.from_numpy(workloads.gaussian_source(2)(x, y, z).ravel()).cuda())
u = torch.zeros_like(b)
rep = d.solve(b, u, tol=1e-10)
assert rep.relative_residual <= 1e-10
np.save(sys.argv[1], u.cpu().numpy())
"""


def test_autotuned_launch_shapes_match_fixed_ones(tmp_path):
    """The launch shapes of the DG apply and the split-K factor of the tensor-core GEMM are timed
    and chosen per process; with DG_AUTOTUNE=0 the grid-size heuristics are used instead. Both
    must reach the same solution (the split changes only the FP32 summation order)."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "solve.py"
    script.write_text(_SOLVE_SCRIPT)
    out = {}
    for tune in ("1", "0"):
        f = tmp_path / f"u{tune}.npy"
        env = dict(os.environ, DG_AUTOTUNE=tune)
        subprocess.run([sys.executable, str(script), str(f), root], env=env, check=True, timeout=600)
        out[tune] = np.load(f)
    assert rel(out["1"], out["0"]) < 1e-10


@pytest.mark.parametrize("n", [(4, 4, 4), (8, 8, 8)])
def test_every_gemm_split_matches_simt(monkeypatch, n):
    """Each K split of the tensor-core GEMM (1, 2, 4 or 8 CTAs of a cluster, partial tiles summed
    through distributed shared memory) at every tile width (64 columns; 256 columns: 16 + split; 128
    columns: 32 + split), pinned with DG_GEMM_SPLIT, gives the CUDA-core FP32 smoothing step to TF32
    accuracy. N = 8 offers every split (40 K chunks of 32); 8^3 elements give classes of up to 96
    subdomains in one 128- or 256-wide tile, 4^3 classes of at most 24."""
    N, ov = 8, 2
    grid = box(n, N)
    b = torch.from_numpy(rand(83, (grid.n_elements * N**3,))).cuda()
    u0 = torch.from_numpy(rand(84, (grid.n_elements * N**3,))).cuda()
    ref = dgg.Domain(n=n, N=N, mg_levels=1, overlap=ov, precision="mixed", gemm="simt")
    du_s = ref.schwarz_smooth(0, b, u0.clone(), 1).cpu().numpy() - u0.cpu().numpy()
    for split in (1, 2, 4, 8, 16, 17, 18, 20, 24, 32, 33, 34, 36, 40):
        monkeypatch.setenv("DG_GEMM_SPLIT", str(split))
        d = dgg.Domain(n=n, N=N, mg_levels=1, overlap=ov, precision="mixed", gemm="tf32")
        du_t = d.schwarz_smooth(0, b, u0.clone(), 1).cpu().numpy() - u0.cpu().numpy()
        assert rel(du_t, du_s) < 3e-3, split


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_every_cuda_core_gemm_split_matches_oracle(monkeypatch, precision):
    """The CUDA-core class GEMM (FP64 domains, and MIXED with gemm="simt") with its K range split over
    1, 2, 4 or 8 CTAs of a cluster (partial tiles summed in rank order through distributed shared
    memory), pinned with DG_GEMM_SPLIT: one smoothing step equals the oracle's Schwarz step (FP64 to
    1e-10, FP32 to 1e-4)."""
    from oracle import schwarz

    n, N, ov = (4, 4, 4), 6, 2
    grid = box(n, N)
    b = rand(85, (grid.n_elements, N, N, N))
    u0 = rand(86, (grid.n_elements, N, N, N))
    ref = schwarz.SchwarzLevel(grid, ov).smooth(b, u0, 1).ravel()
    tol = 1e-10 if precision == "fp64" else 1e-4
    for split in (1, 2, 4, 8):
        monkeypatch.setenv("DG_GEMM_SPLIT", str(split))
        d = dgg.Domain(n=n, N=N, mg_levels=1, overlap=ov, precision=precision, gemm="simt")
        bt, ut = torch.from_numpy(b.ravel()).cuda(), torch.from_numpy(u0.ravel()).cuda()
        got = d.schwarz_smooth(0, bt, ut, 1).cpu().numpy()
        assert rel(got - u0.ravel(), ref - u0.ravel()) < tol, split
