"""Run one operation of the solver a few times on a seeded input, for kernel profiling.

    python -m paper_2111_06767_gb300.profile_case --op smooth --n 8 --N 8 --reps 3
    python -m paper_2111_06767_gb300.profile_case --op apply --n 80 --N 4 --precision mixed --reps 3
    python -m paper_2111_06767_gb300.profile_case --op solve --n 8 --N 8 --levels 3 --reps 2

--op smooth: Schwarz smoothing steps on the finest level (residual apply, gather, subdomain GEMM,
scatter); --op apply: the DG operator alone (FP32 for --precision mixed, FP64 otherwise);
--op vcycle: full V-cycles; --warp: curved elements (a smooth warp of the box's nodes); --op solve: FGMRES solves to 1e-10 of the 16-Gaussian source (one
untimed solve first, then --reps solves inside the NVTX range "timed", a 256 MB buffer written
before each so that L2 starts cold as in bench.py). The domain is [-1,1]^3 with n^3 elements and
N points per dimension.
"""
from __future__ import annotations

import argparse

import torch

import paper_2111_06767_gb300 as dgg


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", choices=["smooth", "apply", "vcycle", "solve"], default="smooth")
    ap.add_argument("--n", type=int, default=8)
    ap.add_argument("--N", type=int, default=8)
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--gemm", choices=["default", "simt", "tf32"], default="default")
    ap.add_argument("--levels", type=int, default=1)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--warp", action="store_true", help="curved elements: a smooth warp of the box's nodes")
    a = ap.parse_args()
    xyz = None
    if a.warp:
        X, Y, Z = dgg.host_coordinates(dgg.make_desc((-1.0,) * 3, (1.0,) * 3, (a.n,) * 3, a.N))
        xyz = (X + 0.1 * (1 - X**2) * Y, Y + 0.12 * (1 - Y**2) * Z * X, Z + 0.1 * (1 - Z**2) * (X + Y))
    d = dgg.Domain(n=(a.n,) * 3, N=a.N, precision=a.precision, mg_levels=a.levels, overlap=2, gemm=a.gemm,
                   node_xyz=xyz)
    g = torch.Generator(device="cuda").manual_seed(7)
    dt = torch.float32 if (a.op == "apply" and a.precision == "mixed") else torch.float64
    x = torch.empty(d.n_dof, dtype=dt, device="cuda").uniform_(-1, 1, generator=g)
    y = torch.zeros_like(x)
    if a.op == "solve":
        import workloads

        X, Y, Z = d.coordinates()
        b = d.rhs(workloads.gaussian_source(2)(X, Y, Z).contiguous())
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        d.solve(b, y, 1e-10)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        for i in range(a.reps):
            flush.fill_(float(i))
            y.zero_()
            d.solve(b, y, 1e-10)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(f"solve done: n={a.n}^3 N={a.N} dof={d.n_dof}")
        return
    for _ in range(a.reps):
        if a.op == "apply":
            if dt == torch.float32:
                d.apply_f32(x, 0, y)
            else:
                d.apply(x, y)
        elif a.op == "smooth":
            d.schwarz_smooth(0, x, y, 1)
        else:
            d.vcycle(x, y)
    torch.cuda.synchronize()
    print(f"{a.op} done: n={a.n}^3 N={a.N} dof={d.n_dof}")


if __name__ == "__main__":
    main()
