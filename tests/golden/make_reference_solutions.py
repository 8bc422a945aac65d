"""Write the oracle's converged solutions of the benchmark problems to tests/golden/.

Calls only the FP64 CPU oracle (oracle/) and the seeded input generators (workloads.py); nothing
here touches the CUDA library. The GPU solution-parity tests compare against these files.

  python tests/golden/make_reference_solutions.py gauss     # 8^3 elements, N = 8 (about 10 min)
  python tests/golden/make_reference_solutions.py puncture  # 16^3 elements, N = 6 (about an hour)

Each problem is solved far past the 1e-10 residual of the benchmarks (Sec. IV.A; the discrete
solution is unique because A is symmetric positive definite), so that the stored u* differs from
the exact discrete solution by rounding only:
  * Gaussian source: multigrid-Schwarz FGMRES (Sec. III.B-III.E) from u = 0 until the Givens
    estimate of the relative residual is below 1e-14 (the true FP64 residual then stagnates near
    1e-13);
  * punctures: Newton-Raphson (Sec. III.A) with linearized solves to 1e-6 until the nonlinear
    residual is below 1e-13 of its initial value.
Beside each solution a JSON file records the oracle's iteration counts, residuals and wall time.
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402
from oracle import dg, krylov, solve  # noqa: E402


def _write(name, u, meta):
    np.save(os.path.join(HERE, name + "_u.npy"), np.ascontiguousarray(u.ravel(), dtype=np.float64))
    with open(os.path.join(HERE, name + "_u.json"), "w") as fh:
        json.dump(meta, fh, indent=1)
        fh.write("\n")


def gauss():
    cfg = workloads.GAUSS_8x8x8
    t0 = time.perf_counter()
    grid = dg.BoxGrid(cfg.lower, cfg.upper, cfg.n, cfg.N, cfg.penalty)
    pr = solve.Problem(grid, mg_levels=cfg.mg_levels, overlap=cfg.overlap, presmooth=cfg.presmooth,
                       postsmooth=cfg.postsmooth)
    x, y, z = grid.coordinates()
    b = dg.rhs(pr.graphs[0], workloads.gaussian_source(cfg.seed)(x, y, z))
    hist = []
    cb = lambda j, res: (hist.append(res), print(f"  iteration {j}: estimate {res:.3e}", flush=True))
    u, info = krylov.fgmres(pr.apply, b, None, pr.vcycle, 1e-14, 200, callback=cb)
    wall = time.perf_counter() - t0
    r = b.ravel() - pr.apply(u).ravel()
    meta = {"problem": cfg.name, "n_dof": int(u.size), "method": "oracle FGMRES + multigrid-Schwarz V-cycle, FP64",
            "iterations": info["iterations"], "estimate_history": [float(h) for h in info["history"]],
            "true_relative_residual": float(np.linalg.norm(r) / np.linalg.norm(b)), "wall_seconds": wall}
    _write(cfg.name, u, meta)
    print(json.dumps({k: v for k, v in meta.items() if k != "estimate_history"}))


def puncture():
    cfg = workloads.PUNCTURE_16
    t0 = time.perf_counter()
    grid = dg.BoxGrid(cfg.lower, cfg.upper, cfg.n, cfg.N, cfg.penalty)
    pr = solve.PunctureProblem(grid, workloads.BINARY_PUNCTURES, mg_levels=cfg.mg_levels, overlap=cfg.overlap,
                               presmooth=cfg.presmooth, postsmooth=cfg.postsmooth)
    r0 = np.linalg.norm(pr.residual(np.zeros_like(pr.mass)))

    def lin(u, r):
        du, info = pr.linear_solve(u, r, 1e-6)
        print(f"  linear solve: {info['iterations']} iterations, relative {info['history'][-1] / info['r0']:.2e}",
              flush=True)
        return du, info

    from oracle import newton

    u, info = newton.newton(pr.residual, lin, np.zeros_like(pr.mass), 1e-13, 20)
    wall = time.perf_counter() - t0
    rel = float(np.linalg.norm(pr.residual(u)) / r0)
    meta = {"problem": cfg.name, "n_dof": int(u.size),
            "method": "oracle Newton-Raphson, FGMRES + multigrid-Schwarz V-cycle per linearization, FP64",
            "newton_steps": info["steps"], "converged": bool(info["converged"]),
            "krylov_iterations": [li["iterations"] for li in info["linear_iterations"]],
            "residual_history": [float(h) for h in info["history"]],
            "true_relative_residual": rel, "wall_seconds": wall}
    _write(cfg.name, u, meta)
    print(json.dumps(meta))


if __name__ == "__main__":
    targets = sys.argv[1:] or ["gauss"]
    for t in targets:
        {"gauss": gauss, "puncture": puncture}[t]()
