"""The full elliptic solve assembled from the oracle's parts (Sec. III, Fig. overview).

Oracle code (test infrastructure only).

Linear (Poisson): flexible GMRES preconditioned by one multigrid V-cycle per iteration,
with additive Schwarz smoothing (3 pre, 3 post) on every level including the coarsest and
the explicit-inverse subdomain solver (here: exact dense solves of A_S).

Nonlinear (puncture): Newton-Raphson; each linearized problem solved by the same FGMRES +
V-cycle, where the finest level uses the linearized operator A_Delta + M diag(S'(u)) both
for residuals and subdomain problems (subdomain solver: 3 GMRES iterations preconditioned by
the Poisson subdomain inverse, Sec. III.E), and coarser levels use the Poisson operator
(reading: the linearization point is not transferred to coarse grids).
"""
from __future__ import annotations

import numpy as np

from . import dg, krylov, mg, newton, puncture, schwarz


class Problem:
    def __init__(self, grid: dg.BoxGrid, mg_levels=0, overlap=2, presmooth=3, postsmooth=3):
        self.grid = grid
        self.levels = mg.hierarchy(grid, mg_levels)
        self.graphs = [g.graph() for g in self.levels]
        self.schwarz = [schwarz.SchwarzLevel(g, overlap) for g in self.levels]
        self.presmooth, self.postsmooth = presmooth, postsmooth
        self.mass = dg.mass_diag(self.graphs[0])

    def apply(self, u, level=0):
        return dg.apply(self.graphs[level], u)

    def vcycle(self, r, operators=None, smoothers=None):
        if smoothers is None:
            smoothers = [lambda b, u, it, s=s: s.smooth(b, u, it) for s in self.schwarz]
        return mg.vcycle(self.levels, smoothers, r, self.presmooth, self.postsmooth, operators)

    def solve_linear(self, b, u0=None, tol=1e-10, max_iter=200, precondition=True, rel_to="r0"):
        pre = self.vcycle if precondition else None
        return krylov.fgmres(self.apply, b, u0, pre, tol, max_iter, rel_to=rel_to)


class PunctureProblem(Problem):
    def __init__(self, grid, punctures, **kw):
        super().__init__(grid, **kw)
        x, y, z = grid.coordinates()
        self.alpha, self.beta = puncture.alpha_beta(x, y, z, punctures)

    def residual(self, u):
        """b - A(u) with b = 0 and A(u) = A_Delta u + M S(u)."""
        return -(self.apply(u) + self.mass * puncture.source(u, self.alpha, self.beta))

    def linear_solve(self, u, r, tol=1e-4, max_iter=100, subdomain_iterations=3, subdomain_solver="gmres"):
        """One linearized solve (Eq. linearized) by FGMRES with the multigrid-Schwarz V-cycle. The
        finest level's subdomain problems A_S + D_S are solved by GMRES preconditioned with the
        Poisson inverse (subdomain_solver "gmres", Sec. III.E's Laplacian approximation) or by the
        explicit inverse of each subdomain's A_S + D_S ("inverse")."""
        D = self.mass * puncture.source_deriv(u, self.alpha, self.beta)
        lin = lambda du: self.apply(du) + D * du
        ops = [lin] + [lambda x, l=l: self.apply(x, l) for l in range(1, len(self.levels))]
        if subdomain_solver == "gmres":
            fine_solver = schwarz.gmres_subdomain_solver(self.schwarz[0], D, subdomain_iterations)
        elif subdomain_solver == "inverse":
            fine_solver = schwarz.inverse_subdomain_solver(self.schwarz[0], D)
        else:
            raise ValueError(subdomain_solver)
        smoothers = [lambda b, x, it: self.schwarz[0].smooth(b, x, it, lin, fine_solver)]
        smoothers += [lambda b, x, it, s=s: s.smooth(b, x, it) for s in self.schwarz[1:]]
        pre = lambda v: self.vcycle(v, ops, smoothers)
        du, info = krylov.fgmres(lin, r, None, pre, tol, max_iter)
        return du, info

    def solve(self, u0=None, tol=1e-10, linear_tol=1e-4, max_steps=20, subdomain_solver="gmres"):
        u0 = np.zeros_like(self.mass) if u0 is None else u0
        lin = lambda u, r: self.linear_solve(u, r, linear_tol, subdomain_solver=subdomain_solver)
        return newton.newton(self.residual, lin, u0, tol, max_steps)
