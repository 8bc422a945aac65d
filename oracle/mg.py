"""Geometric h-multigrid of Sec. III.C: grid hierarchy, intermesh operators, V-cycle.

Oracle code (test infrastructure only).

Hierarchy (Sec. III.C.1): level l+1 combines two elements of level l into one along every
dimension whose element count is even (a dimension with an odd count keeps its elements:
those children cover the full parent in that dimension). Isotropic order N on all levels.
A_l is the DG discretization of Sec. II on grid l (rediscretized, not a Galerkin product).

Prolongation (Eq. prol): Lagrange interpolation from the parent's points to the child's
points at parent-logical coordinates xi~ = (xi - 1)/2 (lower half), (xi + 1)/2 (upper
half) or xi (child covers the full parent). Restriction R = P^T, with no mass matrices.
"""
from __future__ import annotations

import numpy as np

from . import dg, lgl


def hierarchy(grid: dg.BoxGrid, max_levels: int = 0):
    """Grids of all levels, finest first. max_levels = 0 coarsens while possible."""
    levels = [grid]
    while max_levels == 0 or len(levels) < max_levels:
        n = levels[-1].n
        if all(c % 2 for c in n):
            break
        coarse_n = tuple(c // 2 if c % 2 == 0 else c for c in n)
        levels.append(levels[-1].coarsen(coarse_n))
    return levels


def _interp(N):
    x = lgl.lgl_nodes(N)
    return {
        0: lgl.interp_matrix(N, 0.5 * (x - 1.0)),  # child on the lower half
        1: lgl.interp_matrix(N, 0.5 * (x + 1.0)),  # child on the upper half
        None: lgl.interp_matrix(N, x),  # child covers the full parent
    }


def _parent_map(fine: dg.BoxGrid, coarse: dg.BoxGrid):
    """For every fine element: its parent and, per dimension, its half (None = full)."""
    out = []
    for e in range(fine.n_elements):
        c = fine.element_coords(e)
        pc, halves = [], []
        for d in range(3):
            if coarse.n[d] == fine.n[d]:
                pc.append(c[d])
                halves.append(None)
            else:
                pc.append(c[d] // 2)
                halves.append(c[d] % 2)
        out.append((coarse.element_index(*pc), tuple(halves)))
    return out


def prolongate(fine: dg.BoxGrid, coarse: dg.BoxGrid, uc: np.ndarray) -> np.ndarray:
    """u_fine = P u_coarse (Eq. prol)."""
    I = _interp(fine.N)
    N = fine.N
    uf = np.zeros(uc.shape[:-4] + (fine.n_elements, N, N, N))
    for e, (p, (hx, hy, hz)) in enumerate(_parent_map(fine, coarse)):
        uf[..., e, :, :, :] = np.einsum("kc,jb,ia,...cba->...kji", I[hz], I[hy], I[hx], uc[..., p, :, :, :])
    return uf


def restrict(fine: dg.BoxGrid, coarse: dg.BoxGrid, rf: np.ndarray) -> np.ndarray:
    """b_coarse = R r_fine with R = P^T."""
    I = _interp(fine.N)
    N = fine.N
    bc = np.zeros(rf.shape[:-4] + (coarse.n_elements, N, N, N))
    for e, (p, (hx, hy, hz)) in enumerate(_parent_map(fine, coarse)):
        bc[..., p, :, :, :] += np.einsum("kc,jb,ia,...kji->...cba", I[hz], I[hy], I[hx], rf[..., e, :, :, :])
    return bc


def vcycle(levels, smoothers, b0, presmooth=3, postsmooth=3, operators=None):
    """One V-cycle on A_0 u = b0 from a zero initial guess (Sec. III.C.3).

    levels:    BoxGrids, finest first
    smoothers: callables smooth(b, u, iterations) -> u for every level
    operators: callables A_l(u); default: the Poisson DG operator of each level
    """
    L = len(levels)
    if operators is None:
        graphs = [g.graph() for g in levels]
        operators = [lambda u, gr=gr: dg.apply(gr, u) for gr in graphs]
    b = [None] * L
    u = [None] * L
    b[0] = b0
    for l in range(L - 1):
        u[l] = smoothers[l](b[l], np.zeros_like(b[l]), presmooth)  # presmoothing
        r = b[l] - operators[l](u[l])  # Eq. mg_res
        b[l + 1] = restrict(levels[l], levels[l + 1], r)
    # tip of the V: presmoothing and postsmoothing on the coarsest grid
    u[L - 1] = smoothers[L - 1](b[L - 1], np.zeros_like(b[L - 1]), presmooth)
    u[L - 1] = smoothers[L - 1](b[L - 1], u[L - 1], postsmooth)
    for l in range(L - 2, -1, -1):
        u[l] = u[l] + prolongate(levels[l], levels[l + 1], u[l + 1])
        u[l] = smoothers[l](b[l], u[l], postsmooth)
    return u[0]
