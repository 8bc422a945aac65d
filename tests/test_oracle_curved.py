"""Pins for the oracle's DG operator on curved (mapped) elements, Sec. II with the metric terms of
Eqs. massmat, stiffmat and liftop: reduction to the affine operator, invariance under rigid
motions (full metric tensor, tilted normals), exactness on fields linear in the physical
coordinates for a polynomial map, exact inheritance of a polynomial map by the coarse levels,
spectral convergence on a warped mesh, and the Schwarz/multigrid solver on curved elements; for a
variable coefficient K in -div(K grad u): scaling by a constant K, symmetry and definiteness on
affine elements, interpolation to the coarse levels, and spectral convergence."""
import numpy as np
import pytest

import workloads
from oracle import curved, dg, krylov, mg, schwarz, solve

RNG = np.random.default_rng(3)


def _box(n, N, lower=(-1.0,) * 3, upper=(1.0,) * 3, neumann=(False,) * 6):
    return dg.BoxGrid(tuple(lower), tuple(upper), tuple(n), N, 1.5, neumann)


def _rotation(a, b):
    rz = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    rx = np.array([[1, 0, 0], [0, np.cos(b), -np.sin(b)], [0, np.sin(b), np.cos(b)]])
    return rz @ rx


def warp(X, Y, Z):
    """Smooth warp of [-1,1]^3 that keeps its six faces planar (each term vanishes on the faces
    normal to the coordinate it moves), quadratic in each coordinate."""
    return (X + 0.1 * (1 - X**2) * Y, Y + 0.12 * (1 - Y**2) * Z * X, Z + 0.1 * (1 - Z**2) * (X + Y))


@pytest.mark.parametrize("n,N,neu", [((2, 2, 1), 4, (False,) * 6), ((1, 2, 3), 3, (True, False, False, True, False, False)),
                                     ((2, 1, 2), 5, (False,) * 6)])
def test_identity_map_reduces_to_affine_operator(n, N, neu):
    box = _box(n, N, (-1.0, -0.5, 0.0), (1.0, 0.7, 2.5), neu)
    ident = curved.MappedGrid.from_mapping(box, lambda X, Y, Z: (X, Y, Z))
    u = RNG.uniform(-1, 1, (box.n_elements, N, N, N))
    ref = dg.apply(box.graph(), u)
    assert np.abs(dg.apply(ident.graph(), u) - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.abs(dg.mass_diag(ident.graph()) - dg.mass_diag(box.graph())).max() <= 1e-15


def test_rigid_motion_leaves_operator_unchanged():
    """The Laplacian is invariant under rotations and translations: on a rotated, shifted box
    (every metric entry nonzero, normals off the axes) the operator on the same nodal values is
    the unrotated one."""
    box = _box((2, 2, 1), 4, (-1.0, -0.5, 0.0), (1.0, 0.7, 1.5))
    R = _rotation(0.7, 0.3)
    shift = np.array([0.3, -1.0, 2.0])
    rot = curved.MappedGrid.from_mapping(box, lambda X, Y, Z: tuple(R[i, 0] * X + R[i, 1] * Y + R[i, 2] * Z + shift[i]
                                                                    for i in range(3)))
    gr = rot.graph()
    assert np.abs(gr.G[:, 0, 1]).min() > 1e-2  # off-diagonal metric terms are exercised
    u = RNG.uniform(-1, 1, (box.n_elements, 4, 4, 4))
    ref = dg.apply(box.graph(), u)
    assert np.abs(dg.apply(gr, u) - ref).max() <= 1e-13 * np.abs(ref).max()


def test_linear_fields_are_annihilated_inside():
    """With a map of degree <= N - 1 the element interpolant is exact, so a field linear in the
    physical coordinates is represented exactly, its gradient is the constant vector, every interior
    jump and flux difference vanishes and D of a constant is zero: A u = 0 on the middle element of
    3^3 (the boundary faces' Dirichlet jumps only reach their own elements)."""
    for N in (3, 4, 6):
        g = curved.MappedGrid.from_mapping(_box((3, 3, 3), N), warp)
        x, y, z = g.coordinates()
        u = 0.7 * x - 1.3 * y + 0.4 * z + 0.25
        Au = dg.apply(g.graph(), u)
        mid = g.element_index(1, 1, 1)
        assert np.abs(Au[mid]).max() <= 1e-12 * np.abs(Au).max(), N
        assert np.abs(Au).max() > 1e-3  # boundary elements do see the boundary data


def test_coarse_levels_inherit_a_polynomial_map_exactly():
    """The quadratic warp is reproduced exactly by the fine elements (N >= 3), so the coarse
    level's interpolated nodes are the warp of the coarse box nodes."""
    box = _box((4, 2, 2), 4)
    fine = curved.MappedGrid.from_mapping(box, warp)
    for coarse_n in ((2, 1, 1), (2, 2, 2), (4, 1, 2)):
        got = fine.coarsen(coarse_n).coordinates()
        ref = warp(*box.coarsen(coarse_n).coordinates())
        for c, r in zip(got, ref):
            assert np.abs(c - r).max() <= 1e-13


def test_spectral_convergence_on_a_warped_mesh():
    """u = sin(pi x) sin(pi y) sin(pi z) vanishes on the (planar) faces of the warped box and
    solves -lap u = 3 pi^2 u: the discrete solution on curved elements converges exponentially in N."""
    errs = []
    for N in (4, 6, 8):
        g = curved.MappedGrid.from_mapping(_box((2, 2, 2), N), warp)
        gr = g.graph()
        x, y, z = g.coordinates()
        exact = np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
        b = dg.rhs(gr, 3 * np.pi**2 * exact)
        u = np.linalg.solve(dg.assemble(gr), b.ravel())
        errs.append(np.sqrt(np.mean((u - exact.ravel()) ** 2)))
    assert errs[1] < errs[0] / 10 and errs[2] < errs[1] / 10 and errs[2] < 1e-4, errs


def test_operator_is_positive_definite_not_symmetric():
    """On curved elements the chain-rule strong form is not exactly symmetric (the metric terms sit
    outside the derivatives), but its symmetric part stays positive definite: FGMRES applies, the
    subdomain matrices invert without pivoting."""
    g = curved.MappedGrid.from_mapping(_box((2, 2, 2), 4), warp)
    A = dg.assemble(g.graph())
    asym = np.abs(A - A.T).max() / np.abs(A).max()
    assert 1e-6 < asym < 0.1
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0


def test_curved_schwarz_and_multigrid_solve():
    """Single-element Schwarz is exact; the multigrid-Schwarz FGMRES solve on a warped 4 x 4 x 2 mesh
    (three curved levels) reaches the dense direct solution."""
    g1 = curved.MappedGrid.from_mapping(_box((1, 1, 1), 5), warp)
    gr1 = g1.graph()
    lv = schwarz.SchwarzLevel(g1, 2)
    b = dg.rhs(gr1, RNG.uniform(-1, 1, (1, 5, 5, 5)))
    u = lv.smooth(b, np.zeros_like(b), 1)
    assert np.linalg.norm(b - dg.apply(gr1, u)) <= 1e-12 * np.linalg.norm(b)

    g = curved.MappedGrid.from_mapping(_box((4, 4, 2), 4), warp)
    pr = solve.Problem(g, mg_levels=3)
    assert all(isinstance(level, curved.MappedGrid) for level in pr.levels)
    x, y, z = g.coordinates()
    b = dg.rhs(pr.graphs[0], workloads.gaussian_source(2)(x, y, z))
    u, info = pr.solve_linear(b, tol=1e-10)
    direct = np.linalg.solve(dg.assemble(pr.graphs[0]), b.ravel())
    assert np.linalg.norm(u.ravel() - direct) <= 1e-8 * np.linalg.norm(direct)
    assert info["iterations"] <= 30


# ---------------------------------------------------------------- variable coefficient: -div(K grad u)

def coef(x, y, z):
    return 1.0 + 0.5 * x**2 + 0.2 * y * z


def test_constant_coefficient_scales_the_operator():
    for mapping in (lambda X, Y, Z: (X, Y, Z), warp):
        box = _box((2, 2, 1), 4)
        plain = curved.MappedGrid.from_mapping(box, mapping)
        scaled = curved.MappedGrid.from_mapping(box, mapping, lambda x, y, z: 2.5 + 0 * x)
        u = RNG.uniform(-1, 1, (box.n_elements, 4, 4, 4))
        ref = 2.5 * dg.apply(plain.graph(), u)
        assert np.abs(dg.apply(scaled.graph(), u) - ref).max() <= 1e-13 * np.abs(ref).max()


def test_variable_coefficient_on_affine_elements_is_symmetric_positive_definite():
    """On affine elements the collocated strong form stays symmetric with K inside the divergence
    (summation by parts of the LGL operators), and positive definite."""
    g = curved.MappedGrid.from_mapping(_box((2, 2, 2), 4), lambda X, Y, Z: (X, Y, Z), coef)
    A = dg.assemble(g.graph())
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0


def test_coarse_levels_interpolate_the_coefficient():
    """K(warp(X)) has degree 4 in the logical coordinates, reproduced by N = 6 elements: the coarse
    level's interpolated coefficient is K at the coarse nodes."""
    box = _box((4, 2, 2), 6)
    fine = curved.MappedGrid.from_mapping(box, warp, coef)
    coarse = fine.coarsen((2, 1, 1))
    assert np.abs(coarse.K - coef(*warp(*box.coarsen((2, 1, 1)).coordinates()))).max() <= 1e-12


def test_variable_coefficient_spectral_convergence_on_a_warped_mesh():
    """u = sin(pi x) sin(pi y) sin(pi z) with K = 1 + x^2 / 2 solves -div(K grad u) = f with
    f = 3 pi^2 K u - x du/dx; the discrete solution converges exponentially in N."""
    errs = []
    K = lambda x, y, z: 1.0 + 0.5 * x**2
    for N in (4, 6, 8):
        g = curved.MappedGrid.from_mapping(_box((2, 2, 2), N), warp, K)
        gr = g.graph()
        x, y, z = g.coordinates()
        exact = np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
        f = 3 * np.pi**2 * K(x, y, z) * exact - x * np.pi * np.cos(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
        u = np.linalg.solve(dg.assemble(gr), dg.rhs(gr, f).ravel())
        errs.append(np.sqrt(np.mean((u - exact.ravel()) ** 2)))
    assert errs[1] < errs[0] / 10 and errs[2] < errs[1] / 10 and errs[2] < 1e-4, errs
