"""Pins for the oracle's DG operator (Sec. II, Eqs. dg_op_auxvars, dg_op_primal, numflux,
penalty, bc) against facts fixed by the mathematics, not by the oracle itself."""
import itertools
import math

import numpy as np
import pytest
import sympy as sp

import workloads
from oracle import dg, lgl


def _box(n, N, C=1.5, lower=(-1.0,) * 3, upper=(1.0,) * 3, neumann=(False,) * 6):
    return dg.BoxGrid(tuple(lower), tuple(upper), tuple(n), N, C, tuple(neumann))


def sipg_matrix(grid: dg.BoxGrid) -> np.ndarray:
    """Independent brute-force assembly of the symmetric interior-penalty bilinear form
    a(w,u) = sum_K (grad w, grad u)_K - sum_F ({d_n w}[u] + {d_n u}[w])_F + sum_F (sigma_F [w][u])_F
    with LGL quadrature, sigma_F = C N^2 / h_perp on interior faces and 2 C N^2 / h_perp on
    Dirichlet faces (the mirror ghost of Eq. bc doubles the jump), and no face term at all on
    homogeneous Neumann faces (the natural boundary condition). Summation by parts on LGL points
    turns the paper's strong form into exactly this form."""
    N, E = grid.N, grid.n_elements
    x, w = lgl.lgl_nodes(N), lgl.lgl_weights(N)
    Dh = lgl.diff_matrix(N)
    I = np.eye(N)
    h = grid.h
    n3 = N**3
    G1 = [np.kron(np.kron(I, I), Dh), np.kron(np.kron(I, Dh), I), np.kron(np.kron(Dh, I), I)]  # x, y, z
    W3 = np.kron(np.kron(w, w), w)  # [k, j, i]
    J = np.prod(h) / 8
    ndof = E * n3
    A = np.zeros((ndof, ndof))

    def blk(e):
        return slice(e * n3, (e + 1) * n3)

    G = [2.0 / h[d] * G1[d] for d in range(3)]
    for e in range(E):
        for d in range(3):
            A[blk(e), blk(e)] += G[d].T @ (J * W3[:, None] * G[d])
    kji = np.array(list(itertools.product(range(N), repeat=3)))  # rows (k, j, i)

    def face_rows(d, side):
        along = kji[:, 2 - d]
        return np.nonzero(along == (0 if side == 0 else N - 1))[0]

    sigma = grid.penalty * N**2
    for e in range(E):
        for d in range(3):
            tang = [t for t in range(3) if t != d]
            Jf = np.prod(h[tang]) / 4
            for side in (0, 1):
                rows = face_rows(d, side)
                tw = np.ones(len(rows))
                for t in tang:
                    tw = tw * w[kji[rows, 2 - t]]
                B = np.diag(Jf * tw)
                s = 1.0 if side else -1.0
                q = grid.neighbor(e, 2 * d + side)
                Te = np.zeros((len(rows), ndof))
                Te[np.arange(len(rows)), e * n3 + rows] = 1.0
                dTe = np.zeros((len(rows), ndof))
                dTe[:, blk(e)] = s * G[d][rows]
                if q == dg.EXTERNAL:
                    jump, avg, sig = Te, dTe, 2 * sigma / h[d]
                elif q == dg.NEUMANN:
                    continue
                elif side == 1:  # count each interior face once, from its lower element
                    rows_q = face_rows(d, 0)
                    Tq = np.zeros((len(rows), ndof))
                    Tq[np.arange(len(rows)), q * n3 + rows_q] = 1.0
                    dTq = np.zeros((len(rows), ndof))
                    dTq[:, blk(q)] = s * G[d][rows_q]
                    jump, avg, sig = Te - Tq, 0.5 * (dTe + dTq), sigma / h[d]
                else:
                    continue
                A += -avg.T @ B @ jump - jump.T @ B @ avg + sig * jump.T @ B @ jump
    return A


@pytest.mark.parametrize("n,N", [((1, 1, 1), 2), ((2, 1, 1), 3), ((2, 2, 1), 3), ((2, 2, 2), 4), ((3, 1, 2), 3)])
def test_strong_form_equals_sipg_bilinear_form(n, N):
    grid = _box(n, N, lower=(-1.0, -0.5, 0.0), upper=(1.0, 0.5, 3.0))
    A = dg.assemble(grid.graph())
    S = sipg_matrix(grid)
    assert np.abs(A - S).max() <= 1e-12 * np.abs(S).max()


@pytest.mark.parametrize("n,N", [((1, 1, 1), 2), ((2, 2, 2), 3), ((2, 1, 3), 5), ((1, 2, 1), 4)])
def test_symmetric_positive_definite(n, N):
    A = dg.assemble(_box(n, N).graph())
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
    np.linalg.cholesky(A)  # raises if not positive definite


def test_polynomial_consistency():
    """For u vanishing on the boundary and smooth across faces, every flux difference vanishes and
    D_hat is exact, so A u = M (-Laplace u) at every node."""
    X, Y, Z = sp.symbols("x y z")
    U = (1 - X**2) * (1 - Y**2) * (1 - Z**2) * (1 + sp.Rational(3, 10) * X - sp.Rational(1, 5) * Y * Z)
    lap = sp.lambdify((X, Y, Z), -(sp.diff(U, X, 2) + sp.diff(U, Y, 2) + sp.diff(U, Z, 2)), "numpy")
    uf = sp.lambdify((X, Y, Z), U, "numpy")
    for n, N in [((2, 2, 2), 4), ((3, 2, 1), 5), ((1, 1, 1), 6)]:
        grid = _box(n, N)
        gr = grid.graph()
        x, y, z = grid.coordinates()
        Au = dg.apply(gr, uf(x, y, z))
        ref = dg.mass_diag(gr) * lap(x, y, z)
        assert np.abs(Au - ref).max() <= 1e-13 * np.abs(ref).max()


def test_matrix_free_equals_dense_on_random_vectors():
    grid = _box((2, 2, 1), 4)
    gr = grid.graph()
    A = dg.assemble(gr)
    u = workloads.uniform_vector(7, A.shape[0])
    Au = dg.apply(gr, u.reshape(gr.n_elements, 4, 4, 4)).ravel()
    assert np.abs(Au - A @ u).max() <= 1e-13 * np.abs(Au).max()


def _solve(grid):
    gr = grid.graph()
    A = dg.assemble(gr)
    x, y, z = grid.coordinates()
    b = dg.rhs(gr, workloads.sine_source_3d(x, y, z)).ravel()
    u = np.linalg.solve(A, b)
    return math.sqrt(np.mean((u - workloads.sine_solution_3d(x, y, z).ravel()) ** 2))


def test_manufactured_p_convergence():
    """u = sin(pi x) sin(pi y) sin(pi z), f = 3 pi^2 u: the RMS nodal error decays exponentially in N."""
    errs = [_solve(_box((1, 1, 1), N)) for N in (4, 6, 8, 10)]
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert min(ratios) > 20  # each +2 in N gains more than a factor 20 ...
    assert ratios[2] > 0.9 * ratios[0]  # ... and the gain does not shrink (exponential, not algebraic)
    assert errs[3] < 1e-5


def test_manufactured_h_convergence():
    e1 = _solve(_box((1, 1, 1), 4))
    e2 = _solve(_box((2, 2, 2), 4))
    assert e1 / e2 > 2 ** 3.5  # at least ~h^N order at N = 4


def test_penalty_enters_only_through_jumps():
    """A(C1) - A(C2) is a pure jump (penalty) term: it annihilates fields continuous across
    faces and vanishing on the boundary."""
    grid1, grid2 = _box((2, 2, 2), 3, C=1.0), _box((2, 2, 2), 3, C=2.5)
    x, y, z = grid1.coordinates()
    u = (1 - x**2) * (1 - y**2) * (1 - z**2)
    d = dg.apply(grid1.graph(), u) - dg.apply(grid2.graph(), u)
    assert np.abs(d).max() < 1e-13
    r = workloads.uniform_vector(3, u.size).reshape(u.shape)
    assert np.abs(dg.apply(grid1.graph(), r) - dg.apply(grid2.graph(), r)).max() > 1e-2


def test_scaling_with_element_size():
    """For cubic elements in 3-D every term of A scales as h: A(h) = h A(1)."""
    a = dg.assemble(_box((2, 1, 1), 3, lower=(0, 0, 0), upper=(2, 1, 1)).graph())
    b = dg.assemble(_box((2, 1, 1), 3, lower=(0, 0, 0), upper=(0.5, 0.25, 0.25)).graph())
    assert np.abs(b - 0.25 * a).max() <= 1e-13 * np.abs(a).max()


# ---------------------------------------------------------------- homogeneous Neumann faces
NEU_YZ = (False, False, True, True, True, True)  # Dirichlet at x = +-1, Neumann on the y and z faces


@pytest.mark.parametrize("n,N,neu", [((1, 1, 1), 3, (True,) * 6), ((2, 1, 1), 3, NEU_YZ),
                                     ((2, 2, 1), 3, (True, False, False, True, False, True)),
                                     ((1, 2, 2), 4, NEU_YZ)])
def test_neumann_strong_form_equals_sipg_bilinear_form(n, N, neu):
    grid = _box(n, N, lower=(-1.0, -0.5, 0.0), upper=(1.0, 0.5, 3.0), neumann=neu)
    A = dg.assemble(grid.graph())
    S = sipg_matrix(grid)
    assert np.abs(A - S).max() <= 1e-12 * np.abs(S).max()


def test_pure_neumann_operator_annihilates_constants():
    """With every box face Neumann, constants have zero gradient, zero jumps and zero boundary
    flux, so A 1 = 0 exactly; the operator stays symmetric."""
    for n, N in [((1, 1, 1), 4), ((2, 1, 3), 3), ((2, 2, 2), 5)]:
        gr = _box(n, N, neumann=(True,) * 6).graph()
        one = np.ones((gr.n_elements, N, N, N))
        Au = dg.apply(gr, one)
        A = dg.assemble(gr)
        assert np.abs(Au).max() <= 1e-12 * np.abs(A).max()
        assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()


@pytest.mark.parametrize("n,N,neu", [((2, 2, 2), 3, NEU_YZ), ((1, 2, 1), 4, (True,) * 5 + (False,)),
                                     ((2, 1, 2), 4, (False, True, False, True, False, True))])
def test_mixed_boundaries_symmetric_positive_definite(n, N, neu):
    A = dg.assemble(_box(n, N, neumann=neu).graph())
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
    np.linalg.cholesky(A)  # one Dirichlet face is enough


def test_mixed_boundaries_polynomial_consistency():
    """u = (1 - x^2)(1 - y^2)^2 (1 - z^2)^2 vanishes at x = +-1 and has zero normal derivative on
    the y and z faces: no jump anywhere, every boundary flux exact, so A u = M (-Laplace u)."""
    X, Y, Z = sp.symbols("x y z")
    U = (1 - X**2) * (1 - Y**2) ** 2 * (1 - Z**2) ** 2
    lap = sp.lambdify((X, Y, Z), -(sp.diff(U, X, 2) + sp.diff(U, Y, 2) + sp.diff(U, Z, 2)), "numpy")
    uf = sp.lambdify((X, Y, Z), U, "numpy")
    for n, N in [((2, 2, 2), 5), ((1, 3, 2), 6)]:
        grid = _box(n, N, neumann=NEU_YZ)
        gr = grid.graph()
        x, y, z = grid.coordinates()
        Au = dg.apply(gr, uf(x, y, z))
        ref = dg.mass_diag(gr) * lap(x, y, z)
        assert np.abs(Au - ref).max() <= 1e-12 * np.abs(ref).max()


def test_mixed_boundaries_manufactured_p_convergence():
    """u = sin(pi x) cos(pi y) cos(pi z), f = 3 pi^2 u, Dirichlet at x = +-1 and Neumann on the other
    faces (both hold exactly for this u): the nodal error decays exponentially in N."""
    errs = []
    for N in (4, 6, 8):
        grid = _box((2, 2, 2), N, neumann=NEU_YZ)
        gr = grid.graph()
        x, y, z = grid.coordinates()
        ue = np.sin(math.pi * x) * np.cos(math.pi * y) * np.cos(math.pi * z)
        u = np.linalg.solve(dg.assemble(gr), dg.rhs(gr, 3 * math.pi**2 * ue).ravel())
        errs.append(math.sqrt(np.mean((u - ue.ravel()) ** 2)))
    assert errs[0] / errs[1] > 20 and errs[1] / errs[2] > 0.9 * errs[0] / errs[1]
    assert errs[2] < 1e-5


def _sipg_1d(n, N, h, C):
    """Textbook 1-D symmetric interior-penalty matrix on n elements of width h with LGL quadrature
    and homogeneous Dirichlet ends: sum_K int w' u' - sum_F ({n w'}[u] + {n u'}[w] - sigma [w][u]),
    sigma = C N^2 / h inside, and at an end (mirror ghost) the consistency terms with the interior
    derivative and the penalty doubled. Written from the 1-D weak form, not from the 3-D code."""
    w = lgl.lgl_weights(N)
    D = (2.0 / h) * lgl.diff_matrix(N)
    A = np.zeros((n * N, n * N))
    sig = C * N**2 / h
    blk = lambda e: slice(e * N, (e + 1) * N)
    for e in range(n):
        A[blk(e), blk(e)] += D.T @ np.diag(0.5 * h * w) @ D
    # interior faces: element e (node N-1) | element e+1 (node 0), normal +x
    for e in range(n - 1):
        rows = np.zeros((2, n * N))  # jump [u] = u_e(N-1) - u_{e+1}(0), average of u'
        rows[0, e * N + N - 1] = 1.0
        rows[0, (e + 1) * N] = -1.0
        rows[1, blk(e)] = 0.5 * D[N - 1]
        rows[1, blk(e + 1)] = 0.5 * D[0]
        jump, avg = rows[0], rows[1]
        A += -np.outer(avg, jump) - np.outer(jump, avg) + sig * np.outer(jump, jump)
    # Dirichlet ends: outward normal -1 at node 0 of element 0, +1 at node N-1 of element n-1
    for node, nrm, dl in ((0, -1.0, D[0]), ((n - 1) * N + N - 1, 1.0, D[N - 1])):
        e = 0 if nrm < 0 else n - 1
        val = np.zeros(n * N)
        val[node] = 1.0
        der = np.zeros(n * N)
        der[blk(e)] = nrm * dl
        A += -np.outer(der, val) - np.outer(val, der) + 2.0 * sig * np.outer(val, val)
    return A


@pytest.mark.parametrize("n,N", [(1, 3), (3, 4), (4, 6)])
def test_one_dimensional_reduction(n, N):
    """One element across y and z with homogeneous Neumann faces there and a field constant in y and
    z: the operator is the textbook 1-D SIPG matrix in x times the y and z mass weights."""
    C = 1.5
    grid = _box((n, 1, 1), N, C, lower=(-1.0, 0.0, -0.5), upper=(2.0, 0.8, 1.5),
                neumann=(False, False, True, True, True, True))
    hx, hy, hz = 3.0 / n, 0.8, 2.0
    ux = workloads.uniform_vector(7, n * N).reshape(n, N)
    u = np.broadcast_to(ux[:, None, None, :], (n, N, N, N)).copy()  # [e, k, j, i]
    Au = dg.apply(grid.graph(), u)
    A1 = _sipg_1d(n, N, hx, C) @ ux.ravel()
    w = lgl.lgl_weights(N)
    ref = A1.reshape(n, 1, 1, N) * (0.5 * hz * w)[None, :, None, None] * (0.5 * hy * w)[None, None, :, None]
    assert np.abs(Au - ref).max() <= 1e-12 * np.abs(ref).max()
