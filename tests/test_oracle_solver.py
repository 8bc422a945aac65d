"""Pins for the oracle's multigrid transfers, Schwarz smoother, FGMRES and Newton
(Secs. III.A-III.E) against invariants, special cases and dense direct solves."""
import json
import math
import os

import numpy as np
import pytest

import workloads
from oracle import dg, krylov, lgl, mg, newton, puncture, schwarz, solve

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def _box(n, N, C=1.5, lower=(-1.0,) * 3, upper=(1.0,) * 3):
    return dg.BoxGrid(tuple(lower), tuple(upper), tuple(n), N, C)


# ---------------------------------------------------------------- multigrid (Sec. III.C)

def test_hierarchy_coarsens_even_dimensions():
    lv = mg.hierarchy(_box((8, 4, 3), 4))
    assert [g.n for g in lv] == [(8, 4, 3), (4, 2, 3), (2, 1, 3), (1, 1, 3)]
    assert [g.n for g in mg.hierarchy(_box((8, 8, 8), 4), 3)] == [(8, 8, 8), (4, 4, 4), (2, 2, 2)]


@pytest.mark.parametrize("n", [(2, 2, 2), (4, 2, 1), (2, 3, 2)])
def test_prolongation_exact_on_coarse_polynomials(n):
    N = 4
    fine = _box(n, N, lower=(-1, 0, 2), upper=(1, 3, 4))
    coarse = mg.hierarchy(fine)[1]
    poly = lambda x, y, z: 1 + x - 2 * y + x**3 * y**2 - 0.5 * z**3 + x * y * z
    uc = poly(*coarse.coordinates())
    uf = mg.prolongate(fine, coarse, uc)
    assert np.abs(uf - poly(*fine.coordinates())).max() < 1e-12


def test_restriction_is_transpose_of_prolongation():
    N = 3
    fine = _box((4, 2, 2), N)
    coarse = mg.hierarchy(fine)[1]
    xc = workloads.uniform_vector(1, coarse.n_elements * N**3).reshape(coarse.n_elements, N, N, N)
    yf = workloads.uniform_vector(2, fine.n_elements * N**3).reshape(fine.n_elements, N, N, N)
    lhs = np.sum(mg.prolongate(fine, coarse, xc) * yf)
    rhs = np.sum(xc * mg.restrict(fine, coarse, yf))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


# ---------------------------------------------------------------- Schwarz (Sec. III.D)

def test_smoothstep_and_weight_function_closed_forms():
    assert schwarz.phi(0.5) == pytest.approx((15 * 0.5 - 10 * 0.125 + 3 * 0.03125) / 8, abs=1e-16)
    assert schwarz.phi(1.0) == 1.0 and schwarz.phi(-1.0) == -1.0 and schwarz.phi(2.5) == 1.0
    for delta in (0.3, 0.71, 2.0):
        assert schwarz.w1d(0.0, delta) == pytest.approx(1.0 if delta <= 1 else 0.5 * (2 * schwarz.phi(1 / delta)))
        assert schwarz.w1d(3.0, delta) == 0.0 and schwarz.w1d(-3.0, delta) == 0.0
        assert schwarz.w1d(1.0, delta) == pytest.approx(0.5)


def test_overlap_width_values():
    # first excluded point of a 6-point neighbour at N_overlap = 2 is x_2 = -0.2852315165
    assert schwarz.overlap_width(6, 2) == pytest.approx(0.7147684835, abs=1e-10)
    assert schwarz.overlap_width(8, 2) == pytest.approx(1 - 0.5917001814, abs=1e-10)
    assert schwarz.overlap_width(6, 5) == 2.0


def test_interior_subdomain_size_matches_paper():
    """Sec. III.E: 8^3 points, N_overlap = 2 and five fields give a 6400 x 6400 subdomain matrix."""
    gold = json.load(open(GOLDEN))["xcts_subdomain_matrix_size"]
    lv = schwarz.SchwarzLevel(_box((3, 3, 3), gold["points_per_dim"]), gold["overlap"])
    centre = 13
    assert gold["fields"] * len(lv.subdomains[centre]["glob"]) == gold["value"]


@pytest.mark.parametrize("n,N,ov", [((3, 2, 1), 5, 2), ((3, 3, 3), 4, 1), ((2, 2, 2), 3, 2), ((4, 1, 2), 6, 5)])
def test_weights_partition_of_unity_and_support(n, N, ov):
    lv = schwarz.SchwarzLevel(_box(n, N), ov)
    total = np.zeros(lv.grid.n_elements * N**3)
    for sd in lv.subdomains:
        np.add.at(total, sd["glob"], sd["weight"])
    assert np.abs(total - 1.0).max() < 1e-14
    # every weight a subdomain would give a point outside it is zero
    assert np.all(lv.shares >= -1e-15)
    for e in range(lv.grid.n_elements):
        for f in range(6):
            q = lv.graph.nbr[e, f]
            if q < 0:
                continue
            d, side = divmod(f, 2)
            back = 2 * d + (1 - side)
            along = np.arange(N) if side == 1 else np.arange(N)[::-1]
            outside = np.nonzero(along >= ov)[0]
            sl = [slice(None)] * 3
            sl[2 - d] = outside
            assert np.abs(lv.shares[q][tuple(sl)][..., 1 + back]).max() == 0.0


def test_face_neighbour_weight_is_product_away_from_edges():
    """Eq. schwarz_weight_prod: W = prod_i w(xi^i) where no edge/corner weight is redistributed."""
    N, ov = 6, 2
    lv = schwarz.SchwarzLevel(_box((3, 3, 3), N), ov)
    x = lgl.lgl_nodes(N)
    delta = schwarz.overlap_width(N, ov)
    e = 13  # centre element; its +x neighbour's subdomain reaches into it
    k = j = 2  # away from the y, z faces: no b_y, b_z factors
    for i in (N - 1, N - 2):
        expect = schwarz.w1d(x[i] - 2, delta) * schwarz.w1d(x[j], delta) * schwarz.w1d(x[k], delta)
        assert lv.shares[e, k, j, i, 1 + 1] == pytest.approx(expect, abs=1e-15)
        assert lv.shares[e, k, j, i, 0] == pytest.approx(
            schwarz.w1d(x[i], delta) * schwarz.w1d(x[j], delta) * schwarz.w1d(x[k], delta), abs=1e-15)


def test_subdomain_operator_is_restricted_global_operator():
    grid = _box((3, 2, 2), 3)
    A = dg.assemble(grid.graph())
    lv = schwarz.SchwarzLevel(grid, 2)
    for e in range(grid.n_elements):
        g = lv.subdomains[e]["glob"]
        assert np.abs(lv.subdomain_matrix(e) - A[np.ix_(g, g)]).max() <= 1e-14 * np.abs(A).max()


@pytest.mark.parametrize("neumann", [(False,) * 6, (False, False, True, True, True, True)])
def test_single_element_schwarz_is_exact(neumann):
    grid = dg.BoxGrid((-1.0,) * 3, (1.0,) * 3, (1, 1, 1), 5, 1.5, neumann)
    gr = grid.graph()
    lv = schwarz.SchwarzLevel(grid, 2)
    x, y, z = grid.coordinates()
    b = dg.rhs(gr, workloads.sine_source_3d(x, y, z))
    u = lv.smooth(b, np.zeros_like(b), 1)
    assert np.linalg.norm(b - dg.apply(gr, u)) <= 1e-12 * np.linalg.norm(b)


# ---------------------------------------------------------------- FGMRES (Sec. III.B)

def test_fgmres_matches_direct_solve_and_basis_is_orthonormal():
    grid = _box((2, 2, 2), 4)
    pr = solve.Problem(grid)
    x, y, z = grid.coordinates()
    b = dg.rhs(pr.graphs[0], workloads.sine_source_3d(x, y, z))
    ud = np.linalg.solve(dg.assemble(pr.graphs[0]), b.ravel())
    for pre in (False, True):
        u, info = pr.solve_linear(b, tol=1e-13, precondition=pre)
        assert info["converged"]
        assert np.linalg.norm(u.ravel() - ud) <= 1e-11 * np.linalg.norm(ud)
        h = np.array(info["history"])
        assert np.all(np.diff(h) <= 1e-12 * h[0])
        # Arnoldi basis orthonormal while the residual is well above rounding
        _, info8 = pr.solve_linear(b, tol=1e-8, precondition=pre)
        assert info8["orthonormality"] < 1e-9


def test_fcg_without_preconditioner_is_conjugate_gradients():
    """With M = I the flexible CG reduces to the textbook conjugate gradient method: the same
    iterates as scipy's CG, mutually A-orthogonal search directions, and the dense direct solution
    within n iterations."""
    from scipy.sparse.linalg import cg

    grid = _box((2, 1, 2), 3)
    gr = grid.graph()
    A = dg.assemble(gr)
    n = A.shape[0]
    b = workloads.uniform_vector(21, n, -1.0, 1.0)
    op = lambda u: dg.apply(gr, u.reshape(-1, 3, 3, 3)).ravel()
    steps = []
    cg(A, b, rtol=1e-30, maxiter=8, callback=lambda xk: steps.append(xk.copy()))
    for k, xk in enumerate(steps, start=1):
        xf, _ = krylov.fcg(op, b, tol=1e-30, max_iter=k)
        assert np.linalg.norm(xf - xk) <= 1e-9 * np.linalg.norm(xk)
    x, info = krylov.fcg(op, b, tol=1e-12, max_iter=n + 5, keep_directions=True)
    assert info["converged"] and info["iterations"] <= n
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-10 * np.linalg.norm(x)
    P = [d[0] for d in info["directions"][:6]]
    for i in range(len(P)):
        for j in range(i):
            c = P[i] @ A @ P[j] / math.sqrt((P[i] @ A @ P[i]) * (P[j] @ A @ P[j]))
            assert abs(c) < 1e-8


def test_multigrid_schwarz_with_neumann_faces_matches_direct_solve():
    """Mixed boundaries (Dirichlet at x = +-1, homogeneous Neumann elsewhere) on every level of the
    V-cycle and in every subdomain matrix: FGMRES reaches the direct solution."""
    grid = dg.BoxGrid((-1.0,) * 3, (1.0,) * 3, (4, 2, 2), 4, 1.5, (False, False, True, True, True, True))
    pr = solve.Problem(grid)
    x, y, z = grid.coordinates()
    b = dg.rhs(pr.graphs[0], workloads.gaussian_source(3)(x, y, z))
    ud = np.linalg.solve(dg.assemble(pr.graphs[0]), b.ravel())
    u, info = pr.solve_linear(b, tol=1e-12)
    assert info["converged"] and info["iterations"] < 30
    assert np.linalg.norm(u.ravel() - ud) <= 1e-9 * np.linalg.norm(ud)


def test_fcg_with_multigrid_schwarz_matches_direct_solve():
    """The flexible CG preconditioned by the multigrid-Schwarz V-cycle (not exactly symmetric: the
    Schwarz weights act on one side only) reaches the direct solution, in a number of iterations of
    the order of FGMRES's."""
    grid = _box((4, 4, 2), 4)
    pr = solve.Problem(grid)
    x, y, z = grid.coordinates()
    b = dg.rhs(pr.graphs[0], workloads.gaussian_source(2)(x, y, z))
    ud = np.linalg.solve(dg.assemble(pr.graphs[0]), b.ravel())
    u, info = krylov.fcg(pr.apply, b, precond=pr.vcycle, tol=1e-12)
    assert info["converged"]
    assert np.linalg.norm(u.ravel() - ud) <= 1e-10 * np.linalg.norm(ud)
    _, ginfo = pr.solve_linear(b, tol=1e-12)
    assert info["iterations"] <= 2 * ginfo["iterations"] + 2


def test_multigrid_schwarz_beats_schwarz_beats_unpreconditioned():
    """Sec. IV.A: Schwarz preconditioning cuts iterations by about an order of magnitude,
    multigrid-Schwarz further."""
    grid = _box((4, 4, 4), 4)
    x, y, z = grid.coordinates()
    gr = grid.graph()
    b = dg.rhs(gr, workloads.sine_source_3d(x, y, z))
    u0 = workloads.uniform_vector(11, b.size, -0.5, 0.5).reshape(b.shape)  # random guess as in Sec. IV.A
    plain = krylov.fgmres(lambda u: dg.apply(gr, u), b, u0, tol=1e-8, max_iter=400)[1]["iterations"]
    sw = schwarz.SchwarzLevel(grid, 2)
    only = krylov.fgmres(lambda u: dg.apply(gr, u), b, u0, precond=lambda r: sw.smooth(r, np.zeros_like(r), 3),
                         tol=1e-8)[1]["iterations"]
    mgs = solve.Problem(grid).solve_linear(b, u0, tol=1e-8)[1]["iterations"]
    assert plain > 5 * only and only > 2 * mgs


@pytest.mark.slow
def test_multigrid_iterations_independent_of_h():
    """Sec. IV.A: with one multigrid-Schwarz V-cycle per iteration the count stays flat under h refinement."""
    counts = []
    for n in (2, 4, 8):
        grid = _box((n, n, n), 4)
        x, y, z = grid.coordinates()
        pr = solve.Problem(grid)
        b = dg.rhs(pr.graphs[0], workloads.sine_source_3d(x, y, z))
        counts.append(pr.solve_linear(b, tol=1e-10)[1]["iterations"])
    assert max(counts[1:]) - min(counts[1:]) <= 2, counts
    assert max(counts) <= 12, counts


# ---------------------------------------------------------------- Newton (Sec. III.A)

def test_newton_zero_momentum_gives_zero_solution():
    grid = _box((2, 2, 2), 4, lower=(-20,) * 3, upper=(20,) * 3)
    still = tuple(workloads.Puncture(p.position, p.mass, (0.0, 0.0, 0.0)) for p in workloads.BINARY_PUNCTURES)
    pr = solve.PunctureProblem(grid, still)
    assert np.abs(pr.beta).max() == 0.0
    u, rep = pr.solve()
    assert rep["steps"] == 0 and np.abs(u).max() == 0.0


def test_newton_manufactured_nonlinear_solution():
    """Add a fixed source so that a chosen smooth u_m solves -Lap u + S(u) = f_m exactly in the
    continuum: the discrete Newton solution converges to u_m in N, quadratically in steps."""
    errs = []
    for N in (4, 6):
        grid = _box((2, 2, 2), N, lower=(-4,) * 3, upper=(4,) * 3)
        pr = solve.PunctureProblem(grid, workloads.BINARY_PUNCTURES)
        x, y, z = grid.coordinates()
        c = (math.pi / 8.0)
        um = 0.1 * np.cos(c * x) * np.cos(c * y) * np.cos(c * z)  # vanishes on |x_i| = 4
        fm = 3 * c * c * um + puncture.source(um, pr.alpha, pr.beta)
        b = pr.mass * fm
        res = lambda u: b - (pr.apply(u) + pr.mass * puncture.source(u, pr.alpha, pr.beta))
        u, rep = newton.newton(res, lambda u, r: pr.linear_solve(u, r, tol=1e-10), np.zeros_like(um), tol=1e-12)
        assert rep["converged"]
        h = rep["history"]
        assert h[-1] / h[-2] < 1e-3 * h[-2] / h[-3] or h[-1] < 1e-13 * h[0]
        errs.append(np.sqrt(np.mean((u - um) ** 2)))
    assert errs[1] < errs[0] / 20


def test_newton_result_independent_of_subdomain_solver():
    grid = _box((2, 2, 2), 4, lower=(-20,) * 3, upper=(20,) * 3)
    pr = solve.PunctureProblem(grid, workloads.BINARY_PUNCTURES)
    u1, r1 = pr.solve(tol=1e-10, linear_tol=1e-4)
    # exact dense linearized solves instead of multigrid-Schwarz FGMRES
    Ad = dg.assemble(pr.graphs[0])

    def exact(u, r):
        D = (pr.mass * puncture.source_deriv(u, pr.alpha, pr.beta)).ravel()
        return np.linalg.solve(Ad + np.diag(D), r.ravel()).reshape(r.shape), {}

    u2, r2 = newton.newton(pr.residual, exact, np.zeros_like(u1), tol=1e-10)
    assert r1["converged"] and r2["converged"]
    assert np.linalg.norm(u1 - u2) <= 1e-9 * np.linalg.norm(u2)


def _linearization(grid, seed):
    """A positive diagonal D = M S'(u) at a seeded state u of the binary-puncture source."""
    pr = solve.PunctureProblem(grid, workloads.BINARY_PUNCTURES)
    u = 0.1 * workloads.uniform_vector(seed, pr.mass.size, 0.0, 1.0).reshape(pr.mass.shape)
    return pr, pr.mass * puncture.source_deriv(u, pr.alpha, pr.beta)


def test_linearized_inverse_smoother_single_element_is_exact():
    """n = 1: the one subdomain is the whole domain, so one step of the per-subdomain linearized
    inverse solves (A + D) u = b exactly (dense solve of the assembled operator)."""
    grid = _box((1, 1, 1), 5, lower=(-4,) * 3, upper=(4,) * 3)
    pr, D = _linearization(grid, 7)
    assert D.min() > 0 and D.max() > 1e-3 * np.abs(dg.assemble(pr.graphs[0])).max()
    lv = pr.schwarz[0]
    b = workloads.uniform_vector(8, D.size, -1.0, 1.0).reshape(D.shape)
    lin = lambda x: dg.apply(pr.graphs[0], x) + D * x
    u = lv.smooth(b, np.zeros_like(b), 1, lin, schwarz.inverse_subdomain_solver(lv, D))
    exact = np.linalg.solve(dg.assemble(pr.graphs[0]) + np.diag(D.ravel()), b.ravel())
    assert np.linalg.norm(u.ravel() - exact) <= 1e-12 * np.linalg.norm(exact)


def test_linearized_inverse_smoother_special_cases():
    """D = 0 gives the Poisson smoother; with D != 0 it equals the GMRES subdomain solver run to
    convergence (enough iterations that the Krylov space holds the exact subdomain solution)."""
    grid = _box((3, 2, 2), 3, lower=(-4,) * 3, upper=(4,) * 3)
    pr, D = _linearization(grid, 9)
    lv = pr.schwarz[0]
    b = workloads.uniform_vector(10, D.size, -1.0, 1.0).reshape(D.shape)
    u0 = workloads.uniform_vector(11, D.size, -1.0, 1.0).reshape(D.shape)
    zero = np.zeros_like(D)
    poisson = lv.smooth(b, u0, 2)
    assert np.linalg.norm(lv.smooth(b, u0, 2, None, schwarz.inverse_subdomain_solver(lv, zero)) - poisson) \
        <= 1e-12 * np.linalg.norm(poisson)
    lin = lambda x: dg.apply(pr.graphs[0], x) + D * x
    inv = lv.smooth(b, u0, 2, lin, schwarz.inverse_subdomain_solver(lv, D))
    gm = lv.smooth(b, u0, 2, lin, schwarz.gmres_subdomain_solver(lv, D, 40))
    assert np.linalg.norm(inv - gm) <= 1e-9 * np.linalg.norm(inv)
    # the linearization term does enter the subdomain solves
    no_d = lv.smooth(b, u0, 2, lin, schwarz.inverse_subdomain_solver(lv, zero))
    assert np.linalg.norm(inv - no_d) > 1e-4 * np.linalg.norm(inv)


def test_newton_with_linearized_inverse_subdomains_matches_default():
    """The nonlinear solution does not depend on the subdomain solver; the exact linearized
    subdomain solves take no more Krylov iterations than 3 GMRES iterations on them."""
    grid = _box((2, 2, 2), 4, lower=(-20,) * 3, upper=(20,) * 3)
    pr = solve.PunctureProblem(grid, workloads.BINARY_PUNCTURES)
    u1, r1 = pr.solve(tol=1e-10, linear_tol=1e-4)
    u2, r2 = pr.solve(tol=1e-10, linear_tol=1e-4, subdomain_solver="inverse")
    assert r1["converged"] and r2["converged"]
    assert np.linalg.norm(u1 - u2) <= 1e-9 * np.linalg.norm(u1)
    its = lambda r: sum(info["iterations"] for info in r["linear_iterations"])
    assert its(r2) <= its(r1)


def test_line_search_backtracks_on_overshoot():
    # scalar problem r(u) = b - atan(u): a full Newton step from u = 3 overshoots
    b = 0.0
    res = lambda u: b - np.arctan(u)
    lin = lambda u, r: (r * (1 + u * u), {})
    u, rep = newton.newton(res, lin, np.array([3.0]), tol=1e-12)
    assert rep["converged"] and rep["line_search_steps"] > 0 and abs(u[0]) < 1e-10


# ---------------------------------------------------------------- puncture data

def _bowen_york_abar(X, punctures):
    """Conformal traceless extrinsic curvature of Bowen-York punctures without spin, summed over the
    punctures, at points X (..., 3)."""
    out = np.zeros(X.shape[:-1] + (3, 3))
    for q in punctures:
        dx = X - np.asarray(q.position)
        r = np.linalg.norm(dx, axis=-1)
        l = dx / r[..., None]
        P = np.asarray(q.momentum)
        Pl = l @ P
        out += 1.5 / r[..., None, None] ** 2 * (np.einsum("i,...j->...ij", P, l) + np.einsum("...i,j->...ij", l, P)
                                                - (np.eye(3) - np.einsum("...i,...j->...ij", l, l)) * Pl[..., None, None])
    return out


def test_bowen_york_curvature_traceless_and_divergence_free():
    p = workloads.BINARY_PUNCTURES
    pts = np.array([[0.3, 0.7, -1.1], [5.0, -2.0, 1.0]])
    eps = 1e-4

    def abar(X):
        return _bowen_york_abar(X, p)

    A = abar(pts)
    assert np.abs(np.trace(A, axis1=-2, axis2=-1)).max() < 1e-15
    div = np.zeros((2, 3))
    for j in range(3):
        e = np.zeros(3)
        e[j] = eps
        div += (abar(pts + e)[..., :, j] - abar(pts - e)[..., :, j]) / (2 * eps)
    assert np.abs(div).max() < 1e-7
    # and the oracle's beta is alpha^7 A_ij A^ij / 8 of this curvature
    alpha, beta = puncture.alpha_beta(pts[:, 0], pts[:, 1], pts[:, 2], p)
    assert np.allclose(beta, alpha**7 * np.einsum("...ij,...ij->...", A, A) / 8, rtol=1e-14)
    r = [np.linalg.norm(pts - np.asarray(q.position), axis=-1) for q in p]
    assert np.allclose(1 / alpha, 0.5 / (2 * r[0]) + 0.5 / (2 * r[1]), rtol=1e-15)


def test_bowen_york_adm_momenta():
    """The curvature carries the momenta it is built from: the surface integrals
    P^i = (1/8 pi) oint A^ij n_j dA and J_i = (1/8 pi) oint eps_ijk x^j A^kl n_l dA over a sphere give
    the linear momentum of the punctures inside it and their orbital angular momentum C x P (the
    3/2 normalisation, which tracelessness and zero divergence leave free, is fixed by this).
    Gauss-Legendre in cos(theta) x uniform in phi; the integrands are smooth on these spheres."""
    p = workloads.BINARY_PUNCTURES
    ct, wt = np.polynomial.legendre.leggauss(48)
    ph = np.arange(96) * (2 * np.pi / 96)
    st = np.sqrt(1 - ct**2)
    n = np.stack([st[:, None] * np.cos(ph)[None, :], st[:, None] * np.sin(ph)[None, :],
                  np.broadcast_to(ct[:, None], (48, 96))], axis=-1)
    dOmega = wt[:, None] * np.full(96, 2 * np.pi / 96)[None, :]

    def integrals(center, R):
        X = np.asarray(center) + R * n
        A = _bowen_york_abar(X, p)
        An = np.einsum("...ij,...j->...i", A, n)
        P = np.einsum("ab,abi->i", dOmega, An) * R**2 / (8 * np.pi)
        J = np.einsum("ab,abi->i", dOmega, np.cross(X, An)) * R**2 / (8 * np.pi)
        return P, J

    # a sphere around each puncture alone: its own momentum
    for q in p:
        P, _ = integrals(q.position, 1.0)
        assert np.allclose(P, q.momentum, atol=1e-12)
    # a sphere around both: total momentum and orbital angular momentum sum_n C_n x P_n
    P, J = integrals((0.0, 0.0, 0.0), 10.0)
    assert np.allclose(P, sum(np.asarray(q.momentum) for q in p), atol=1e-12)
    J_ref = sum(np.cross(q.position, q.momentum) for q in p)
    assert np.allclose(J, J_ref, atol=1e-12)
    assert abs(J_ref[2]) > 0.1  # the binary orbits: a nonzero reference


# ---------------------------------------------------------------- V-cycle and subdomain GMRES, in closed form

def _schwarz_matrix(level: schwarz.SchwarzLevel) -> np.ndarray:
    """M^-1 = sum_S R_S^T W_S A_S^-1 R_S (Eqs. schwarz_subd_problem, schwarz_weighting) as a dense
    matrix, from each subdomain's point list, weights and dense A_S."""
    n = level.grid.n_elements * level.N**3
    Minv = np.zeros((n, n))
    for e, sd in enumerate(level.subdomains):
        g = sd["glob"]
        Minv[np.ix_(g, g)] += sd["weight"][:, None] * np.linalg.inv(level.subdomain_matrix(e))
    return Minv


def _prolongation_matrix(fine, coarse) -> np.ndarray:
    N = fine.N
    nc = coarse.n_elements * N**3
    eye = np.eye(nc).reshape(nc, coarse.n_elements, N, N, N)
    return mg.prolongate(fine, coarse, eye).reshape(nc, -1).T.copy()


@pytest.mark.parametrize("n,levels,pre,post", [((4, 2, 2), 2, 3, 3), ((8, 2, 2), 3, 3, 3), ((8, 2, 2), 3, 2, 1)])
def test_vcycle_equals_multigrid_error_propagation_operator(n, levels, pre, post):
    """Sec. III.C.3 as error propagation (Hackbusch, Multi-Grid Methods, Sec. 2.4/7.1): with the
    Schwarz iteration matrix S_l = I - M_l^-1 A_l, a V-cycle from zero initial guesses is the linear
    map B_l with I - B_l A_l = S_l^post (I - P_l B_{l+1} R_l A_l) S_l^pre, and on the coarsest level
    (presmoothing then postsmoothing from zero) I - B_c A_c = S_c^(pre + post). Evaluated with dense
    matrices, independently of the oracle's sequential step list. The coarsest level has two or more
    elements, so that its Schwarz step is not an exact solve (a dropped coarse postsmooth shows).
    Also pins the multi-step smoother: k steps from u give S^k u + (I - S^k) A^-1 b."""
    N = 2
    grid = _box(n, N)
    pr = solve.Problem(grid, mg_levels=levels, overlap=1, presmooth=pre, postsmooth=post)
    L = len(pr.levels)
    assert L == levels and pr.levels[-1].n_elements >= 2
    A = [dg.assemble(g) for g in pr.graphs]
    Ainv = [np.linalg.inv(a) for a in A]
    S = [np.eye(a.shape[0]) - _schwarz_matrix(s) @ a for s, a in zip(pr.schwarz, A)]
    P = [_prolongation_matrix(pr.levels[l], pr.levels[l + 1]) for l in range(L - 1)]
    mp = np.linalg.matrix_power
    B = (np.eye(A[-1].shape[0]) - mp(S[-1], pre + post)) @ Ainv[-1]
    for l in range(L - 2, -1, -1):
        I = np.eye(A[l].shape[0])
        B = (I - mp(S[l], post) @ (I - P[l] @ B @ P[l].T @ A[l]) @ mp(S[l], pre)) @ Ainv[l]
    for seed in (41, 42):
        r = workloads.uniform_vector(seed, A[0].shape[0]).reshape(-1, N, N, N)
        z = pr.vcycle(r).ravel()
        want = B @ r.ravel()
        assert np.linalg.norm(z - want) <= 1e-12 * np.linalg.norm(want)
    # the smoother itself: k Schwarz steps of the stationary iteration
    b = workloads.uniform_vector(43, A[0].shape[0]).reshape(-1, N, N, N)
    u0 = workloads.uniform_vector(44, A[0].shape[0]).reshape(-1, N, N, N)
    for k in (1, 3):
        got = pr.schwarz[0].smooth(b, u0, k).ravel()
        Sk = mp(S[0], k)
        want = Sk @ u0.ravel() + (np.eye(A[0].shape[0]) - Sk) @ (Ainv[0] @ b.ravel())
        assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


def test_truncated_subdomain_gmres_is_the_krylov_least_squares_minimiser():
    """Sec. III.E's subdomain solver: m right-preconditioned GMRES iterations from zero (Saad,
    Iterative Methods, Sec. 9.3.2) return z = M y with y the minimiser of ||r - A M y|| over the
    Krylov space K_m(A M, r) = span{r, (A M) r, ..., (A M)^(m-1) r}. Built here from the monomial
    basis and a dense least-squares solve on a linearized subdomain operator A_S + D_S with the
    Poisson inverse as M, for m = 1, 2, 3 (none converged: the residual stays well above zero)."""
    grid = _box((3, 2, 2), 3)
    lv = schwarz.SchwarzLevel(grid, 2)
    e = 4  # an interior-ish element with four face neighbours
    A_S = lv.subdomain_matrix(e)
    nS = A_S.shape[0]
    D = 40.0 * workloads.uniform_vector(45, nS, 0.0, 1.0)  # strong diagonal: M is far from exact
    op = lambda z: A_S @ z + D * z
    Minv = np.linalg.inv(A_S)
    r = workloads.uniform_vector(46, nS)
    AM = (A_S + np.diag(D)) @ Minv
    for m in (1, 2, 3):
        W = np.stack([np.linalg.matrix_power(AM, i) @ r for i in range(m)], axis=1)
        c = np.linalg.lstsq(AM @ W, r, rcond=None)[0]
        want = Minv @ (W @ c)
        got = schwarz._gmres_right(op, lambda v: Minv @ v, r, m)
        assert np.linalg.norm(r - op(want)) >= 1e-3 * np.linalg.norm(r)
        assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want), m
