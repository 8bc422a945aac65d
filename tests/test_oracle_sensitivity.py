"""The oracle's pins are sensitive: each case below plants one plausible mistake in the oracle
(monkeypatched, on the CPU, for the duration of the case) and checks that a pin of
test_oracle_lgl / test_oracle_dg / test_oracle_solver / test_oracle_curved then fails. A pin that still passed with
the mistake in place would not be pinning that part of the oracle."""
import numpy as np
import pytest

import test_oracle_curved as tcur
import test_oracle_dg as tdg
import test_oracle_lgl as tlgl
import test_oracle_solver as tsol
from oracle import curved, dg, lgl, mg, puncture, schwarz

_FAIL = (AssertionError, np.linalg.LinAlgError)


def _fails(pin, *args):
    with pytest.raises(_FAIL):
        pin(*args)


def test_pins_pass_without_a_planted_mistake():
    """The same pins, unpatched, pass (so the failures below come from the plants)."""
    tlgl.test_diff_matrix_exact_on_polynomials(5)
    tlgl.test_weights_sum_and_endpoints(5)
    tlgl.test_closed_form_nodes()
    tdg.test_polynomial_consistency()
    tdg.test_strong_form_equals_sipg_bilinear_form((2, 2, 1), 3)
    tsol.test_overlap_width_values()
    tsol.test_smoothstep_and_weight_function_closed_forms()
    tsol.test_face_neighbour_weight_is_product_away_from_edges()
    tsol.test_prolongation_exact_on_coarse_polynomials((2, 2, 2))
    tsol.test_restriction_is_transpose_of_prolongation()
    tsol.test_bowen_york_curvature_traceless_and_divergence_free()


def test_transposed_differentiation_matrix_is_caught(monkeypatch):
    orig = lgl.diff_matrix
    monkeypatch.setattr(lgl, "diff_matrix", lambda N: orig(N).T.copy())
    _fails(tlgl.test_diff_matrix_exact_on_polynomials, 5)
    _fails(tdg.test_polynomial_consistency)


def test_uniform_quadrature_weights_are_caught(monkeypatch):
    # (A u = M (-Laplace u) holds for any diagonal M, so the operator pins cannot see the weights;
    # the quadrature pins do)
    monkeypatch.setattr(lgl, "lgl_weights", lambda N: np.full(N, 2.0 / N))
    _fails(tlgl.test_weights_sum_and_endpoints, 5)
    _fails(tlgl.test_quadrature_exact_to_degree_2N_minus_3, 5)


def test_equispaced_nodes_are_caught(monkeypatch):
    monkeypatch.setattr(lgl, "lgl_nodes", lambda N: np.linspace(-1.0, 1.0, N))
    _fails(tlgl.test_closed_form_nodes)


def test_trace_from_the_opposite_face_is_caught(monkeypatch):
    orig = dg._face
    monkeypatch.setattr(dg, "_face", lambda a, d, side, N: orig(a, d, 1 - side, N))
    _fails(tdg.test_strong_form_equals_sipg_bilinear_form, (2, 2, 1), 3)


def test_lift_onto_the_opposite_face_is_caught(monkeypatch):
    orig = dg._lift_to_volume
    monkeypatch.setattr(dg, "_lift_to_volume", lambda fv, d, side, N: orig(fv, d, 1 - side, N))
    _fails(tdg.test_strong_form_equals_sipg_bilinear_form, (2, 2, 1), 3)


def test_overlap_width_one_layer_short_is_caught(monkeypatch):
    monkeypatch.setattr(schwarz, "overlap_width",
                        lambda N, ov: 1.0 + lgl.lgl_nodes(N)[ov - 1] if ov < N else 2.0)
    _fails(tsol.test_overlap_width_values)


def test_cubic_smoothstep_is_caught(monkeypatch):
    def cubic(x):
        x = np.asarray(x, dtype=np.float64)
        t = 0.5 * (x + 1.0)
        return np.where(np.abs(x) <= 1.0, 2.0 * (3 * t**2 - 2 * t**3) - 1.0, np.sign(x))

    monkeypatch.setattr(schwarz, "phi", cubic)
    _fails(tsol.test_smoothstep_and_weight_function_closed_forms)


def test_weights_kept_by_the_own_subdomain_are_caught(monkeypatch):
    def own_only(N, overlap, has_lo, has_hi):
        sh = np.zeros((N, N, N, 7))
        sh[..., 0] = 1.0
        return sh

    monkeypatch.setattr(schwarz, "weight_shares", own_only)
    _fails(tsol.test_face_neighbour_weight_is_product_away_from_edges)


def test_swapped_child_halves_in_prolongation_are_caught(monkeypatch):
    orig = mg._interp

    def swapped(N):
        I = orig(N)
        return {0: I[1], 1: I[0], None: I[None]}

    monkeypatch.setattr(mg, "_interp", swapped)
    _fails(tsol.test_prolongation_exact_on_coarse_polynomials, (2, 2, 2))


def test_scaled_restriction_is_caught(monkeypatch):
    orig = mg.restrict
    monkeypatch.setattr(mg, "restrict", lambda fine, coarse, rf: 0.125 * orig(fine, coarse, rf))
    _fails(tsol.test_restriction_is_transpose_of_prolongation)


def test_bowen_york_normalisation_is_caught(monkeypatch):
    """beta built from a curvature with prefactor 1 instead of 3/2 (beta scales with its square)."""
    orig = puncture.alpha_beta

    def wrong(x, y, z, punctures):
        a, b = orig(x, y, z, punctures)
        return a, b * (1.0 / 1.5) ** 2

    monkeypatch.setattr(puncture, "alpha_beta", wrong)
    _fails(tsol.test_bowen_york_curvature_traceless_and_divergence_free)


# ---------------------------------------------------------------- curved elements


def test_curved_pins_pass_without_a_planted_mistake():
    tcur.test_rigid_motion_leaves_operator_unchanged()
    tcur.test_identity_map_reduces_to_affine_operator((2, 2, 1), 4, (False,) * 6)


def test_transposed_inverse_jacobian_is_caught(monkeypatch):
    """G^j_i = dxi^j/dx^i stored as dxi^i/dx^j: invisible on axis-aligned boxes, not under rotation."""
    orig = curved.metric

    def transposed(N, x, y, z):
        J, G = orig(N, x, y, z)
        return J, np.swapaxes(G, 1, 2).copy()

    monkeypatch.setattr(curved, "metric", transposed)
    tcur.test_identity_map_reduces_to_affine_operator((2, 2, 1), 4, (False,) * 6)
    _fails(tcur.test_rigid_motion_leaves_operator_unchanged)


def test_face_size_without_its_factor_two_is_caught(monkeypatch):
    """h = 1 / |G^d| instead of 2 / |G^d| doubles the penalty against the affine operator."""
    orig = curved.face_size
    monkeypatch.setattr(curved, "face_size", lambda N, J, G, d, side: 0.5 * orig(N, J, G, d, side))
    _fails(tcur.test_identity_map_reduces_to_affine_operator, (2, 2, 1), 4, (False,) * 6)


# ---------------------------------------------------------------- V-cycle step order, subdomain GMRES


def _vcycle_planted(mistake):
    """The V-cycle of Sec. III.C.3 with one planted mistake."""

    def vcycle(levels, smoothers, b0, presmooth=3, postsmooth=3, operators=None):
        L = len(levels)
        if operators is None:
            graphs = [g.graph() for g in levels]
            operators = [lambda u, gr=gr: dg.apply(gr, u) for gr in graphs]
        b, u = [None] * L, [None] * L
        b[0] = b0
        for l in range(L - 1):
            u[l] = smoothers[l](b[l], np.zeros_like(b[l]), presmooth)
            r = b[l] - operators[l](u[l])
            b[l + 1] = mg.restrict(levels[l], levels[l + 1], r)
        start = b[L - 1].copy() if mistake == "coarse_guess_b" else np.zeros_like(b[L - 1])
        u[L - 1] = smoothers[L - 1](b[L - 1], start, presmooth)
        if mistake != "no_coarse_postsmooth":
            u[L - 1] = smoothers[L - 1](b[L - 1], u[L - 1], postsmooth)
        for l in range(L - 2, -1, -1):
            if mistake == "smooth_before_correction":
                u[l] = smoothers[l](b[l], u[l], postsmooth)
                u[l] = u[l] + mg.prolongate(levels[l], levels[l + 1], u[l + 1])
            else:
                u[l] = u[l] + mg.prolongate(levels[l], levels[l + 1], u[l + 1])
                u[l] = smoothers[l](b[l], u[l], postsmooth)
        return u[0]

    return vcycle


def test_vcycle_pin_passes_with_the_unplanted_copy(monkeypatch):
    monkeypatch.setattr(mg, "vcycle", _vcycle_planted(None))
    tsol.test_vcycle_equals_multigrid_error_propagation_operator((8, 2, 2), 3, 3, 3)


# (a wrong coarse initial guess decays as S_c^(pre + post); with 3 + 3 steps on a two-element coarse
# level it falls below rounding, so that plant runs with 2 + 1 steps)
@pytest.mark.parametrize("mistake,case", [("no_coarse_postsmooth", ((4, 2, 2), 2, 3, 3)),
                                          ("coarse_guess_b", ((8, 2, 2), 3, 2, 1)),
                                          ("smooth_before_correction", ((4, 2, 2), 2, 3, 3))])
def test_vcycle_step_order_mistakes_are_caught(monkeypatch, mistake, case):
    monkeypatch.setattr(mg, "vcycle", _vcycle_planted(mistake))
    _fails(tsol.test_vcycle_equals_multigrid_error_propagation_operator, *case)


def test_left_preconditioned_subdomain_gmres_is_caught(monkeypatch):
    """GMRES minimising ||M (r - A z)|| (left preconditioning) instead of ||r - A z||."""

    def left(op, prec, r, iterations):
        Mop = lambda z: prec(op(z))
        Mr = prec(r)
        beta = np.linalg.norm(Mr)
        V = [Mr / beta]
        H = np.zeros((iterations + 1, iterations))
        for j in range(iterations):
            w = Mop(V[j])
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j])
        e1 = np.zeros(iterations + 1)
        e1[0] = beta
        y = np.linalg.lstsq(H, e1, rcond=None)[0]
        return np.stack(V[:iterations], axis=1) @ y

    monkeypatch.setattr(schwarz, "_gmres_right", left)
    _fails(tsol.test_truncated_subdomain_gmres_is_the_krylov_least_squares_minimiser)


def test_galerkin_instead_of_least_squares_subdomain_step_is_caught(monkeypatch):
    """The square Hessenberg system (FOM, a Galerkin condition) solved in place of the least-squares
    problem of GMRES."""
    orig_lstsq = np.linalg.lstsq

    def fom(op, prec, r, iterations):
        def square(H, e1, rcond=None):
            k = H.shape[1]
            return (np.linalg.solve(H[:k, :k], e1[:k]),)

        np.linalg.lstsq = square
        try:
            return schwarz.__dict__["_gmres_right_orig"](op, prec, r, iterations)
        finally:
            np.linalg.lstsq = orig_lstsq

    monkeypatch.setitem(schwarz.__dict__, "_gmres_right_orig", schwarz._gmres_right)
    monkeypatch.setattr(schwarz, "_gmres_right", fom)
    _fails(tsol.test_truncated_subdomain_gmres_is_the_krylov_least_squares_minimiser)
