"""Pins for the oracle's LGL collocation (Sec. II, Eqs. field_expansion, lagrprod)."""
import math

import numpy as np
import pytest

from oracle import lgl


@pytest.mark.parametrize("N", range(2, 13))
def test_weights_sum_and_endpoints(N):
    w = lgl.lgl_weights(N)
    assert abs(w.sum() - 2.0) < 1e-14
    assert abs(w[0] - 2.0 / (N * (N - 1))) < 1e-14
    assert np.all(w > 0)


@pytest.mark.parametrize("N", range(2, 13))
def test_quadrature_exact_to_degree_2N_minus_3(N):
    x, w = lgl.lgl_nodes(N), lgl.lgl_weights(N)
    for m in range(0, 2 * N - 2):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(w @ x**m - exact) < 1e-13, m
    # and not exact at degree 2N - 2 (LGL is one degree short of Gauss)
    m = 2 * N - 2
    assert abs(w @ x**m - 2.0 / (m + 1)) > 1e-10


def test_closed_form_nodes():
    # N = 3: 0; N = 4: +-1/sqrt(5); N = 5: 0, +-sqrt(3/7); N = 6: +-sqrt(1/3 -+ 2 sqrt(7)/21)
    assert abs(lgl.lgl_nodes(3)[1]) < 1e-16
    assert abs(lgl.lgl_nodes(4)[2] - 1 / math.sqrt(5)) < 1e-15
    assert abs(lgl.lgl_nodes(5)[3] - math.sqrt(3 / 7)) < 1e-15
    x6 = lgl.lgl_nodes(6)
    assert abs(x6[3] - math.sqrt(1 / 3 - 2 * math.sqrt(7) / 21)) < 1e-15
    assert abs(x6[4] - math.sqrt(1 / 3 + 2 * math.sqrt(7) / 21)) < 1e-15
    np.testing.assert_allclose(x6[3:], [0.2852315165, 0.7650553239, 1.0], atol=1e-10)
    np.testing.assert_allclose(lgl.lgl_nodes(8)[4:], [0.2092992179, 0.5917001814, 0.8717401485, 1.0], atol=1e-10)


@pytest.mark.parametrize("N", [2, 3, 5, 8, 10])
def test_diff_matrix_exact_on_polynomials(N):
    x = lgl.lgl_nodes(N)
    D = lgl.diff_matrix(N)
    for m in range(N):
        dx = m * x ** (m - 1) if m else np.zeros(N)
        assert np.abs(D @ x**m - dx).max() < 1e-12 * max(1, m * m)
    # rows of D annihilate constants; D is centro-antisymmetric on the symmetric point set
    assert np.abs(D.sum(axis=1)).max() < 1e-13
    assert np.abs(D + D[::-1, ::-1]).max() < 1e-12


def test_interpolation_reproduces_polynomials():
    N = 6
    t = np.linspace(-1, 1, 17)
    I = lgl.interp_matrix(N, t)
    x = lgl.lgl_nodes(N)
    for m in range(N):
        assert np.abs(I @ x**m - t**m).max() < 1e-13
