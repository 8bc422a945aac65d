"""Puncture-method source terms (Sec. V lists puncture problems among those the solver handles).

Oracle code (test infrastructure only). The paper gives no formulas for this problem; the
reading used here is the textbook Brandt-Bruegmann puncture method with Bowen-York extrinsic
curvature:

    1/alpha = sum_n m_n / (2 r_n)
    A^ij    = sum_n 3 / (2 r_n^2) [P^i l^j + P^j l^i - (delta^ij - l^i l^j) P_k l^k],  l = (x - C_n)/r_n
    beta    = alpha^7 A_ij A^ij / 8

and the equation  -Laplace(u) + S(u) = 0  with  S(u) = -beta (1 + alpha (1 + u))^-7,
S'(u) = 7 alpha beta (1 + alpha (1 + u))^-8.  The paper prints no values for alpha and beta;
they are pinned by physics instead: the curvature beta is built from is traceless and
divergence-free and carries, through its surface integrals, the linear and orbital angular
momenta of the punctures, and 1/alpha is checked against its closed form.
"""
from __future__ import annotations

import numpy as np


def alpha_beta(x, y, z, punctures):
    X = np.stack([x, y, z], axis=-1)
    inv_alpha = np.zeros(x.shape)
    Abar = np.zeros(x.shape + (3, 3))
    eye = np.eye(3)
    for p in punctures:
        dx = X - np.asarray(p.position, dtype=np.float64)
        r = np.sqrt(np.sum(dx * dx, axis=-1))
        l = dx / r[..., None]
        P = np.asarray(p.momentum, dtype=np.float64)
        Pl = np.einsum("k,...k->...", P, l)
        inv_alpha += p.mass / (2.0 * r)
        t = (np.einsum("i,...j->...ij", P, l) + np.einsum("...i,j->...ij", l, P)
             - (eye - np.einsum("...i,...j->...ij", l, l)) * Pl[..., None, None])
        Abar += 1.5 / (r * r)[..., None, None] * t
    alpha = 1.0 / inv_alpha
    beta = alpha**7 * np.einsum("...ij,...ij->...", Abar, Abar) / 8.0
    return alpha, beta


def source(u, alpha, beta):
    return -beta * (1.0 + alpha * (1.0 + u)) ** -7


def source_deriv(u, alpha, beta):
    return 7.0 * alpha * beta * (1.0 + alpha * (1.0 + u)) ** -8
