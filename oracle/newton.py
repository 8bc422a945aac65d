"""Newton-Raphson with line-search globalization (Sec. III.A, Eq. linearized).

Oracle code (test infrastructure only). Each step solves dA/du(u) du = b - A(u) to a
relative tolerance, then u <- u + lambda du with lambda = 1 first. Sufficient decrease
(the fraction c of the decrease a linear problem would give):
    ||b - A(u + lambda du)|| <= (1 - c lambda) ||b - A(u)||.
Reading (the paper cites Dennis-Schnabel Alg. 6.1.3 without constants): c = 1e-4 and
backtracking to the minimiser of the quadratic model of ||r(lambda)||^2 / 2, clamped to
[0.1 lambda, 0.5 lambda].
"""
from __future__ import annotations

import numpy as np


def newton(residual, linear_solve, u0, tol=1e-10, max_steps=20, c=1e-4, max_backtracks=10):
    """residual(u) -> b - A(u); linear_solve(u, r) -> du with dA/du(u) du ~= r.
    Stops when ||r|| <= tol * ||r_0||. Returns u and a report."""
    u = np.array(u0, dtype=np.float64, copy=True)
    r = residual(u)
    r0 = np.linalg.norm(r)
    rn = r0
    report = {"steps": 0, "history": [r0], "line_search_steps": 0, "linear_iterations": []}
    if r0 == 0.0:
        report["converged"] = True
        return u, report
    for step in range(max_steps):
        if rn <= tol * r0:
            break
        du, lin_info = linear_solve(u, r)
        report["linear_iterations"].append(lin_info)
        lam = 1.0
        for _ in range(max_backtracks + 1):
            r_new = residual(u + lam * du)
            rn_new = np.linalg.norm(r_new)
            if rn_new <= (1.0 - c * lam) * rn:
                break
            # quadratic model g(l) = |r(l)|^2/2, g(0) = rn^2/2, g'(0) = -rn^2
            g0, g1, dg0 = 0.5 * rn**2, 0.5 * rn_new**2, -(rn**2)
            lam_q = -dg0 * lam**2 / (2.0 * (g1 - g0 - dg0 * lam))
            lam = min(max(lam_q, 0.1 * lam), 0.5 * lam)
            report["line_search_steps"] += 1
        u = u + lam * du
        r, rn = r_new, rn_new
        report["history"].append(rn)
        report["steps"] = step + 1
    report["converged"] = rn <= tol * r0
    return u, report
