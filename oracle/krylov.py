"""Flexible GMRES (Sec. III.B; Saad, Iterative Methods, Alg. 9.6).

Oracle code (test infrastructure only). Right-preconditioned, flexible (the preconditioner
may change between iterations), Arnoldi with modified Gram-Schmidt (one inner product per
previous basis vector: the "k reductions in iteration k"), no restart. The least-squares
problem min ||beta e1 - H y|| is solved directly at every iteration to monitor the residual;
at exit the true residual ||b - A x|| is recomputed. Norms are Euclidean over all nodal values.
"""
from __future__ import annotations

import numpy as np


def fgmres(op, b, x0=None, precond=None, tol=1e-10, max_iter=200, rel_to="r0", callback=None):
    """Solve op(x) = b. Stops when ||b - A x_k|| <= tol * ||b - A x_0|| (rel_to="r0") or
    tol * ||b|| (rel_to="b"). Returns x, info with iterations, residual history and the
    orthonormality defect of the Arnoldi basis."""
    shape = b.shape
    bf = b.ravel()
    x = np.zeros_like(bf) if x0 is None else np.asarray(x0, dtype=np.float64).ravel().copy()
    A = lambda v: op(v.reshape(shape)).ravel()
    M = (lambda v: v) if precond is None else (lambda v: precond(v.reshape(shape)).ravel())
    r0 = bf - A(x)
    beta = np.linalg.norm(r0)
    ref = beta if rel_to == "r0" else np.linalg.norm(bf)
    history = [beta]
    info = {"iterations": 0, "history": history, "converged": beta <= tol * ref}
    if beta == 0.0 or info["converged"]:
        info["true_residual"] = beta
        return x.reshape(shape), info
    n = bf.size
    V = [r0 / beta]
    Z = []
    H = np.zeros((max_iter + 1, max_iter))
    y = None
    for j in range(max_iter):
        z = M(V[j])  # flexible: keep the preconditioned vector
        Z.append(z)
        w = A(z)
        for i in range(j + 1):  # modified Gram-Schmidt
            H[i, j] = w @ V[i]
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        e1 = np.zeros(j + 2)
        e1[0] = beta
        y, *_ = np.linalg.lstsq(H[: j + 2, : j + 1], e1, rcond=None)
        res = np.linalg.norm(e1 - H[: j + 2, : j + 1] @ y)
        history.append(res)
        info["iterations"] = j + 1
        if callback is not None:
            callback(j + 1, res)
        if res <= tol * ref or H[j + 1, j] == 0.0:
            break
        V.append(w / H[j + 1, j])
    x = x + np.stack(Z, axis=1) @ y
    Vm = np.stack(V, axis=1)
    info["orthonormality"] = np.abs(Vm.T @ Vm - np.eye(Vm.shape[1])).max()
    info["true_residual"] = np.linalg.norm(bf - A(x))
    info["converged"] = info["true_residual"] <= tol * ref * (1 + 1e-6) or history[-1] <= tol * ref
    info["r0"] = beta
    return x.reshape(shape), info


def fcg(op, b, x0=None, precond=None, tol=1e-10, max_iter=400, rel_to="r0", keep_directions=False):
    """Flexible conjugate gradients for symmetric positive definite op (the alternative to FGMRES
    for the SPD Poisson problem that Sec. III.B names: one search direction instead of a growing
    basis). Each new direction is the preconditioned residual made A-orthogonal to the previous
    direction (the flexible variant with one stored direction, so a preconditioner that is not
    exactly symmetric or changes between iterations is tolerated):
        z = M r,  p = z - (z.q_old / p_old.q_old) p_old,  q = A p,
        alpha = (p.r) / (p.q),  x += alpha p,  r -= alpha q.
    Stops when ||r|| <= tol * ||b - A x0|| (rel_to="r0") or tol * ||b||; the true residual is
    recomputed at exit. With the identity preconditioner this is the conjugate gradient method."""
    shape = b.shape
    bf = b.ravel()
    x = np.zeros_like(bf) if x0 is None else np.asarray(x0, dtype=np.float64).ravel().copy()
    A = lambda v: op(v.reshape(shape)).ravel()
    M = (lambda v: v) if precond is None else (lambda v: precond(v.reshape(shape)).ravel())
    r = bf - A(x)
    r0 = np.linalg.norm(r)
    ref = r0 if rel_to == "r0" else np.linalg.norm(bf)
    history = [r0]
    info = {"iterations": 0, "history": history, "r0": r0, "directions": []}  # (p, A p) if kept
    p = q = None
    res = r0
    for k in range(max_iter):
        if res <= tol * ref or res == 0.0:
            break
        z = M(r)
        if p is None:
            p = z.copy()
        else:
            p = z - (z @ q) / (p @ q) * p
        q = A(p)
        alpha = (p @ r) / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        res = np.linalg.norm(r)
        history.append(res)
        info["iterations"] = k + 1
        if keep_directions:
            info["directions"].append((p, q))
    info["true_residual"] = np.linalg.norm(bf - A(x))
    info["converged"] = info["true_residual"] <= tol * ref * (1 + 1e-6)
    return x.reshape(shape), info
