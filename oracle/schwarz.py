"""Additive Schwarz smoother of Sec. III.D with the subdomain solvers of Sec. III.E.

Oracle code (test infrastructure only).

Subdomain geometry (Sec. III.D.1): S_k is element k's N^3 points plus, for every face
neighbour, that neighbour's first N_overlap point layers counted from the shared face
(the neighbour's face points included, its far face never: N_overlap <= N - 1). No edge
or corner neighbours.

Subdomain operator (Eq. schwarz_subd_problem): A_S = R_S A R_S^T, evaluated as the DG
operator on the patch (central element + face neighbours) with zero data outside S.

Weights (Eqs. schwarz_weighting, schwarz_weight_prod, schwarz_weight_function): the
quintic smoothstep phi, the 1-D w(xi) = (phi((xi+1)/delta) - phi((xi-1)/delta))/2 with
delta the logical distance from the element face to the first point outside the overlap,
W = prod_i w(xi^i). Readings where the paper is silent:
  * edges and corners: prod_i (a_i + b_i^+ + b_i^-) = 1 is expanded per node (a_i = w(xi_i),
    b_i^+- = w(xi_i -+ 2)); a term with m >= 1 neighbour factors is split equally among
    those m face neighbours' subdomains, the term without one stays with the element's own;
  * external boundaries: a side without a neighbour replaces its phi term by +-1, so a_i
    absorbs the missing b_i and conservation stays exact.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import dg, lgl


def phi(x):
    """Second-order (quintic) smoothstep on [-1, 1], sign(x) outside."""
    x = np.asarray(x, dtype=np.float64)
    inside = (15.0 * x - 10.0 * x**3 + 3.0 * x**5) / 8.0
    return np.where(np.abs(x) <= 1.0, inside, np.sign(x))


def w1d(xi, delta):
    """Eq. schwarz_weight_function."""
    return 0.5 * (phi((xi + 1.0) / delta) - phi((xi - 1.0) / delta))


def overlap_width(N: int, overlap: int) -> float:
    """delta: distance from the element boundary (xi = 1) to the first point outside the overlap,
    in the central element's logical units (equal element sizes): 1 + x_{N_overlap} (0-based)."""
    x = lgl.lgl_nodes(N)
    return 1.0 + x[overlap] if overlap < N else 2.0


def weight_shares(N: int, overlap: int, has_lo, has_hi):
    """For every node of one element: the weight each overlapping subdomain gives it.

    Returns an array shares[k, j, i, s] for s = 0 (the element's own subdomain) and
    s = 1 + f for the subdomain centred on the face neighbour across face f = 2 d + side.
    """
    x = lgl.lgl_nodes(N)
    delta = overlap_width(N, overlap)
    a = np.zeros((3, N))
    bp = np.zeros((3, N))
    bm = np.zeros((3, N))
    for d in range(3):
        lo = phi((x + 1.0) / delta) if has_lo[d] else np.ones(N)
        hi = phi((x - 1.0) / delta) if has_hi[d] else -np.ones(N)
        a[d] = 0.5 * (lo - hi)
        bp[d] = w1d(x - 2.0, delta) if has_hi[d] else 0.0
        bm[d] = w1d(x + 2.0, delta) if has_lo[d] else 0.0
    shares = np.zeros((N, N, N, 7))
    for k, j, i in itertools.product(range(N), repeat=3):
        idx = (i, j, k)  # node index along x, y, z
        for choice in itertools.product((0, 1, 2), repeat=3):  # per dim: a, b^-, b^+
            term = 1.0
            owners = []
            for d, c in enumerate(choice):
                if c == 0:
                    term *= a[d][idx[d]]
                elif c == 1:
                    term *= bm[d][idx[d]]
                    owners.append(1 + 2 * d)
                else:
                    term *= bp[d][idx[d]]
                    owners.append(1 + 2 * d + 1)
            if not owners:
                shares[k, j, i, 0] += term
            else:
                for o in owners:
                    shares[k, j, i, o] += term / len(owners)
    return shares


class SchwarzLevel:
    """Subdomains, weights and subdomain operators of one grid."""

    def __init__(self, grid: dg.BoxGrid, overlap: int):
        if not 1 <= overlap <= grid.N - 1:
            raise ValueError("need 1 <= N_overlap <= N - 1")
        self.grid = grid
        self.graph = grid.graph()
        self.overlap = overlap
        N = grid.N
        E = grid.n_elements
        self.N = N
        # per element: which face neighbours exist, and the weight shares of its nodes
        nbr = self.graph.nbr
        self.shares = np.zeros((E, N, N, N, 7))
        cache = {}
        for e in range(E):
            has_lo = tuple(nbr[e, 2 * d] >= 0 for d in range(3))
            has_hi = tuple(nbr[e, 2 * d + 1] >= 0 for d in range(3))
            key = (has_lo, has_hi)
            if key not in cache:
                cache[key] = weight_shares(N, overlap, has_lo, has_hi)
            self.shares[e] = cache[key]
        self.subdomains = [self._subdomain(e) for e in range(E)]
        self.classes = {}
        for e, sd in enumerate(self.subdomains):
            self.classes.setdefault(sd["key"], []).append(e)
        self._A_S = {}

    def _subdomain(self, e):
        N, ov = self.N, self.overlap
        nbr = self.graph.nbr
        slots = [e]
        for f in range(6):
            if nbr[e, f] >= 0:
                slots.append(int(nbr[e, f]))
        slot_of = {g: s for s, g in enumerate(slots)}
        # patch graph: neighbours outside the patch carry zero data
        pn = np.full((len(slots), 6), dg.ZERO, dtype=np.int64)
        for s, g in enumerate(slots):
            for f in range(6):
                q = nbr[g, f]
                if q in (dg.EXTERNAL, dg.NEUMANN):
                    pn[s, f] = q
                elif q in slot_of:
                    pn[s, f] = slot_of[q]
        patch = self.graph.subgraph(slots, pn)
        # points of S: all of the centre, then N_overlap layers of each face neighbour
        glob, local, weight = [], [], []
        kk, jj, ii = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
        allnodes = np.stack([kk.ravel(), jj.ravel(), ii.ravel()], axis=1)
        for k, j, i in allnodes:
            glob.append(e * N**3 + k * N * N + j * N + i)
            local.append(k * N * N + j * N + i)
            weight.append(self.shares[e, k, j, i, 0])
        s = 1
        for f in range(6):
            q = nbr[e, f]
            if q < 0:
                continue
            d, side = divmod(f, 2)
            # the neighbour sees this element across its face on the opposite side
            f_back = 2 * d + (1 - side)
            for k, j, i in allnodes:
                along = (i, j, k)[d]
                depth = along if side == 1 else N - 1 - along
                if depth < ov:
                    glob.append(q * N**3 + k * N * N + j * N + i)
                    local.append(s * N**3 + k * N * N + j * N + i)
                    weight.append(self.shares[q, k, j, i, 1 + f_back])
            s += 1
        key = (tuple(map(tuple, pn.tolist())),)
        if self.graph.per_element:  # curved elements: every subdomain has its own operator
            key = key + (e,)
        return {
            "slots": slots,
            "patch": patch,
            "glob": np.array(glob, dtype=np.int64),
            "local": np.array(local, dtype=np.int64),
            "weight": np.array(weight),
            "key": key,
        }

    def subdomain_matrix(self, e: int) -> np.ndarray:
        """A_S = R_S A R_S^T, column by column from the matrix-free patch apply."""
        sd = self.subdomains[e]
        key = sd["key"]
        if key in self._A_S:
            return self._A_S[key]
        N = self.N
        P = len(sd["slots"])
        nS = len(sd["local"])
        cols = np.zeros((nS, P * N**3))
        cols[np.arange(nS), sd["local"]] = 1.0  # R_S^T e_c
        Acols = dg.apply(sd["patch"], cols.reshape(nS, P, N, N, N)).reshape(nS, P * N**3)
        A_S = Acols[:, sd["local"]].T.copy()  # R_S (A R_S^T e_c) as column c
        self._A_S[key] = A_S
        return A_S

    def smooth(self, b, u, iterations, operator=None, subdomain_solve=None):
        """Schwarz iterations (Sec. III.D.5): r = b - A u; r_S = R_S r; A_S du_S = r_S;
        u <- u + sum_S R_S^T (w_S du_S)."""
        if operator is None:
            operator = lambda x: dg.apply(self.graph, x)
        u = np.array(u, dtype=np.float64, copy=True)
        shape = u.shape
        for _ in range(iterations):
            r = (b - operator(u)).ravel()
            du_total = np.zeros(r.size)
            for key, members in self.classes.items():
                A_S = self.subdomain_matrix(members[0])
                idx = np.stack([self.subdomains[e]["glob"] for e in members])  # (m, nS)
                wts = np.stack([self.subdomains[e]["weight"] for e in members])
                rS = r[idx]
                if subdomain_solve is None:
                    duS = np.linalg.solve(A_S, rS.T).T
                else:
                    duS = subdomain_solve(A_S, rS, members)
                np.add.at(du_total, idx.ravel(), (wts * duS).ravel())
            u = u + du_total.reshape(shape)
        return u


def gmres_subdomain_solver(level: SchwarzLevel, diag: np.ndarray, iterations: int = 3):
    """Subdomain solver of Sec. III.E for a linearized operator A_S + D_S (D_S diagonal):
    GMRES from a zero guess, a fixed number of iterations, right-preconditioned by the
    explicit inverse of the Poisson subdomain matrix A_S (the Laplacian approximation,
    Eq. lapl_approx, solved by the explicit-inverse solver)."""
    dflat = diag.ravel()

    def solve(A_S, rS, members):
        out = np.zeros_like(rS)
        A_S_inv = np.linalg.inv(A_S)
        for m, e in enumerate(members):
            D = dflat[level.subdomains[e]["glob"]]
            op = lambda z: A_S @ z + D * z
            out[m] = _gmres_right(op, lambda v: A_S_inv @ v, rS[m], iterations)
        return out

    return solve


def inverse_subdomain_solver(level: SchwarzLevel, diag: np.ndarray):
    """Subdomain solver for a linearized operator A_S + D_S (D_S diagonal) by the explicit inverse
    of every subdomain's own linearized matrix: Sec. III.E's explicit-inverse solver applied to the
    full linearized operator instead of its Laplacian approximation. The matrices depend on the
    linearization point, so they are formed afresh for every linearization: one solver object
    per linearization, which keeps each subdomain's inverse after its first use."""
    dflat = diag.ravel()
    inverses = {}  # per subdomain: formed on first use, kept for this linearization

    def solve(A_S, rS, members):
        out = np.zeros_like(rS)
        for m, e in enumerate(members):
            if e not in inverses:
                D = dflat[level.subdomains[e]["glob"]]
                inverses[e] = np.linalg.inv(A_S + np.diag(D))
            out[m] = inverses[e] @ rS[m]
        return out

    return solve


def _gmres_right(op, prec, r, iterations):
    """Right-preconditioned GMRES with a zero initial guess (Saad Alg. 9.5), fixed iterations."""
    beta = np.linalg.norm(r)
    n = r.size
    if beta == 0.0:
        return np.zeros(n)
    V = np.zeros((iterations + 1, n))
    Z = np.zeros((iterations, n))
    H = np.zeros((iterations + 1, iterations))
    V[0] = r / beta
    k = 0
    for j in range(iterations):
        Z[j] = prec(V[j])
        w = op(Z[j])
        for i in range(j + 1):
            H[i, j] = w @ V[i]
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        k = j + 1
        if H[j + 1, j] == 0.0:
            break
        V[j + 1] = w / H[j + 1, j]
    e1 = np.zeros(k + 1)
    e1[0] = beta
    y = np.linalg.lstsq(H[: k + 1, :k], e1, rcond=None)[0]
    return Z[:k].T @ y
