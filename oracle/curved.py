"""Strong-form DG operator of Sec. II for -div(K grad u) = f on curved (mapped) hexahedral elements,
with a positive scalar coefficient field K (K = 1: the Poisson operator).

Oracle code (test infrastructure only).

Each element carries the map x(xi) from its reference cube, given isoparametrically by the
physical coordinates of its N^3 LGL nodes (the map is the degree N-1 Lagrange interpolant of
those coordinates). With the Jacobian Jac^i_j = dx^i/dxi^j (from the logical derivative of the
nodal coordinates), its determinant J and inverse G^j_i = dxi^j/dx^i at the nodes, the
quadrature of Eqs. massmat, stiffmat and liftop (flat metric, sqrt g = 1) becomes

    M_pp     = w_p J_p                                   (LGL collocation, diagonal)
    (MD_i)_pq = w_p J_p G^j_i(p) Dhat_j,pq               (chain rule at the node)
    ML       = w_a w_b J^f on face nodes,  J^f = J |G^d|   (surface Jacobian, Nanson's relation)

and the operator is Eqs. dg_op_auxvars and dg_op_primal with the fluxes F_v^i_j = u delta^i_j and
F_u^i = K v^i and the flux of Eq. numflux:

    v_i  = G^j_i Dhat_j u + L (n_i (u* - u))
    A u  = -M G^j_i Dhat_j (K v^i) - ML ((n.F_u)* - K n.v)
    (n.F_u)* = (K n.grad u + K^ext n.grad u^ext) / 2 - sigma (K u - K^ext u^ext)

Readings where the paper is silent:
  * the unit normal at a face node is the element's own, n_i = s G^d_i / |G^d|, and the
    exterior normal is its negative (the paper's n^ext = -n^int);
  * h in the penalty (Eq. penalty) is the element size normal to the face at each face node,
    h = 2 J / J^f = 2 / |G^d| (the element width for affine elements), and sigma takes the
    smaller of the two sides' values at the node; external faces use the interior value;
  * the coarse multigrid levels inherit the geometry of the fine one: a coarse element's nodes
    are placed on the fine elements' interpolated map (the coarse map interpolates the fine one),
    and the coefficient K is interpolated the same way;
  * on a boundary face the coefficient of the exterior state is the interior one.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import dg, lgl


def metric(N: int, x, y, z):
    """J (E, N, N, N) and G (E, 3, 3, N, N, N) with G[:, j, i] = dxi^j/dx^i, from the nodal
    coordinates of the isoparametric map."""
    Dhat = lgl.diff_matrix(N)
    X = (np.asarray(x, float), np.asarray(y, float), np.asarray(z, float))
    jac = np.empty(X[0].shape[:1] + (3, 3) + X[0].shape[1:])
    for i in range(3):
        for j in range(3):
            jac[:, i, j] = dg._deriv(X[i], j, Dhat)  # dx^i / dxi^j
    jm = np.moveaxis(jac, (1, 2), (-2, -1))  # (E, k, j, i, 3, 3)
    J = np.linalg.det(jm)
    G = np.moveaxis(np.linalg.inv(jm), (-2, -1), (1, 2))
    return J, G


@dataclasses.dataclass
class CurvedGraph:
    """Elements of one order N with their face connectivity and nodal metric.

    nbr[e, f]       exterior element, dg.EXTERNAL, dg.NEUMANN or dg.ZERO
    K[e]            coefficient at the nodes
    J[e]            Jacobian determinant at the nodes
    G[e, j, i]      dxi^j / dx^i at the nodes
    hf_ext[e, f]    the exterior element's normal size at the face nodes (the interior's at
                    external faces), shaped (E, 6, N, N) in the face layout of dg._face
    """

    N: int
    penalty: float
    nbr: np.ndarray
    J: np.ndarray
    G: np.ndarray
    hf_ext: np.ndarray
    K: np.ndarray = None

    def __post_init__(self):
        if self.K is None:
            self.K = np.ones_like(self.J)

    @property
    def n_elements(self) -> int:
        return self.J.shape[0]

    per_element = True  # operators differ between elements with the same neighbour pattern

    def subgraph(self, slots, pn):
        return CurvedGraph(self.N, self.penalty, pn, self.J[slots], self.G[slots], self.hf_ext[slots], self.K[slots])

    def mass(self):
        w = lgl.lgl_weights(self.N)
        return self.J * (w[:, None, None] * w[None, :, None] * w[None, None, :])

    def apply_operator(self, u):
        return apply(self, u)


def face_size(N, J, G, d, side):
    """h = 2 / |G^d| at the nodes of face (d, side), (E, N, N)."""
    Gd = np.stack([dg._face(G[:, d, i], d, side, N) for i in range(3)])
    return 2.0 / np.sqrt((Gd**2).sum(axis=0))


def make_graph(N, penalty, nbr, J, G, K=None) -> CurvedGraph:
    E = J.shape[0]
    hf_ext = np.zeros((E, 6, N, N))
    for f in range(6):
        d, side = divmod(f, 2)
        own = face_size(N, J, G, d, side)
        other = face_size(N, J, G, d, 1 - side)  # every element's opposite face
        has = nbr[:, f] >= 0
        hf_ext[:, f] = np.where(has[:, None, None], other[np.where(has, nbr[:, f], 0)], own)
    return CurvedGraph(N, penalty, nbr, J, G, hf_ext, K)


def apply(graph: CurvedGraph, u: np.ndarray) -> np.ndarray:
    """A u for nodal data u[..., E, N, N, N] on curved elements (homogeneous boundary data)."""
    K = graph.K
    N, E = graph.N, graph.n_elements
    u = np.asarray(u, dtype=np.float64)
    assert u.shape[-4:] == (E, N, N, N), u.shape
    w = lgl.lgl_weights(N)
    Dhat = lgl.diff_matrix(N)
    W3 = w[:, None, None] * w[None, :, None] * w[None, None, :]
    Mdiag = graph.J * W3
    G = graph.G
    # local gradients (chain rule at the node): grad_i u = G^j_i Dhat_j u
    du = [dg._deriv(u, j, Dhat) for j in range(3)]
    grad = [sum(G[:, j, i] * du[j] for j in range(3)) for i in range(3)]
    v = [g.copy() for g in grad]

    prim_face = []
    for f in range(6):
        d, side = divmod(f, 2)
        s = 1.0 if side else -1.0
        nbr = graph.nbr[:, f]
        has = nbr >= 0
        nb = np.where(has, nbr, 0)
        mask = has.astype(np.float64)[:, None, None]
        ext_bc = (nbr == dg.EXTERNAL)[:, None, None]
        ext_neu = (nbr == dg.NEUMANN)[:, None, None]

        Gd = [dg._face(G[:, d, i], d, side, N) for i in range(3)]
        norm = np.sqrt(sum(g * g for g in Gd))
        n = [s * g / norm for g in Gd]  # unit outward normal one-form
        Jf = dg._face(graph.J, d, side, N) * norm  # surface Jacobian
        Bf = Jf * (w[:, None] * w[None, :])  # face quadrature weights [t_slow, t_fast]

        u_int = dg._face(u, d, side, N)
        u_ext = dg._face(u, d, 1 - side, N)[..., nb, :, :] * mask
        g_int = [dg._face(grad[i], d, side, N) for i in range(3)]
        g_ext = [dg._face(grad[i], d, 1 - side, N)[..., nb, :, :] * mask for i in range(3)]
        K_int = dg._face(K, d, side, N)
        K_nbr = dg._face(K, d, 1 - side, N)[nb]
        K_ext = np.where(has[:, None, None], K_nbr, K_int)  # boundary: the interior coefficient

        # auxiliary normal fluxes n_i F_v^i_j = n_j u, vector over j; exterior per Eq. bc
        nFv_int = [n[j] * u_int for j in range(3)]
        nFv_nbr = [-n[j] * u_ext for j in range(3)]  # n^ext = -n^int
        nFv_ext = [np.where(ext_bc, nFv_int[j], np.where(ext_neu, -nFv_int[j], nFv_nbr[j])) for j in range(3)]
        # primal normal fluxes of the local gradients, n_i F_u^i = K n . grad u
        nFu_int = K_int * sum(n[i] * g_int[i] for i in range(3))
        nFu_nbr = -K_ext * sum(n[i] * g_ext[i] for i in range(3))
        nFu_ext = np.where(ext_bc, -nFu_int, np.where(ext_neu, nFu_int, nFu_nbr))

        aux_star = [0.5 * (nFv_int[j] - nFv_ext[j]) for j in range(3)]  # Eq. numfluxaux
        h_int = face_size(N, graph.J, G, d, side)
        sigma = graph.penalty * N**2 / np.minimum(h_int, graph.hf_ext[:, f])  # Eq. penalty, p = N - 1
        # n^int.F_u(n^int F_v(u^int)) - n^ext.F_u(n^ext F_v(u^ext)) = K u^int + K^ext n . nFv_ext
        pen = K_int * u_int + K_ext * sum(n[j] * nFv_ext[j] for j in range(3))
        prim_star = 0.5 * (nFu_int - nFu_ext) - sigma * pen  # Eq. numfluxprimal

        for j in range(3):
            v[j] = v[j] + dg._lift_to_volume(Bf * (aux_star[j] - nFv_int[j]), d, side, N) / Mdiag
        prim_face.append((d, side, n, Bf, prim_star))

    Au = np.zeros_like(u)
    for i in range(3):
        for j in range(3):
            Au -= Mdiag * (G[:, j, i] * dg._deriv(K * v[i], j, Dhat))
    for d, side, n, Bf, prim_star in prim_face:
        nv_int = dg._face(K, d, side, N) * sum(n[i] * dg._face(v[i], d, side, N) for i in range(3))
        Au -= dg._lift_to_volume(Bf * (prim_star - nv_int), d, side, N)
    return Au


def _coarse_eval_matrices(N):
    """Per half h of a coarsened dimension: C[h][c, q] = l_q(2 xi_c -+ 1) for the coarse nodes c
    that lie in child h (xi_c <= 0: lower child, else upper), zero rows for the others."""
    x = lgl.lgl_nodes(N)
    lower = x <= 0.0
    C0 = lgl.interp_matrix(N, np.where(lower, 2.0 * x + 1.0, 0.0)) * lower[:, None]
    C1 = lgl.interp_matrix(N, np.where(~lower, 2.0 * x - 1.0, 0.0)) * (~lower)[:, None]
    return {0: C0, 1: C1, None: np.eye(N)}


@dataclasses.dataclass
class MappedGrid(dg.BoxGrid):
    """A box of n[0] x n[1] x n[2] elements in logical space whose elements are mapped
    isoparametrically to the given physical node coordinates xyz = (x, y, z), each (E, N, N, N),
    with the coefficient K at the nodes (None: K = 1)."""

    xyz: tuple = None
    K: np.ndarray = None

    @classmethod
    def from_mapping(cls, box: dg.BoxGrid, mapping, coefficient=None):
        """Nodes placed by a smooth map of the box's own node coordinates; coefficient(x, y, z) gives
        K at the mapped nodes."""
        xyz = tuple(np.asarray(c, float) for c in mapping(*box.coordinates()))
        K = None if coefficient is None else np.asarray(coefficient(*xyz), float)
        return cls(box.lower, box.upper, box.n, box.N, box.penalty, box.neumann, xyz, K)

    def coordinates(self):
        return tuple(c.copy() for c in self.xyz)

    def graph(self) -> CurvedGraph:
        E = self.n_elements
        nbr = np.array([[self.neighbor(e, f) for f in range(6)] for e in range(E)], dtype=np.int64)
        J, G = metric(self.N, *self.xyz)
        return make_graph(self.N, self.penalty, nbr, J, G, self.K)

    def coarsen(self, coarse_n):
        """The next multigrid level: coarse nodes on the interpolated fine map."""
        N = self.N
        box = dg.BoxGrid(self.lower, self.upper, tuple(coarse_n), N, self.penalty, self.neumann)
        C = _coarse_eval_matrices(N)
        fields = list(self.xyz) + ([] if self.K is None else [self.K])
        out = [np.zeros((box.n_elements, N, N, N)) for _ in fields]
        for e in range(self.n_elements):
            c = self.element_coords(e)
            pc, halves = [], []
            for d in range(3):
                if coarse_n[d] == self.n[d]:
                    pc.append(c[d])
                    halves.append(None)
                else:
                    pc.append(c[d] // 2)
                    halves.append(c[d] % 2)
            p = box.element_index(*pc)
            hx, hy, hz = halves
            for i, fld in enumerate(fields):
                out[i][p] += np.einsum("kc,jb,ia,cba->kji", C[hz], C[hy], C[hx], fld[e])
        K = out[3] if self.K is not None else None
        return MappedGrid(self.lower, self.upper, tuple(coarse_n), N, self.penalty, self.neumann, tuple(out[:3]), K)
