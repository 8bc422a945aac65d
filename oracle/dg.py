"""Strong-form DG operator of Sec. II for the Poisson system, on an element graph.

Oracle code (test infrastructure only).

Flux form (Eq. fluxform, Eq. poisson_fluxform): auxiliary flux F_v^i_j = u delta^i_j with
S_v = v (so S~_v = 0), primal flux F_u^i = v^i with S_u = 0, f_u = f. The operator is
evaluated in two steps, Eq. dg_op_auxvars then Eq. dg_op_primal:

    v_j  = D_i F_v^i_j + L ((n_i F_v^i_j)^* - n_i F_v^i_j)
    A u  = -MD_i F_u^i - ML ((n_i F_u^i)^* - n_i F_u^i)             (massive form, b = M f)

with the generalized internal-penalty flux (Eq. numflux), the penalty (Eq. penalty) and
boundary conditions imposed through the exterior fluxes (Eq. bc).

Readings where the paper is silent:
  * quadrature: the integrals of Eqs. massmat, stiffmat and liftop are evaluated with the
    LGL collocation quadrature, so M and the face mass are diagonal, MD_i = M D_i exactly
    and L only touches face nodes;
  * h in the penalty: the element width along the face normal (affine boxes);
  * Dirichlet boundaries are homogeneous (u_b = 0) in the operator; the paper's n^ext = -n^int;
  * Neumann boundaries (optional, per box face) are homogeneous: Eq. bc with the auxiliary
    boundary flux taken from the interior, (n F_v)^b = (n F_v)^int (so u* = u^int), and the
    primal boundary flux prescribed, (n F_u)^b = n . grad u_b = 0.

Layout: nodal data u[..., e, k, j, i] with i (x) fastest; faces f = 2 d + side, d in
{0: x, 1: y, 2: z}, side 0 = lower (n = -e_d), 1 = upper (n = +e_d).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import lgl

EXTERNAL = -1  # external boundary face: Dirichlet fluxes of Eq. bc
ZERO = -2      # internal face whose exterior data is zero (outside a Schwarz subdomain)
NEUMANN = -3   # external boundary face: homogeneous Neumann fluxes of Eq. bc

# node axis of dimension d in an array [..., e, k, j, i]
_NODE_AXIS = {0: -1, 1: -2, 2: -3}


@dataclasses.dataclass
class ElementGraph:
    """Elements of one isotropic order N with their face connectivity.

    h[e, d]    element width along d
    nbr[e, f]  exterior element index, EXTERNAL, NEUMANN or ZERO
    h_ext[e,f] width of the exterior element along the face normal (interior width at
               external faces)
    """

    N: int
    penalty: float
    h: np.ndarray
    nbr: np.ndarray
    h_ext: np.ndarray

    @property
    def n_elements(self) -> int:
        return self.h.shape[0]

    per_element = False  # one operator per neighbour pattern (uniform affine elements)

    def subgraph(self, slots, pn):
        """The elements `slots` with the face connectivity pn (a Schwarz patch)."""
        return ElementGraph(self.N, self.penalty, self.h[slots], pn, self.h_ext[slots])


@dataclasses.dataclass
class BoxGrid:
    """A box [lower, upper] split uniformly into n[0] x n[1] x n[2] affine elements. neumann[f]
    marks box face f (-x, +x, -y, +y, -z, +z) as homogeneous Neumann (Dirichlet otherwise)."""

    lower: tuple
    upper: tuple
    n: tuple
    N: int
    penalty: float
    neumann: tuple = (False,) * 6

    @property
    def n_elements(self) -> int:
        return int(np.prod(self.n))

    @property
    def h(self) -> np.ndarray:
        return (np.asarray(self.upper, float) - np.asarray(self.lower, float)) / np.asarray(self.n, float)

    def element_index(self, ex, ey, ez):
        return ex + self.n[0] * (ey + self.n[1] * ez)

    def element_coords(self, e):
        nx, ny, _ = self.n
        return e % nx, (e // nx) % ny, e // (nx * ny)

    def neighbor(self, e: int, f: int) -> int:
        c = list(self.element_coords(e))
        d, side = divmod(f, 2)
        c[d] += 1 if side else -1
        if c[d] < 0 or c[d] >= self.n[d]:
            return NEUMANN if self.neumann[f] else EXTERNAL
        return self.element_index(*c)

    def graph(self) -> ElementGraph:
        E = self.n_elements
        h = np.tile(self.h, (E, 1))
        nbr = np.array([[self.neighbor(e, f) for f in range(6)] for e in range(E)], dtype=np.int64)
        h_ext = np.repeat(h, 2, axis=1)
        return ElementGraph(self.N, self.penalty, h, nbr, h_ext)

    def coarsen(self, coarse_n):
        """The grid of the next multigrid level, with coarse_n elements per dimension."""
        return BoxGrid(self.lower, self.upper, tuple(coarse_n), self.N, self.penalty, self.neumann)

    def coordinates(self):
        """Physical coordinates (x, y, z) of every node, each shaped (E, N, N, N)."""
        xi = lgl.lgl_nodes(self.N)
        E = self.n_elements
        out = []
        for d in range(3):
            c = np.array([self.element_coords(e)[d] for e in range(E)], dtype=np.float64)
            lo = self.lower[d] + c * self.h[d]
            x1 = lo[:, None] + 0.5 * (xi[None, :] + 1.0) * self.h[d]  # (E, N)
            shape = [E, 1, 1, 1]
            shape[4 + _NODE_AXIS[d]] = self.N
            out.append(np.broadcast_to(x1.reshape(shape), (E, self.N, self.N, self.N)).copy())
        return tuple(out)


def _face(a, d, side, N):
    """Restriction E_f to the face nodes: a[..., e, k, j, i] -> [..., e, t1, t2]."""
    return np.take(a, 0 if side == 0 else N - 1, axis=_NODE_AXIS[d])


def _lift_to_volume(face_vals, d, side, N):
    """E_f^T: place face data onto the face plane of a zero volume array."""
    shape = list(face_vals.shape)
    ax = len(shape) + 1 + _NODE_AXIS[d]
    shape.insert(ax, N)
    vol = np.zeros(shape)
    idx = [slice(None)] * len(shape)
    idx[ax] = 0 if side == 0 else N - 1
    vol[tuple(idx)] = face_vals
    return vol


def _deriv(a, d, Dhat):
    """Logical derivative along dimension d: sum_l Dhat[p, l] a[..., l, ...]."""
    ax = _NODE_AXIS[d]
    return np.moveaxis(np.tensordot(np.moveaxis(a, ax, -1), Dhat, axes=([-1], [1])), -1, ax)


def operators(N):
    """1-D LGL quadrature matrices: mass[p, q] = sum_r w_r l_p(x_r) l_q(x_r) and
    stiff[p, q] = sum_r w_r l_p(x_r) l_q'(x_r) (Eqs. massmat, stiffmat on [-1, 1])."""
    x = lgl.lgl_nodes(N)
    w = lgl.lgl_weights(N)
    Dhat = lgl.diff_matrix(N)
    L = np.stack([lgl.lagrange(x, p, x) for p in range(N)])  # L[p, r] = l_p(x_r)
    dL = Dhat.T  # dL[q, r] = l_q'(x_r)
    mass = np.einsum("r,pr,qr->pq", w, L, L)
    stiff = np.einsum("r,pr,qr->pq", w, L, dL)
    return x, w, Dhat, mass, stiff


def apply(graph: ElementGraph, u: np.ndarray, dirichlet_value: float = 0.0) -> np.ndarray:
    """A u for nodal data u[..., E, N, N, N] (Eqs. dg_op_auxvars and dg_op_primal)."""
    if hasattr(graph, "apply_operator"):  # curved elements (oracle.curved)
        return graph.apply_operator(u)
    N = graph.N
    E = graph.n_elements
    u = np.asarray(u, dtype=np.float64)
    assert u.shape[-4:] == (E, N, N, N), u.shape
    x, w, Dhat, mass, stiff = operators(N)
    # LGL quadrature makes the 1-D mass diagonal: keep its diagonal
    m1 = np.diag(mass)
    W3 = m1[:, None, None] * m1[None, :, None] * m1[None, None, :]  # [k, j, i]
    J = np.prod(graph.h, axis=1) / 8.0  # affine Jacobian determinant, sqrt(g) = 1
    Mdiag = J[:, None, None, None] * W3  # (E, N, N, N)
    inv_jac = 2.0 / graph.h  # (E, 3): d xi^d / d x^d

    # D_i F_v^i_j: with F_v^i_j = u delta^i_j this is the gradient g_j = (2/h_j) D_hat_j u
    g = [inv_jac[:, d][:, None, None, None] * _deriv(u, d, Dhat) for d in range(3)]
    v = [gd.copy() for gd in g]

    prim_face = []  # per face: (n_i F_u^i)^*, needs the lifted v afterwards
    for f in range(6):
        d, side = divmod(f, 2)
        s = 1.0 if side else -1.0
        nbr = graph.nbr[:, f]
        has = nbr >= 0
        nb = np.where(has, nbr, 0)
        ext_type = nbr.copy()

        u_int = _face(u, d, side, N)
        gd_int = _face(g[d], d, side, N)
        u_ext = _face(u, d, 1 - side, N)[..., nb, :, :]
        gd_ext = _face(g[d], d, 1 - side, N)[..., nb, :, :]
        mask = has.astype(np.float64)[:, None, None]
        u_ext = u_ext * mask
        gd_ext = gd_ext * mask

        ext_bc = (ext_type == EXTERNAL)[:, None, None]
        ext_neu = (ext_type == NEUMANN)[:, None, None]
        # auxiliary normal fluxes (component d only): n_i F_v^i_d(u) = n_d u
        nFv_int = s * u_int
        nFv_ext = np.where(ext_bc, nFv_int - 2.0 * s * dirichlet_value, -s * u_ext)  # Eq. bc, Dirichlet
        nFv_ext = np.where(ext_neu, -nFv_int, nFv_ext)  # Neumann: (n F_v)^b = (n F_v)^int
        # primal normal fluxes of the local gradients: n_i F_u^i(grad u) = n . g
        nFu_int = s * gd_int
        nFu_ext = np.where(ext_bc, nFu_int - 2.0 * nFu_int, -s * gd_ext)  # Eq. bc, (nF_u)^b = (nF_u)^int
        nFu_ext = np.where(ext_neu, nFu_int, nFu_ext)  # Neumann: (n F_u)^b = n . grad u_b = 0

        # Eq. numfluxaux: component d of (n_i F_v^i)^*
        aux_star = 0.5 * (nFv_int - nFv_ext)
        # Eq. penalty, p = N - 1 on both sides
        p = N - 1
        h_int = graph.h[:, d]
        h_ext = graph.h_ext[:, f]
        sigma = graph.penalty * (p + 1) ** 2 / np.minimum(h_int, h_ext)
        # Eq. numfluxprimal: n^int.F_u(n^int F_v(u^int)) = u^int; n^ext.F_u(n^ext F_v(u^ext)) = -n_d (nFv_ext)
        pen = u_int - (-s * nFv_ext)
        prim_star = 0.5 * (nFu_int - nFu_ext) - sigma[:, None, None] * pen

        # lifting L = M^-1 ML of the auxiliary flux difference (Eq. liftop with LGL quadrature)
        tang = [t for t in range(3) if t != d]
        Jf = np.prod(graph.h[:, tang], axis=1) / 4.0  # surface Jacobian
        # face quadrature weights: tangential 1-D weights on the face grid [t_slow, t_fast]
        Bf = Jf[:, None, None] * (m1[:, None] * m1[None, :])
        lifted = _lift_to_volume(Bf * (aux_star - nFv_int), d, side, N) / Mdiag
        v[d] = v[d] + lifted
        prim_face.append((d, side, s, Bf, prim_star))

    # Eq. dg_op_primal: -MD_i v^i - ML ((n.v)^* - n.v)
    Au = np.zeros_like(u)
    for d in range(3):
        Au -= Mdiag * (inv_jac[:, d][:, None, None, None] * _deriv(v[d], d, Dhat))
    for d, side, s, Bf, prim_star in prim_face:
        nv_int = s * _face(v[d], d, side, N)
        Au -= _lift_to_volume(Bf * (prim_star - nv_int), d, side, N)
    return Au


def mass_diag(graph: ElementGraph) -> np.ndarray:
    """Diagonal of the LGL mass matrix M (Eq. massmat), shaped (E, N, N, N)."""
    if hasattr(graph, "mass"):  # curved elements (oracle.curved)
        return graph.mass()
    _, _, _, mass, _ = operators(graph.N)
    m1 = np.diag(mass)
    W3 = m1[:, None, None] * m1[None, :, None] * m1[None, None, :]
    J = np.prod(graph.h, axis=1) / 8.0
    return J[:, None, None, None] * W3


def rhs(graph: ElementGraph, f_nodal: np.ndarray) -> np.ndarray:
    """b = M f (right-hand side of Eq. dg_op_primal, homogeneous boundary data)."""
    return mass_diag(graph) * f_nodal


def assemble(graph: ElementGraph) -> np.ndarray:
    """Dense A, built column by column from the matrix-free apply (tiny grids only)."""
    N, E = graph.N, graph.n_elements
    n = E * N**3
    eye = np.eye(n).reshape(n, E, N, N, N)
    cols = apply(graph, eye).reshape(n, n)  # cols[c] = A e_c
    return cols.T.copy()
