"""GB300-native DG multigrid-Schwarz elliptic solver (arXiv 2111.06767), Python binding.

Thin wrapper over the C ABI of `libdg_elliptic.so` (include/dg_elliptic.h): PyTorch provides
device memory and streams, the library's CUDA kernels do all the work. Importing this package
loads the library and fails loudly if it has not been built.
"""
from __future__ import annotations

import ctypes as C
import dataclasses

import torch

from . import _native as nat
from ._native import NativeError, check

_lib = nat.load()

__all__ = ["Domain", "Batch", "Server", "solve_opts", "NativeError", "lib"]


def lib():
    return _lib


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


GEMM_MODES = {"default": 0, "simt": 1, "tf32": 2}


def make_desc(lower, upper, n, N, penalty=1.5, precision="fp64", mg_levels=0, overlap=2, presmooth=3,
              postsmooth=3, problem="poisson", punctures=(), gemm="default", neumann=(), node_xyz=None,
              coef=None):
    """neumann: indices of the box faces (0 -x, 1 +x, 2 -y, 3 +y, 4 -z, 5 +z) with homogeneous
    Neumann conditions (the others are homogeneous Dirichlet). node_xyz: None for the affine box,
    else the physical (x, y, z) of every LGL node (three arrays of n_dof values in the element-major
    layout) of curved elements; coef: None for K = 1, else K at every node (-div(K grad u)). The
    returned descriptor points at float64 host copies kept as desc.node_xyz_host / desc.coef_host."""
    d = nat.dg_domain_desc()
    for i in range(3):
        d.lower[i], d.upper[i], d.n[i] = lower[i], upper[i], n[i]
    d.N, d.penalty = N, penalty
    d.precision = {"fp64": nat.PRECISION_FP64, "mixed": nat.PRECISION_MIXED}[precision]
    d.mg_levels, d.overlap, d.presmooth, d.postsmooth = mg_levels, overlap, presmooth, postsmooth
    d.problem = {"poisson": nat.PROBLEM_POISSON, "puncture": nat.PROBLEM_PUNCTURE}[problem]
    d.n_punctures = len(punctures)
    for q, p in enumerate(punctures):
        for i in range(3):
            d.punctures[q].position[i] = p.position[i]
            d.punctures[q].momentum[i] = p.momentum[i]
        d.punctures[q].mass = p.mass
    d.subdomain_gemm = GEMM_MODES[gemm]
    d.neumann_faces = sum(1 << int(f) for f in set(neumann))
    if node_xyz is not None:
        import numpy as np

        parts = [c.detach().cpu().numpy() if isinstance(c, torch.Tensor) else c for c in node_xyz]
        host = np.ascontiguousarray(np.stack([np.asarray(c, dtype=np.float64).ravel() for c in parts]))
        if host.shape[1] != n[0] * n[1] * n[2] * N**3:
            raise ValueError("node_xyz needs n_dof coordinates per dimension")
        d.node_xyz = host.ctypes.data_as(C.POINTER(C.c_double))
        d.node_xyz_host = host
    if coef is not None:
        import numpy as np

        k = coef.detach().cpu().numpy() if isinstance(coef, torch.Tensor) else coef
        host_k = np.ascontiguousarray(np.asarray(k, dtype=np.float64).ravel())
        if host_k.size != n[0] * n[1] * n[2] * N**3:
            raise ValueError("coef needs n_dof values")
        d.coef = host_k.ctypes.data_as(C.POINTER(C.c_double))
        d.coef_host = host_k
    return d


def host_coordinates(desc):
    """(x, y, z) numpy arrays of the node coordinates of the grid `desc` describes (host only)."""
    import numpy as np

    n = desc.n[0] * desc.n[1] * desc.n[2] * desc.N**3
    out = [np.empty(n) for _ in range(3)]
    ptrs = [a.ctypes.data_as(C.POINTER(C.c_double)) for a in out]
    check(_lib.dg_layout_coordinates_host(C.byref(desc), *ptrs))
    return tuple(out)


KRYLOV = {"fgmres": 0, "fcg": 1}


SUBDOMAIN_SOLVERS = {"gmres": 0, "inverse": 1}


def solve_opts(max_iterations=200, precondition=2, linear_tol=1e-4, max_newton_steps=20, subdomain_iterations=3,
               relative_to_b=False, krylov="fgmres", subdomain_solver="gmres"):
    return nat.dg_solve_opts(max_iterations, precondition, linear_tol, max_newton_steps, subdomain_iterations,
                             int(relative_to_b), KRYLOV[krylov], SUBDOMAIN_SOLVERS[subdomain_solver])


def debug_bounds_check():
    """First kernel source line whose set-up-table index was out of range since the last call (0: none),
    in the bounds-checked build (DG_DEBUG_BUILD=1); -1 in the release build."""
    return int(_lib.dg_debug_bounds_check())


@dataclasses.dataclass
class SolveReport:
    status: int
    iterations: int
    newton_steps: int
    line_search_steps: int
    initial_residual: float
    final_residual: float
    relative_residual: float
    seconds: float


class Domain:
    """A discretized box with its multigrid hierarchy and Schwarz subdomain inverses."""

    def __init__(self, lower=(-1.0,) * 3, upper=(1.0,) * 3, n=(2, 2, 2), N=6, penalty=1.5, precision="fp64",
                 mg_levels=0, overlap=2, presmooth=3, postsmooth=3, problem="poisson", punctures=(), stream=None,
                 gemm="default", neumann=(), node_xyz=None, coef=None):
        self.desc = make_desc(lower, upper, n, N, penalty, precision, mg_levels, overlap, presmooth, postsmooth,
                              problem, punctures, gemm, neumann, node_xyz, coef)
        self._h = C.c_void_p()
        st = _lib.dg_domain_create(C.byref(self.desc), _stream(stream), C.byref(self._h))
        if st != nat.DG_OK:
            msg = _lib.dg_last_error(None)
            raise NativeError(st, msg.decode() if msg else "")
        self.layout = nat.dg_layout()
        check(_lib.dg_domain_layout(self._h, C.byref(self.layout)), self._h)
        self.n_dof = int(self.layout.n_dof)
        self.N = N
        self.n_elements = int(self.layout.n_elements)
        self.mg_levels = int(self.layout.mg_levels)

    def close(self):
        if self._h:
            _lib.dg_domain_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def level_dofs(self, level):
        n = self.layout.level_n[level]
        return n[0] * n[1] * n[2] * self.N**3

    def coordinates(self):
        """(x, y, z) node coordinates as FP64 CUDA tensors (copies of library-owned memory)."""
        out = tuple(self._new() for _ in range(3))
        check(_lib.dg_copy_coordinates(self._h, *[_ptr(t) for t in out], _stream(None)), self._h)
        return out

    def _new(self, dtype=torch.float64, level=0):
        return torch.empty(self.level_dofs(level), dtype=dtype, device="cuda")

    def apply(self, u, out=None, stream=None):
        out = self._new() if out is None else out
        check(_lib.dg_apply(self._h, _ptr(u), _ptr(out), _stream(stream)), self._h)
        return out

    def apply_level(self, level, u, out=None, stream=None):
        out = self._new(level=level) if out is None else out
        check(_lib.dg_apply_level(self._h, level, _ptr(u), _ptr(out), _stream(stream)), self._h)
        return out

    def apply_f32(self, u, level=0, out=None, stream=None):
        out = self._new(torch.float32, level) if out is None else out
        check(_lib.dg_apply_f32(self._h, level, _ptr(u), _ptr(out), _stream(stream)), self._h)
        return out

    def rhs(self, f, out=None, stream=None):
        out = self._new() if out is None else out
        check(_lib.dg_rhs(self._h, _ptr(f), _ptr(out), _stream(stream)), self._h)
        return out

    def restrict(self, level, r_fine, out=None, stream=None):
        out = self._new(level=level + 1) if out is None else out
        check(_lib.dg_mg_restrict(self._h, level, _ptr(r_fine), _ptr(out), _stream(stream)), self._h)
        return out

    def prolongate_add(self, level, u_coarse, u_fine, stream=None):
        check(_lib.dg_mg_prolongate_add(self._h, level, _ptr(u_coarse), _ptr(u_fine), _stream(stream)), self._h)
        return u_fine

    def schwarz_smooth(self, level, b, u, iterations, stream=None):
        check(_lib.dg_schwarz_smooth(self._h, level, _ptr(b), _ptr(u), iterations, _stream(stream)), self._h)
        return u

    def vcycle(self, r, out=None, stream=None):
        out = self._new() if out is None else out
        check(_lib.dg_vcycle(self._h, _ptr(r), _ptr(out), _stream(stream)), self._h)
        return out

    def dot(self, V, w, out=None, stream=None):
        """out[k] = V[k] . w for the rows of a (m, n_dof) FP64 CUDA tensor V."""
        m = V.shape[0]
        out = torch.empty(m, dtype=torch.float64, device="cuda") if out is None else out
        check(_lib.dg_dot(self._h, m, _ptr(V), V.stride(0), _ptr(w), _ptr(out), _stream(stream)), self._h)
        return out

    def nonlinear_residual(self, u, b=None, out=None, stream=None):
        out = self._new() if out is None else out
        check(_lib.dg_nonlinear_residual(self._h, _ptr(u), _ptr(b), _ptr(out), _stream(stream)), self._h)
        return out

    def set_linearization(self, u, stream=None):
        check(_lib.dg_set_linearization(self._h, _ptr(u), _stream(stream)), self._h)

    def set_subdomain_solver(self, solver="gmres", iterations=3, stream=None):
        check(_lib.dg_set_subdomain_solver(self._h, SUBDOMAIN_SOLVERS[solver], iterations, _stream(stream)), self._h)

    def puncture_fields(self):
        a, b = self._new(), self._new()
        check(_lib.dg_puncture_fields(self._h, _ptr(a), _ptr(b), _stream(None)), self._h)
        return a, b

    def profile(self, enable=True):
        check(_lib.dg_profile_enable(self._h, int(enable)), self._h)

    def profile_read(self):
        arr = (nat.dg_phase_stats * len(nat.PHASES))()
        check(_lib.dg_profile_read(self._h, arr), self._h)
        return {name: {"launches": int(a.launches), "ms": a.milliseconds, "bytes": a.bytes, "flops": a.flops}
                for name, a in zip(nat.PHASES, arr)}

    def solve_host(self, f_host, u_host, tol=1e-10, opts=None, check_status=True):
        """elliptic_solve_host: f_host, u_host are contiguous float64 host arrays (numpy, or CPU
        tensors; pinned ones make the copies DMA transfers); u_host is overwritten with the solution."""
        import numpy as np

        def hp(a):
            if a is None:
                return None
            if isinstance(a, torch.Tensor):
                assert a.device.type == "cpu" and a.dtype == torch.float64 and a.is_contiguous()
                return C.c_void_p(a.data_ptr())
            assert isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
            return C.c_void_p(a.ctypes.data)

        rep = nat.dg_solve_report()
        o = opts if opts is not None else solve_opts()
        st = _lib.elliptic_solve_host(self._h, hp(f_host), hp(u_host), tol, C.byref(o), C.byref(rep))
        if check_status and st != nat.DG_OK:
            msg = _lib.dg_last_error(self._h)
            raise NativeError(st, msg.decode() if msg else "")
        return SolveReport(rep.status, rep.iterations, rep.newton_steps, rep.line_search_steps, rep.initial_residual,
                           rep.final_residual, rep.relative_residual, rep.seconds)

    def solve(self, b, u, tol=1e-10, opts=None, check_status=True):
        """Run elliptic_solve on the domain's stream (synchronises it with torch's current stream)."""
        torch.cuda.current_stream().synchronize()
        rep = nat.dg_solve_report()
        o = opts if opts is not None else solve_opts()
        st = _lib.elliptic_solve(self._h, _ptr(b), _ptr(u), tol, C.byref(o), C.byref(rep))
        if check_status and st != nat.DG_OK:
            msg = _lib.dg_last_error(self._h)
            raise NativeError(st, msg.decode() if msg else "")
        return SolveReport(rep.status, rep.iterations, rep.newton_steps, rep.line_search_steps, rep.initial_residual,
                           rep.final_residual, rep.relative_residual, rep.seconds)


class Batch:
    """Many independent linear solves captured as one CUDA graph (elliptic_batch_*): `domains`,
    `bs` and `us` are equal-length sequences of Domain objects and their FP64 CUDA right-hand sides
    and solution vectors (fixed for the life of the batch; us hold the initial guesses)."""

    def __init__(self, domains, bs, us, tol=1e-10, opts=None):
        n = len(domains)
        self._keep = (list(domains), list(bs), list(us))
        arr = lambda xs: (C.c_void_p * n)(*[x for x in xs])
        self._d = arr([d._h.value for d in domains])
        self._b = arr([_ptr(b).value for b in bs])
        self._u = arr([_ptr(u).value for u in us])
        self.count = n
        self._h = C.c_void_p()
        o = opts if opts is not None else solve_opts()
        torch.cuda.current_stream().synchronize()
        st = _lib.elliptic_batch_create(self._d, self._b, self._u, n, tol, C.byref(o), C.byref(self._h))
        if st != nat.DG_OK:
            msg = _lib.dg_last_error(None)
            raise NativeError(st, msg.decode() if msg else "")

    def run(self, stream=None):
        """Launch every solve (one graph launch) and wait; returns one SolveReport per solve."""
        reps = (nat.dg_solve_report * self.count)()
        st = _lib.elliptic_batch_run(self._h, _stream(stream), reps)
        if st != nat.DG_OK:
            msg = _lib.dg_last_error(None)
            raise NativeError(st, msg.decode() if msg else "")
        return [SolveReport(r.status, r.iterations, r.newton_steps, r.line_search_steps, r.initial_residual,
                            r.final_residual, r.relative_residual, r.seconds) for r in reps]

    def close(self):
        if self._h:
            _lib.elliptic_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching solve server (elliptic_serve_*)."""

    def __init__(self, memory_budget_bytes=0, max_active=4, queue_capacity=4096, n_streams=4):
        d = nat.dg_serve_desc(memory_budget_bytes, max_active, queue_capacity, n_streams)
        self._h = C.c_void_p()
        check(_lib.elliptic_serve_create(C.byref(d), C.byref(self._h)))
        self._keep = {}

    def submit(self, desc, f_host=None, tol=1e-10, opts=None):
        import numpy as np

        req = nat.dg_request()
        req.domain = desc
        if f_host is not None:
            arr = np.ascontiguousarray(f_host, dtype=np.float64)
            req.f_host = arr.ctypes.data_as(C.POINTER(C.c_double))
        req.tol = tol
        req.opts = opts if opts is not None else solve_opts()
        t = C.c_uint64()
        st = _lib.elliptic_serve_submit(self._h, C.byref(req), C.byref(t))
        if st != nat.DG_OK:
            raise NativeError(st, "submit")
        return int(t.value)

    def poll(self, ticket, u_out=None):
        """Returns (status, dg_result) ; status DG_PENDING (1) while running."""
        res = nat.dg_result()
        if u_out is not None:
            res.u_host = u_out.ctypes.data_as(C.POINTER(C.c_double))
        st = _lib.elliptic_serve_poll(self._h, C.c_uint64(ticket), C.byref(res))
        return st, res

    def cancel(self, ticket):
        """Cancel a waiting or running request (its poll then returns DG_ERR_CANCELLED)."""
        return _lib.elliptic_serve_cancel(self._h, C.c_uint64(ticket))

    def clock(self):
        return _lib.elliptic_serve_clock(self._h)

    def close(self):
        if self._h:
            _lib.elliptic_serve_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
