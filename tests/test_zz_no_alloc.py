"""The allocation-free inner products (dg_dot_noalloc) against the allocating dg_dot.

dg_dot_noalloc serves callers that cannot allocate device memory when they need the FGMRES inner
products (stream capture, fixed-memory serving loops, embedding hosts that own all allocations).
It keeps its partial sums in a fixed device array instead of a domain workspace. The header
promises the same result as dg_dot bit for bit (same kernels, same reduction order), call after
call; an exactly rounded sum (math.fsum) checks both against the definition of the inner product.
This file is collected last so that a run stopping at the first failure has already run every
other test; it also passes alone in a fresh process.
"""
import ctypes as C
import math

import numpy as np
import pytest
import torch

from gpu_util import rand

pytestmark = pytest.mark.gpu

dgg = pytest.importorskip("paper_2111_06767_gb300")
from paper_2111_06767_gb300 import _native  # noqa: E402


def _noalloc(lib, V, w, out, stream):
    m, ld = V.shape[0], V.stride(0)
    assert V.stride(1) == 1
    return lib.dg_dot_noalloc(w.numel(), m, C.c_void_p(V.data_ptr()), ld, C.c_void_p(w.data_ptr()),
                              C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))


def _exact(V, w):
    """Correctly rounded inner products and the sums of |V_ki w_i| (the scale of their rounding)."""
    Vh, wh = V.cpu().numpy(), w.cpu().numpy()
    return (np.array([math.fsum(row * wh) for row in Vh]), np.abs(Vh * wh).sum(axis=1))


def _dg_dot(lib, d, V, w, stream):
    """dg_dot through the C ABI (the rows of V may be a strided view, ld = V.stride(0))."""
    out = torch.full((V.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
    assert lib.dg_dot(d.handle, V.shape[0], C.c_void_p(V.data_ptr()), V.stride(0), C.c_void_p(w.data_ptr()),
                      C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream)) == _native.DG_OK
    return out.cpu().numpy()


def _call(lib, V, w, stream):
    out = torch.full((V.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
    assert _noalloc(lib, V, w, out, stream) == _native.DG_OK, lib.dg_last_error(None)
    return out.cpu().numpy()


def test_noalloc_dot_matches_dg_dot_on_consecutive_calls():
    lib = _native.load()
    d = dgg.Domain(n=(4, 4, 4), N=6, mg_levels=1, overlap=1)
    n = d.n_dof
    stream = torch.cuda.current_stream()
    # two calls in a row with different shapes, then a strided view (ld > n) and a single vector
    for call, (m, seed, pad) in enumerate([(9, 71, 0), (64, 72, 0), (5, 73, 40), (1, 74, 0)]):
        big = torch.from_numpy(rand(seed, (m, n + pad))).cuda()
        V = big[:, :n]
        w = torch.from_numpy(rand(seed + 100, (n,))).cuda()
        ref = _dg_dot(lib, d, V, w, stream)
        got = _call(lib, V, w, stream)
        assert np.array_equal(got, ref), (call, np.abs(got - ref).max())
        exact, scale = _exact(V, w)
        assert np.all(np.abs(got - exact) <= 1e-14 * scale), (call, np.abs(got - exact).max())
    # the same inputs again after other shapes: the shared array holds the last call's partial sums,
    # which must not leak into this one
    V = torch.from_numpy(rand(71, (9, n))).cuda()
    w = torch.from_numpy(rand(171, (n,))).cuda()
    assert np.array_equal(_call(lib, V, w, stream), _dg_dot(lib, d, V, w, stream))


def test_noalloc_rejects_sizes_beyond_the_fixed_array():
    lib = _native.load()
    stream = torch.cuda.current_stream()
    V = torch.zeros((65, 16), dtype=torch.float64, device="cuda")
    w = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(65, dtype=torch.float64, device="cuda")
    assert _noalloc(lib, V, w, out, stream) == -1  # DG_ERR_INVALID_ARG
    assert b"DG_NOALLOC_MAX_VECTORS" in lib.dg_last_error(None)
    # a later failed domain creation reports its own error, not the earlier one
    with pytest.raises(_native.NativeError) as err:
        dgg.Domain(n=(2, 2, 2), N=1)
    assert "DG_NOALLOC_MAX_VECTORS" not in str(err.value)
    assert b"DG_NOALLOC_MAX_VECTORS" not in lib.dg_last_error(None)
    # and a successful call clears the message
    V = torch.ones((2, 16), dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    assert _noalloc(lib, V, torch.ones(16, dtype=torch.float64, device="cuda"), out, stream) == _native.DG_OK
    assert lib.dg_last_error(None) == b""
    assert out.cpu().tolist() == [16.0, 16.0]
