"""The allocation-free inner products (dg_dot_noalloc) against the allocating dg_dot.

dg_dot_noalloc serves callers that cannot allocate device memory when they need the FGMRES inner
products (stream capture, fixed-memory serving loops, embedding hosts that own all allocations).
It keeps its partial sums in a fixed device array instead of a domain workspace; its results must
equal dg_dot's, call after call. This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from gpu_util import rand

pytestmark = pytest.mark.gpu

dgg = pytest.importorskip("paper_2111_06767_gb300")
from paper_2111_06767_gb300 import _native  # noqa: E402


def _noalloc(lib, V, w, out, stream):
    m, ld = V.shape[0], V.stride(0)
    return lib.dg_dot_noalloc(w.numel(), m, C.c_void_p(V.data_ptr()), ld, C.c_void_p(w.data_ptr()),
                              C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))


def test_noalloc_dot_matches_dg_dot_on_consecutive_calls():
    lib = _native.load()
    d = dgg.Domain(n=(4, 4, 4), N=6, mg_levels=1, overlap=1)
    n = d.n_dof
    stream = torch.cuda.current_stream()
    for call, (m, seed) in enumerate([(9, 71), (64, 72)]):  # two calls in a row, different shapes
        V = torch.from_numpy(rand(seed, (m, n))).cuda()
        w = torch.from_numpy(rand(seed + 100, (n,))).cuda()
        ref = d.dot(V, w).cpu().numpy()
        out = torch.full((m,), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(lib, V, w, out, stream) == _native.DG_OK, lib.dg_last_error(None)
        got = out.cpu().numpy()
        scale = np.abs(V.cpu().numpy()).sum(axis=1).max()
        assert np.abs(got - ref).max() <= 1e-13 * scale, call
    # sizes beyond the fixed scratch are rejected with a message, nothing is launched
    V = torch.zeros((65, 16), dtype=torch.float64, device="cuda")
    w = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(65, dtype=torch.float64, device="cuda")
    assert _noalloc(lib, V, w, out, stream) == -1
    assert b"DG_NOALLOC_MAX_VECTORS" in lib.dg_last_error(None)
