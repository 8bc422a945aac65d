"""Helpers for the GPU parity tests: seeded inputs, oracle grids, relative errors."""
import numpy as np

import workloads
from oracle import dg


def box(n, N, C=1.5, lower=(-1.0,) * 3, upper=(1.0,) * 3):
    return dg.BoxGrid(tuple(lower), tuple(upper), tuple(n), N, C)


def rand(seed, shape, lo=-1.0, hi=1.0):
    return workloads.uniform_vector(seed, int(np.prod(shape)), lo, hi).reshape(shape)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
