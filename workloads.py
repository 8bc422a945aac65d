"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds only input generation: a counter-based pseudo-random stream
(splitmix64, Steele, Lea & Flood 2014), the parameters of the source terms and
the named problem configurations. It contains none of the method's arithmetic
(no LGL grids, no DG operator, no solver), so both the CPU oracle and the CUDA
path can draw identical inputs from it without sharing any computation.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64 stream: state += golden gamma, then two xor-shift-multiply mixes."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        """Uniform double in [lo, hi) from the top 53 bits."""
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / 9007199254740992.0))

    def uniform_array(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        return np.array([self.uniform(lo, hi) for _ in range(n)], dtype=np.float64)

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in the closed range [lo, hi]."""
        return lo + int(self.uniform() * (hi - lo + 1))


def uniform_vector(seed: int, n: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """A length-n vector of U[lo, hi) values, vectorised splitmix64 (bitwise equal to the scalar stream)."""
    idx = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + idx * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


@dataclasses.dataclass(frozen=True)
class GaussianSource:
    """f(x) = sum_g A_g exp(-|x - c_g|^2 / s_g^2) (the exp(-r^2/w^2) convention)."""

    amp: tuple
    center: tuple
    width: tuple

    def __call__(self, x, y, z):
        xp = np if isinstance(x, np.ndarray) or np.isscalar(x) else _torch()
        f = 0.0 * x
        for a, c, s in zip(self.amp, self.center, self.width):
            r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
            f = f + a * xp.exp(-r2 / (s * s))
        return f


def _torch():
    import torch

    return torch


def gaussian_source(seed: int, count: int = 16, box=(-1.0, 1.0)) -> GaussianSource:
    """Seeded sum of `count` Gaussians: A ~ U[-1,1], centres ~ U[-0.8,0.8]^3 (scaled to the box),
    widths ~ U[0.1,0.4] (scaled to the box half-width)."""
    rng = SplitMix64(seed)
    half = 0.5 * (box[1] - box[0])
    mid = 0.5 * (box[1] + box[0])
    amp, center, width = [], [], []
    for _ in range(count):
        amp.append(rng.uniform(-1.0, 1.0))
        center.append(tuple(mid + half * rng.uniform(-0.8, 0.8) for _ in range(3)))
        width.append(half * rng.uniform(0.1, 0.4))
    return GaussianSource(tuple(amp), tuple(center), tuple(width))


def sine_source_3d(x, y, z):
    """f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z): -Laplace of the manufactured solution below."""
    xp = np if isinstance(x, np.ndarray) or np.isscalar(x) else _torch()
    return 3.0 * math.pi**2 * xp.sin(math.pi * x) * xp.sin(math.pi * y) * xp.sin(math.pi * z)


def sine_solution_3d(x, y, z):
    xp = np if isinstance(x, np.ndarray) or np.isscalar(x) else _torch()
    return xp.sin(math.pi * x) * xp.sin(math.pi * y) * xp.sin(math.pi * z)


@dataclasses.dataclass(frozen=True)
class Puncture:
    position: tuple
    mass: float
    momentum: tuple


# Two punctures at (+-3, 0, 0), bare masses 0.5, momenta +-(0, 0.1, 0).
BINARY_PUNCTURES = (
    Puncture((3.0, 0.0, 0.0), 0.5, (0.0, 0.1, 0.0)),
    Puncture((-3.0, 0.0, 0.0), 0.5, (0.0, -0.1, 0.0)),
)


@dataclasses.dataclass(frozen=True)
class ProblemConfig:
    name: str
    lower: tuple
    upper: tuple
    n: tuple
    N: int
    penalty: float
    mg_levels: int  # 0 = coarsen until a dimension count is odd
    overlap: int
    presmooth: int
    postsmooth: int
    problem: str  # "poisson" | "puncture"
    source: str  # "sine" | "gaussian" | "puncture"
    seed: int

    @property
    def n_elements(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def n_dof(self) -> int:
        return self.n_elements * self.N**3


SINE_2x2x2 = ProblemConfig("poisson-sine-2x2x2-N6", (-1.0,) * 3, (1.0,) * 3, (2, 2, 2), 6, 1.5,
                           0, 2, 3, 3, "poisson", "sine", 1)
GAUSS_8x8x8 = ProblemConfig("poisson-gauss16-8x8x8-N8", (-1.0,) * 3, (1.0,) * 3, (8, 8, 8), 8, 1.5,
                            3, 2, 3, 3, "poisson", "gaussian", 2)
PUNCTURE_16 = ProblemConfig("puncture-16x16x16-N6", (-20.0,) * 3, (20.0,) * 3, (16, 16, 16), 6, 1.5,
                            0, 2, 3, 3, "puncture", "puncture", 3)


def batched_shapes(seed: int = 4, count: int = 512):
    """Per-solve (n_x, n_y, n_z, N) for the batched workload: n_i ~ U{2..8}, N ~ U{4..9}."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        n = tuple(rng.randint(2, 8) for _ in range(3))
        out.append((n, rng.randint(4, 9)))
    return out


def poisson_arrivals(seed: int = 5, rate: float = 200.0, duration: float = 20.0):
    """Poisson-process arrival times with mean rate `rate` over `duration` seconds, plus per-request
    kind ('poisson' | 'puncture'), cubic element count n ~ U{2..12} and N ~ U{4..8}."""
    rng = SplitMix64(seed)
    t, out = 0.0, []
    while True:
        t += -math.log(1.0 - rng.uniform()) / rate
        if t >= duration:
            return out
        kind = "poisson" if rng.uniform() < 0.5 else "puncture"
        out.append((t, kind, rng.randint(2, 12), rng.randint(4, 8), rng.next_u64() & 0xFFFFFFFF))
