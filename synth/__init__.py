"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and the benchmark.

This module holds no arithmetic of the solver: only counter-based random numbers, random
arrays and the records that describe a workload (degree, dofs, geometry amplitude, rank
caps, arrival times).  Both the FP64 oracle and the CUDA path read their inputs from here,
so the two sides see bit-identical inputs.
"""
from __future__ import annotations

import dataclasses
import numpy as np

_MASK64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """One step of the splitmix64 generator (Steele, Lea, Flood 2014), as a pure function."""
    z = (x + 0x9E3779B97F4A7C15) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def unit_from_seed(seed: int, stream: int = 0) -> float:
    """A float in [0, 1) drawn from ``seed`` (53 random bits)."""
    return (splitmix64((seed * 0x100000001B3 + stream) & _MASK64) >> 11) / float(1 << 53)


def amp_from_seed(seed: int) -> float:
    """Twist amplitude of the twisted quarter-annulus family, uniform in [0, 0.3]."""
    return 0.3 * unit_from_seed(seed, 1)


# ----------------------------------------------------------------------------------------
# Workload records
# ----------------------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Problem:
    """One Poisson (or elasticity) problem: geometry kind, amplitude, degree and dofs."""
    kind: str          # "cube" | "twist"
    degree: int        # spline degree p
    n: int             # dofs per direction (n = n_el + p - 2)
    amp: float = 0.0   # twist amplitude (twist only)
    seed: int = 0
    physics: str = "poisson"   # "poisson" | "elasticity"
    lame_lambda: float = 1.0
    lame_mu: float = 1.0

    @property
    def n_el(self) -> int:
        return self.n - self.degree + 2


CUBE_SMALL = Problem(kind="cube", degree=2, n=32)                                     # unit cube p=2 n=32
TWIST_128 = Problem(kind="twist", degree=3, n=128, amp=amp_from_seed(7), seed=7)      # twisted annulus p=3 n=128
TWIST_512 = Problem(kind="twist", degree=3, n=512, amp=amp_from_seed(7), seed=7)      # twisted annulus p=3 n=512


def batch_mix(count: int, seed0: int = 0, caps=(20, 60)):
    """Mixed batch of independent Poisson problems: n in {32..256}, p in {2,3,4},
    amplitude in [0, 0.3], rank caps uniform in [caps[0], caps[1]] (one record per solve)."""
    ns = (32, 64, 96, 128, 192, 256)
    out = []
    for s in range(seed0, seed0 + count):
        n = ns[int(unit_from_seed(s, 2) * len(ns))]
        p = 2 + int(unit_from_seed(s, 3) * 3)
        cap = caps[0] + int(unit_from_seed(s, 4) * (caps[1] - caps[0] + 1))
        out.append((Problem(kind="twist", degree=p, n=n, amp=amp_from_seed(s), seed=s), cap))
    return out


def poisson_arrivals(rate_hz: float, count: int, seed: int = 0) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process with the given rate."""
    g = np.random.default_rng(seed)
    return np.cumsum(g.exponential(1.0 / rate_hz, size=count))


# ----------------------------------------------------------------------------------------
# Random Tucker tensors (plain random numbers; no orthogonalisation)
# ----------------------------------------------------------------------------------------
def random_factors(n, ranks, seed):
    g = np.random.default_rng(seed)
    return [g.standard_normal((n[t], ranks[t])) for t in range(3)]


def random_core(ranks, seed, decay: float | None = None):
    """Random core; with ``decay`` the entry (i,j,k) is scaled by decay**(i+j+k), which gives
    mode singular values that fall off geometrically."""
    g = np.random.default_rng(seed)
    c = g.standard_normal(tuple(ranks))
    if decay is not None:
        i, j, k = np.meshgrid(*[np.arange(r) for r in ranks], indexing="ij")
        c = c * decay ** (i + j + k)
    return c


def random_tucker(n, ranks, seed, decay=None):
    """(core, [U1, U2, U3]) with core shape ``ranks`` and factor U_t of shape n_t x r_t."""
    return random_core(ranks, seed, decay), random_factors(n, ranks, seed + 1)


def random_banded(n: int, p: int, count: int, seed: int, symmetric: bool = True):
    """``count`` random banded n x n matrices with half-bandwidth p, as dense arrays."""
    g = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        a = g.standard_normal((n, n))
        if symmetric:
            a = a + a.T
        i, j = np.indices((n, n))
        a[np.abs(i - j) > p] = 0.0
        out.append(a)
    return out
