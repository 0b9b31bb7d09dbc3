"""Helpers shared by the GPU parity tests: oracle problems handed to the CUDA library as arrays, and
host reconstruction of device Tucker tensors.  Inputs flow oracle -> CUDA library, never back."""
from __future__ import annotations

import functools

import numpy as np

import synth
from oracle import fd, lowrank, tucker


@functools.lru_cache(maxsize=None)
def oracle_problem(kind: str, amp: float, n: int, p: int, bc=(0, 0)):
    """Operator, rhs, preconditioner and its tables from the oracle; bc = (k0, k1) marks Neumann ends."""
    terms = lowrank.operator_terms(kind, amp, n, p, bc=bc)
    f = lowrank.rhs_tucker(kind, amp, n, p, bc=bc)
    P = fd.ApproxFD(n, p, bc=bc)
    W, mu, _ = fd.sine_factorization(n, p, bc)
    n1, n2 = fd.split_dims(n - p + 2 - bc[0] - bc[1], p, bc)
    tables = {"lam": P.lam, "mu": mu, "W": W, "v2u2": P.U[:, n1:], "omega": P.omega, "alpha": P.alpha,
              "lambda_min": P.lmin, "bc": bc}
    return terms, f, P, tables


def gpu_problem(kind: str, amp: float, n: int, p: int, dtype=0, bc=(0, 0)):
    from paper_2306_00632_gb300 import api
    terms, f, P, tables = oracle_problem(kind, amp, n, p, bc)
    return api.tpcg_problem_create(n, p, terms, f[0], f[1], tables, dtype=dtype)


def random_banded_terms(n: int, p: int, R: int, seed: int):
    mats = [synth.random_banded(n, p, R, seed + t) for t in range(3)]
    g = np.random.default_rng(seed + 99)
    return [(float(g.uniform(0.5, 1.5)), [mats[0][j], mats[1][j], mats[2][j]]) for j in range(R)]


def identity_tables(n: int):
    """Preconditioner tables of the identity-free trivial kind (used where only A matters)."""
    return {"lam": np.arange(1, n + 1, dtype=float), "mu": np.ones(n), "W": np.eye(n), "v2u2": np.zeros((n, 0)),
            "omega": np.array([1.0]), "alpha": np.array([1.0]), "lambda_min": 3.0}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def full(T):
    return tucker.full(T)
