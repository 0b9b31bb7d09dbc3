"""Truncated Preconditioned Conjugate Gradient, Alg. 5 (with Alg. 1, 2 and 4).

Oracle module (test infrastructure only).

Readings:
  * the stopping test is relative, ||r_k|| <= tol ||f~||, and ||f|| in eq. rel_tol_iterates is ||f~||;
  * the truncation parameter beta of eq. rel_tol_iterates is called ``beta_trunc``; the CG
    coefficient beta_k keeps its name;
  * eps_min defaults to tol ||f~|| / 10 (Sec. 5) unless given;
  * x_0 = 0, so r_0 = f~ (Alg. 5 step 1 needs no truncation).
"""
from __future__ import annotations

import dataclasses
import numpy as np

from . import rounding, tucker


@dataclasses.dataclass
class Params:
    tol: float = 1e-6
    eps0: float = 0.1
    eps_min: float | None = None
    alpha: float = 0.5
    delta: float = 1e-3
    beta_trunc: float = 0.1
    max_it: int = 500
    caps: tuple | None = None


def tpcg(terms, f, prec, prm: Params, record=None):
    """Alg. 5.  ``terms`` is the Kronecker-sum operator, ``f`` the Tucker rhs, ``prec`` a callable
    S -> P~^{-1} S (unrounded Tucker).  Returns (x, info)."""
    A = lambda X: tucker.matvec(terms, X)
    nf = tucker.norm(f)
    eps_min = prm.eps_min if prm.eps_min is not None else prm.tol * nf * 0.1
    n = [u.shape[0] for u in f[1]]
    x = (np.zeros((0, 0, 0)), [np.zeros((n[t], 0)) for t in range(3)])
    r = f
    nr = tucker.norm(r)
    eta = prm.beta_trunc * prm.tol * nf / nr
    z = rounding.t_rel(prec(r), eta, prm.caps)
    p = z
    q = rounding.t_rel(A(p), eta, prm.caps)
    xi = tucker.dot(p, q)
    eps = prm.eps0
    k = 0
    hist = [nr / nf]
    while nr > prm.tol * nf and k < prm.max_it:
        omega = tucker.dot(r, p) / xi
        x_tilde = tucker.add(x, tucker.scale(p, omega))
        x, eps, trials = rounding.t_dt(x, x_tilde, eps, prm.alpha, eps_min, prm.delta, prm.caps)
        r = rounding.t_rel(tucker.add(f, tucker.scale(A(x), -1.0)), eta, prm.caps)
        nr = tucker.norm(r)
        eta = prm.beta_trunc * prm.tol * nf / nr
        z = rounding.t_rel(prec(r), eta, prm.caps)
        beta_k = -tucker.dot(z, q) / xi
        p = rounding.t_rel(tucker.add(z, tucker.scale(p, beta_k)), eta, prm.caps)
        q = rounding.t_rel(A(p), eta, prm.caps)
        xi = tucker.dot(p, q)
        k += 1
        hist.append(nr / nf)
        if record is not None:
            record.append({"k": k, "omega": omega, "beta": beta_k, "xi": xi, "eps": eps, "eta": eta,
                           "rank_x": tucker.ranks(x), "res": nr / nf, "trials": trials})
    return x, {"iters": k, "res": nr / nf, "hist": hist}
