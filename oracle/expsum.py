"""Best exponential sums for 1/lambda on [1, M] (Prop. 1, eq. estimate_approx_diag) and the preconditioner
rank R_P of eq. estimate_prec_rel.

Test infrastructure: only tests/, __graft_entry__.smoke() and bench.py's CPU baseline use the oracle.

The paper takes omega_j, alpha_j and E_R(M) from published tables, which are not available here. This module
computes the best approximation itself:

* In the maximum norm on [1, M], 1/lambda has a unique best approximation s_R(lambda) = sum_j omega_j
  exp(-alpha_j lambda) with R terms. It is characterised by equioscillation: the error 1/lambda - s_R(lambda)
  reaches its largest modulus E_R(M) at 2R + 1 points, with alternating signs (the alternation theorem for
  exponential sums; D. Braess, Nonlinear Approximation Theory, Springer 1986).
* It is found with the Remez exchange algorithm. Given 2R + 1 trial points x_0 < ... < x_2R, the 2R + 1
  equations 1/x_i - s(x_i) = (-1)^i E are solved for (alpha, omega, E) by Newton's method. The unknowns are
  log alpha and log omega, which keeps both positive. The trial points are then replaced by the alternating
  extrema of the new error, and the two steps repeat until the largest error equals |E|.
* The exchange needs a start whose error already alternates 2R + 1 times. It comes from a weighted
  least-squares fit on a logarithmic grid, reweighted a few times towards the maximum norm (Lawson's
  iteration); when the exchange does not converge from it, a longer and more heavily reweighted fit is
  the second start. Both fits start from the (R - 1)-term best sum, its log alpha / log omega profile
  stretched to R terms; R = 1 starts from omega = alpha = 1/2.

R_P = min{R : E_R(M_P) <= eps_prec / M_P} (eq. estimate_prec_rel) is then found by increasing R.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import least_squares


def error(lam, omega, alpha):
    """1/lambda - s_R(lambda) at the points lam."""
    lam = np.asarray(lam, dtype=float)
    return 1.0 / lam - np.exp(-np.outer(lam, alpha)) @ omega


def _grid(M: float, npts: int) -> np.ndarray:
    return np.exp(np.linspace(0.0, np.log(M), npts))


def alternants(omega, alpha, M: float, npts: int = 60000):
    """The alternating extrema of the error on a fine logarithmic grid of [1, M]: the points, the error values
    there, and the largest error modulus on the grid.  Neighbouring extrema of the same sign are merged into
    the larger one, so consecutive entries alternate in sign."""
    x = _grid(M, npts)
    e = error(x, omega, alpha)
    d = np.diff(e)
    idx = [0] + list(np.nonzero(d[:-1] * d[1:] <= 0)[0] + 1) + [npts - 1]
    keep: list[int] = []
    for i in idx:
        if keep and np.sign(e[i]) == np.sign(e[keep[-1]]):
            if abs(e[i]) > abs(e[keep[-1]]):
                keep[-1] = i
        else:
            keep.append(i)
    return x[keep], e[keep], float(np.max(np.abs(e)))


def _solve_levelled(pts, omega, alpha, E, it: int = 80):
    """Newton's method for 1/x_i - s(x_i) = sign_i E, i = 0..2R, in (log alpha, log omega, E), with step
    halving on the residual norm."""
    R = len(alpha)
    sign = np.sign(error(pts[:1], omega, alpha))[0] * (-1.0) ** np.arange(len(pts))
    u = np.concatenate([np.log(alpha), np.log(omega), [abs(E)]])

    def resid(v):
        return 1.0 / pts - np.exp(-np.outer(pts, np.exp(v[:R]))) @ np.exp(v[R:2 * R]) - sign * v[2 * R]

    for _ in range(it):
        a, o = np.exp(u[:R]), np.exp(u[R:2 * R])
        A = np.exp(-np.outer(pts, a))
        f = resid(u)
        J = np.empty((len(pts), 2 * R + 1))
        J[:, :R] = A * (o * a)[None, :] * pts[:, None]     # d/d log alpha_j of -omega_j exp(-alpha_j x)
        J[:, R:2 * R] = -A * o[None, :]                    # d/d log omega_j
        J[:, 2 * R] = -sign
        du = np.linalg.lstsq(J, -f, rcond=None)[0]
        step, f0 = 1.0, np.linalg.norm(f)
        while step > 1e-6 and not np.linalg.norm(resid(u + step * du)) < f0:
            step *= 0.5
        u = u + step * du
        if np.linalg.norm(step * du) < 1e-14 * (1.0 + np.linalg.norm(u)):
            break
    return np.exp(u[R:2 * R]), np.exp(u[:R]), float(u[2 * R])


def remez(M: float, omega, alpha, iters: int = 60):
    """Remez exchange from a start (omega, alpha) whose error alternates at least 2R + 1 times on [1, M].
    Returns (omega, alpha, E_R(M), converged); converged means the largest error equals the levelled |E|."""
    R = len(alpha)
    E = None
    emax = float("inf")
    for _ in range(iters):
        pts, ev, emax = alternants(omega, alpha, M)
        if len(pts) < 2 * R + 1:
            return omega, alpha, emax, False
        if len(pts) > 2 * R + 1:   # keep 2R + 1 consecutive alternants, dropping the smaller ends
            lo, hi = 0, len(pts)
            while hi - lo > 2 * R + 1:
                if abs(ev[lo]) < abs(ev[hi - 1]):
                    lo += 1
                else:
                    hi -= 1
            pts, ev = pts[lo:hi], ev[lo:hi]
        if E is None:
            E = float(np.mean(np.abs(ev)))
        omega, alpha, E = _solve_levelled(pts, omega, alpha, E)
        _, _, emax = alternants(omega, alpha, M)
        if emax <= abs(E) * (1.0 + 1e-8):
            return omega, alpha, emax, True
    return omega, alpha, emax, False


def _least_squares_start(M: float, omega, alpha, npts: int = 800, lawson: int = 2):
    """Weighted least squares of 1/lambda - s(lambda) on a log grid, reweighted towards the maximum norm."""
    R = len(alpha)
    x = _grid(M, npts)
    w = np.ones(npts)
    lo = np.concatenate([np.full(R, np.log(0.01 / M)), np.full(R, -40.0)])
    hi = np.concatenate([np.full(R, np.log(200.0)), np.full(R, 10.0)])
    u = np.clip(np.concatenate([np.log(alpha), np.log(omega)]), lo + 1e-9, hi - 1e-9)
    for _ in range(lawson + 1):
        def resid(v, w=w):
            return w * (1.0 / x - np.exp(-np.outer(x, np.exp(v[:R]))) @ np.exp(v[R:]))

        def jac(v, w=w):
            a, o = np.exp(v[:R]), np.exp(v[R:])
            A = np.exp(-np.outer(x, a))
            J = np.empty((npts, 2 * R))
            J[:, :R] = A * (o * a)[None, :] * x[:, None]
            J[:, R:] = -A * o[None, :]
            return w[:, None] * J

        u = least_squares(resid, u, jac=jac, bounds=(lo, hi), method="trf", xtol=1e-15, ftol=1e-15,
                          gtol=1e-15, max_nfev=3000).x
        e = error(x, np.exp(u[R:]), np.exp(u[:R]))
        w = w * np.sqrt(np.abs(e))
        w = np.maximum(w / w.max(), 1e-3)
    return np.exp(u[R:]), np.exp(u[:R])


def _stretch(omega, alpha):
    """R terms -> R + 1 terms: log alpha and log omega, sorted by alpha, interpolated over the term index."""
    o = np.argsort(alpha)
    la, lw = np.log(alpha[o]), np.log(omega[o])
    R = len(alpha)
    t0, t1 = np.linspace(0.0, 1.0, R), np.linspace(0.0, 1.0, R + 1)
    return np.exp(np.interp(t1, t0, lw)), np.exp(np.interp(t1, t0, la))


def best_sums(M: float, rmax: int, stop=None):
    """Best sums for R = 1, 2, ... on [1, M] by continuation in R; yields (R, omega, alpha, E_R(M), converged).
    Stops after rmax terms, or after the first R for which stop(E) holds."""
    omega, alpha = np.array([0.5]), np.array([0.5])
    for R in range(1, rmax + 1):
        if R > 1:
            omega, alpha = _stretch(omega, alpha)
        o1, a1 = _least_squares_start(M, omega, alpha)
        o1, a1, E, ok = remez(M, o1, a1)
        if not ok:   # a start that did not lead to equioscillation: a longer, more heavily reweighted fit
            o1, a1 = _least_squares_start(M, omega, alpha, npts=4000, lawson=6)
            o1, a1, E, ok = remez(M, o1, a1)
        omega, alpha = o1, a1
        yield R, omega, alpha, E, ok
        if stop is not None and stop(E):
            return


def best_expsum(R: int, M: float):
    """The best R-term sum on [1, M]: (omega, alpha, E_R(M), converged)."""
    out = None
    for out in best_sums(M, R):
        pass
    return out[1], out[2], out[3], out[4]


def rp_best(M: float, eps_prec: float = 0.1, rmax: int = 60):
    """eq. estimate_prec_rel with best sums: (R_P, omega, alpha, E_{R_P}(M), E_{R_P - 1}(M))."""
    prev = np.inf
    for R, omega, alpha, E, ok in best_sums(M, rmax, stop=lambda E: E <= eps_prec / M):
        if E <= eps_prec / M:
            return R, omega, alpha, E, prev
        prev = E
    raise RuntimeError("rp_best: no R <= rmax meets the bound")
