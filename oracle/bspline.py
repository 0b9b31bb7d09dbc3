"""Univariate B-splines and the 1-D Galerkin matrices (Sec. 2.1, Sec. 2.2, App. A).

Oracle module (test infrastructure only).  Dense arrays throughout; obviously-correct forms
of the Cox-de Boor recursion, not the element-local algorithm the CUDA library's host setup uses.
"""
from __future__ import annotations

import numpy as np

QUAD_EXTRA = 3   # Gauss-Legendre points per knot span = p + QUAD_EXTRA


def open_uniform_knots(n_el: int, p: int) -> np.ndarray:
    """Open knot vector on [0,1] with n_el uniform spans: 0 and 1 repeated p+1 times (Sec. 2.1)."""
    inner = np.arange(1, n_el) / n_el
    return np.concatenate([np.zeros(p + 1), inner, np.ones(p + 1)])


def _div(a, b):
    """a / b with the convention 0/0 = 0 used by the recursion (Sec. 2.1)."""
    return np.where(b == 0.0, 0.0, a / np.where(b == 0.0, 1.0, b))


def basis(knots: np.ndarray, p: int, x: np.ndarray, der: int = 0) -> np.ndarray:
    """All B-splines of degree p (or their ``der``-th derivative) at the points x.

    Returns B with B[i, k] = d^der/dx^der b_i^(p)(x_k), i = 0..m-1 (m = len(knots) - p - 1).
    Degree 0: indicator of [xi_i, xi_{i+1}) (the last non-empty span is closed at 1).
    Degree p: Cox-de Boor recursion of Sec. 2.1.  Derivatives: d/dx b_{i,p} =
    p b_{i,p-1}/(xi_{i+p}-xi_i) - p b_{i+1,p-1}/(xi_{i+p+1}-xi_{i+1}) (de Boor).
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    t = knots
    if p == 0:
        nb = len(t) - 1
        B = np.zeros((nb, x.size))
        last = np.max(np.nonzero(t[1:] > t[:-1])[0])
        for i in range(nb):
            B[i] = (t[i] <= x) & (x < t[i + 1])
            if i == last:
                B[i] = np.logical_or(B[i] > 0, x == t[i + 1])
        if der > 0:
            return np.zeros_like(B)
        return B
    lower = basis(t, p - 1, x, der - 1 if der > 0 else 0)
    nb = len(t) - p - 1
    B = np.zeros((nb, x.size))
    for i in range(nb):
        d1 = t[i + p] - t[i]
        d2 = t[i + p + 1] - t[i + 1]
        if der == 0:
            B[i] = _div(x - t[i], d1) * lower[i] + _div(t[i + p + 1] - x, d2) * lower[i + 1]
        else:
            B[i] = p * (_div(lower[i], d1) - _div(lower[i + 1], d2))
    return B


def quadrature(n_el: int, p: int):
    """Gauss-Legendre points and weights on every knot span of [0,1] (p + QUAD_EXTRA per span)."""
    q = p + QUAD_EXTRA
    g, w = np.polynomial.legendre.leggauss(q)
    a = np.arange(n_el)[:, None] / n_el
    h = 1.0 / n_el
    xs = (a + (g[None, :] + 1.0) * 0.5 * h).ravel()
    ws = np.tile(w * 0.5 * h, n_el)
    return xs, ws


def dirichlet_basis(n_el: int, p: int, x: np.ndarray, der: int = 0) -> np.ndarray:
    """The n = n_el + p - 2 B-splines vanishing at 0 and 1 (drop first and last, Sec. 2.2)."""
    B = basis(open_uniform_knots(n_el, p), p, x, der)
    return B[1:-1]


def bc_basis(n_el: int, p: int, x: np.ndarray, der: int = 0, bc=(0, 0)) -> np.ndarray:
    """The B-splines of the space with the boundary conditions bc = (k0, k1) at 0 and 1 (App. B's flags:
    1 = Neumann, 0 = Dirichlet).  A Dirichlet end drops the one function that does not vanish there (Sec.
    2.2); a Neumann end keeps it (natural condition).  n = n_el + p - 2 + k0 + k1 functions."""
    k0, k1 = bc
    B = basis(open_uniform_knots(n_el, p), p, x, der)
    return B[(0 if k0 else 1):(B.shape[0] if k1 else B.shape[0] - 1)]


def n_el_of(n: int, p: int, bc=(0, 0)) -> int:
    """Knot spans of the space with n functions, degree p and boundary conditions bc."""
    return n - p + 2 - bc[0] - bc[1]


def weighted_matrix(n_el: int, p: int, di: int, dj: int, g=None, bc=(0, 0)) -> np.ndarray:
    """C[i,j] = int_0^1 b_i^(di) b_j^(dj) g dx over the basis of bc (App. A, matrices C)."""
    xs, ws = quadrature(n_el, p)
    Bi = bc_basis(n_el, p, xs, di, bc)
    Bj = bc_basis(n_el, p, xs, dj, bc)
    gw = ws if g is None else ws * g(xs)
    return (Bi * gw) @ Bj.T


def mass(n_el: int, p: int, bc=(0, 0)) -> np.ndarray:
    return weighted_matrix(n_el, p, 0, 0, bc=bc)


def stiffness(n_el: int, p: int, bc=(0, 0)) -> np.ndarray:
    return weighted_matrix(n_el, p, 1, 1, bc=bc)
