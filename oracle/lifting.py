"""Non-homogeneous Dirichlet conditions by lifting (the Remark in Sec. 3).

Oracle module (test infrastructure only).

With u = g on the boundary, the discrete solution is u_h = sum_i c_i B_i + w_h, where B_i runs over the whole
B-spline basis (boundary functions included), c are the coefficients of an approximation of g, and w_h
vanishes on the boundary.  Testing with the functions that vanish on the boundary gives the homogeneous
system of eq. approx_ls with the right-hand side f~ - A~_dOmega g~: A~_dOmega is the operator between the
interior test functions and the boundary trial functions, g~ the boundary coefficients of c.

Readings:
  * g~ comes from the L2 projection, on the parametric cube, of a smooth extension G of g (G composed with
    the map, sampled on the Chebyshev grid and compressed as the coefficients of App. A are); only its
    boundary coefficients enter (the interior ones are what w_h solves for);
  * A~_dOmega g~ = A~_(I,all) c - A~_(I,I) c_I: the operator with trial functions on the whole basis applied to
    c, minus the homogeneous operator applied to c's interior coefficients.  Both are Tucker products
    (eq. tt_product), so the corrected right-hand side stays in Tucker format.
"""
from __future__ import annotations

import numpy as np

from . import bspline, geometry, lowrank, rounding, tucker


def physical_points(kind: str, amp: float, e1, e2, e3):
    """F(eta) for the geometries of geometry.py."""
    if kind == "cube":
        return e1, e2, e3
    if kind == "twist":
        return geometry.twist_map(e1, e2, e3, amp)
    raise ValueError(kind)


def projection_coefficients(G, kind: str, amp: float, n: int, p: int, eps: float = 1e-10):
    """Tucker coefficients (core, [C_t]) with C_t of size (n + 2) x r_t: the L2 projection on the parametric
    cube of G(F(eta)) onto the full tensor B-spline space (boundary functions included)."""
    n_el = n - p + 2
    xc = lowrank.cheb_points()
    e1, e2, e3 = np.meshgrid(xc, xc, xc, indexing="ij")
    core, U = lowrank.tucker_of_samples(G(*physical_points(kind, amp, e1, e2, e3)), eps)
    xs, ws = bspline.quadrature(n_el, p)
    Bf = bspline.basis(bspline.open_uniform_knots(n_el, p), p, xs, 0)     # (n + 2) x nq
    M = (Bf * ws) @ Bf.T
    C = [np.linalg.solve(M, (Bf * ws) @ lowrank.cheb_eval(U[t], xs)) for t in range(3)]
    return core, C


def rhs_of(fun, kind: str, amp: float, n: int, p: int, eps: float = 1e-10):
    """Tucker load vector of det J * fun(F(eta)) against the interior basis (as rhs_tucker does for the
    geometries' own f)."""
    n_el = n - p + 2
    xc = lowrank.cheb_points()
    e1, e2, e3 = np.meshgrid(xc, xc, xc, indexing="ij")
    _, om = geometry.coefficients(kind, amp, e1, e2, e3)         # det J (times the geometry's own f)
    det = om if kind == "twist" else np.ones_like(e1)
    core, U = lowrank.tucker_of_samples(det * fun(*physical_points(kind, amp, e1, e2, e3)), eps)
    xs, ws = bspline.quadrature(n_el, p)
    B0 = bspline.dirichlet_basis(n_el, p, xs, 0)
    return core, [(B0 * ws) @ lowrank.cheb_eval(U[t], xs) for t in range(3)]


def interior(c):
    """The interior coefficients of a full-basis Tucker tensor (boundary rows of every factor removed)."""
    core, C = c
    return core, [Ct[1:-1] for Ct in C]


def lifted_rhs(terms_full, terms, f, c, eps: float = 1e-12):
    """f~ - A~_dOmega g~ = f~ - A~_(I,all) c + A~_(I,I) c_I, rounded by Alg. 1 to relative accuracy eps."""
    y = tucker.add(f, tucker.scale(tucker.matvec(terms_full, c), -1.0))
    y = tucker.add(y, tucker.matvec(terms, interior(c)))
    return rounding.t_rel(y, eps)


def full_solution(c, x):
    """Full-basis coefficients of u_h: c on the boundary, x on the interior, i.e. u = c + E(x - c_I) with E the
    extension by zero boundary rows (every index whose three entries are all interior is an interior dof)."""
    xc, X = tucker.add(x, tucker.scale(interior(c), -1.0))
    pad = [np.vstack([np.zeros((1, Xt.shape[1])), Xt, np.zeros((1, Xt.shape[1]))]) for Xt in X]
    return tucker.add(c, (xc, pad))
