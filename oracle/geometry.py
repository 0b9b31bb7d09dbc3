"""Parametric coefficients of the Poisson problem (App. A, eq. matrix_param / rhs_param).

Oracle module (test infrastructure only).

For a map F: [0,1]^3 -> Omega the stiffness matrix and load vector become integrals over the
parametric cube with Q(eta) = det(J) J^-1 J^-T and omega(eta) = det(J) f(F(eta)).

Geometries (synthetic stand-ins for the paper's domains):
  cube   -- identity map, f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z); with Neumann flags bc = (k0, k1) on the
            faces eta_t = 0 / 1 of every direction, f = 3 w^2 s(x) s(y) s(z) with s(t) = sin(w t + k0 pi/2),
            w = (1 - k0/2 - k1/2) pi, so that u = s(x) s(y) s(z) solves the problem with those conditions
  twist  -- quarter annulus (rho = 1 + eta1 in [1,2], theta = pi/2 eta2) extruded along z = eta3,
            with the cross-section rotated about its centroid c by tau(eta3) = amp sin(pi eta3); f = 1.
"""
from __future__ import annotations

import numpy as np

CENTROID = 28.0 / (9.0 * np.pi)   # centroid (c, c) of {1 <= rho <= 2, 0 <= theta <= pi/2}


def twist_map(e1, e2, e3, amp):
    """F(eta) for the twisted quarter annulus; returns (x, y, z)."""
    rho = 1.0 + e1
    th = 0.5 * np.pi * e2
    tau = amp * np.sin(np.pi * e3)
    px, py = rho * np.cos(th) - CENTROID, rho * np.sin(th) - CENTROID
    c, s = np.cos(tau), np.sin(tau)
    return CENTROID + c * px - s * py, CENTROID + s * px + c * py, e3


def twist_jacobian(e1, e2, e3, amp):
    """Analytic Jacobian J[..., a, b] = dF_a / d eta_b of ``twist_map``."""
    e1, e2, e3 = np.broadcast_arrays(np.asarray(e1, float), np.asarray(e2, float), np.asarray(e3, float))
    rho = 1.0 + e1
    th = 0.5 * np.pi * e2
    tau = amp * np.sin(np.pi * e3)
    dtau = amp * np.pi * np.cos(np.pi * e3)
    c, s = np.cos(tau), np.sin(tau)
    # derivatives of the cross-section point P(rho, theta)
    p1 = (np.cos(th), np.sin(th))                                   # dP/d eta1
    p2 = (-0.5 * np.pi * rho * np.sin(th), 0.5 * np.pi * rho * np.cos(th))   # dP/d eta2
    px, py = rho * np.cos(th) - CENTROID, rho * np.sin(th) - CENTROID
    J = np.zeros(e1.shape + (3, 3))
    for b, (vx, vy) in enumerate((p1, p2)):
        J[..., 0, b] = c * vx - s * vy
        J[..., 1, b] = s * vx + c * vy
    # d/d eta3 of Rot(tau) (P - c) = tau' Rot'(tau) (P - c)
    J[..., 0, 2] = dtau * (-s * px - c * py)
    J[..., 1, 2] = dtau * (c * px - s * py)
    J[..., 2, 2] = 1.0
    return J


def cube_solution_1d(t, bc=(0, 0)):
    """s(t) = sin(w t + k0 pi/2), w = (1 - k0/2 - k1/2) pi: zero at the Dirichlet ends, zero slope at the
    Neumann ends; -s'' = w^2 s."""
    w = (1.0 - 0.5 * (bc[0] + bc[1])) * np.pi
    return np.sin(w * np.asarray(t, float) + 0.5 * np.pi * bc[0]), w


def coefficients(kind: str, amp: float, e1, e2, e3, bc=(0, 0)):
    """Q (shape (..., 3, 3)) and omega (shape (...)) at the parametric points (App. A)."""
    e1, e2, e3 = np.broadcast_arrays(np.asarray(e1, float), np.asarray(e2, float), np.asarray(e3, float))
    if kind == "cube":
        Q = np.zeros(e1.shape + (3, 3))
        Q[..., 0, 0] = Q[..., 1, 1] = Q[..., 2, 2] = 1.0
        s1, w = cube_solution_1d(e1, bc)
        om = 3.0 * w ** 2 * s1 * cube_solution_1d(e2, bc)[0] * cube_solution_1d(e3, bc)[0]
        return Q, om
    if kind == "twist":
        J = twist_jacobian(e1, e2, e3, amp)
        det = np.linalg.det(J)
        Ji = np.linalg.inv(J)
        Q = det[..., None, None] * (Ji @ np.swapaxes(Ji, -1, -2))
        return Q, det * 1.0
    raise ValueError(kind)
