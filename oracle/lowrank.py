"""Low-rank (Tucker) approximation of the system matrix and right-hand side (App. A).

Oracle module (test infrastructure only).

The paper runs chebfun3f; it is not available, so this oracle follows the same idea in its
own plain form: sample each coefficient on a tensor Chebyshev grid, compress the samples with
ST-HOSVD to relative tolerance eps, and read the factor columns as values of univariate
Chebyshev interpolants (App. A, eq. approxQ / approxW).  The 1-D matrices are

    [C^{(k,l)}_{(t,r)}]_{ij} = int_0^1 delta^{(l,t)}(b_i) delta^{(k,t)}(b_j) u^{(k,l)}_{t,r}(eta) d eta

(App. A, eq. matrix_CP).  Each block's Tucker core is folded along its largest-rank mode into
a Kronecker sum  A~ = sum_j w_j K3^j (x) K2^j (x) K1^j  (reading of eq. matrix_CP as a sum of
rank-one Kronecker terms), which is the operator form the solver consumes.
"""
from __future__ import annotations

import numpy as np

from . import bspline, geometry
from .rounding import sthosvd

N_CHEB = 33   # Chebyshev points per direction for the coefficient samples


def cheb_points(N: int = N_CHEB) -> np.ndarray:
    """Chebyshev points of the second kind mapped to [0,1]."""
    return 0.5 * (1.0 - np.cos(np.pi * np.arange(N) / (N - 1)))


def cheb_eval(values: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Evaluate the polynomial interpolant through (cheb_points, values) at x.

    Plain form: solve for the Chebyshev coefficients c with sum_k c_k T_k(2 x_j - 1) = values_j,
    then sum the series.  ``values`` may have trailing columns.
    """
    N = values.shape[0]
    xc = cheb_points(N)
    V = np.polynomial.chebyshev.chebvander(2.0 * xc - 1.0, N - 1)
    coef = np.linalg.solve(V, values)
    return np.polynomial.chebyshev.chebval(2.0 * x - 1.0, coef).T if values.ndim > 1 else \
        np.polynomial.chebyshev.chebval(2.0 * x - 1.0, coef)


def sample(kind: str, amp: float, N: int = N_CHEB, bc=(0, 0)):
    """Q[k,l] and omega sampled on the N^3 Chebyshev grid; arrays indexed [i1, i2, i3]."""
    xc = cheb_points(N)
    e1, e2, e3 = np.meshgrid(xc, xc, xc, indexing="ij")
    Q, om = geometry.coefficients(kind, amp, e1, e2, e3, bc)
    return Q, om


def tucker_of_samples(T: np.ndarray, eps: float):
    """ST-HOSVD of a sample tensor; returns (core, [U1, U2, U3]) with U_t the factor columns."""
    core, S, _ = sthosvd(T, eps)
    return core, S


def operator_terms(kind: str, amp: float, n: int, p: int, eps: float = 1e-8, trial: str = "dirichlet", bc=(0, 0)):
    """Kronecker-sum operator: list of (w, [K1, K2, K3]) with dense n x n matrices.

    A~ = sum_j w_j K3^j (x) K2^j (x) K1^j acts on vec(X) with mode 1 fastest (Sec. 2.3).
    With trial="full" the trial functions run over the whole B-spline basis (boundary functions included):
    the matrices are n x (n + 2), the operator between the interior test functions and all trial functions
    that the non-homogeneous Dirichlet problem of the Remark in Sec. 3 needs.  bc = (k0, k1) marks Neumann ends
    (the same in every direction): their end functions stay in the test and trial spaces.
    """
    n_el = bspline.n_el_of(n, p, bc)
    Q, _ = sample(kind, amp)
    xs, ws = bspline.quadrature(n_el, p)
    B0 = bspline.bc_basis(n_el, p, xs, 0, bc)
    B1 = bspline.bc_basis(n_el, p, xs, 1, bc)
    knots = bspline.open_uniform_knots(n_el, p)
    T0 = bspline.basis(knots, p, xs, 0) if trial == "full" else B0
    T1 = bspline.basis(knots, p, xs, 1) if trial == "full" else B1
    norms = np.array([[np.linalg.norm(Q[..., k, l]) for l in range(3)] for k in range(3)])
    terms = []
    for k in range(3):
        for l in range(3):
            if norms[k, l] <= 1e-13 * norms.max():
                continue
            core, U = tucker_of_samples(Q[..., k, l], eps)
            R = core.shape
            # fold the mode with the largest rank (ties: the highest mode index)
            mstar = max(range(3), key=lambda t: (R[t], t))
            others = [t for t in range(3) if t != mstar]
            g = [cheb_eval(U[t], xs) for t in range(3)]     # (nq, R_t) values at quadrature points
            for a in range(R[others[0]]):
                for b in range(R[others[1]]):
                    idx = [slice(None)] * 3
                    idx[others[0]] = a
                    idx[others[1]] = b
                    h = g[mstar] @ core[tuple(idx)]
                    funcs = {others[0]: g[others[0]][:, a], others[1]: g[others[1]][:, b], mstar: h}
                    mats = []
                    for t in range(3):
                        Bi = B1 if t == l else B0     # delta^{(l,t)} acts on the test function b_i
                        Bj = T1 if t == k else T0     # delta^{(k,t)} acts on the trial function b_j
                        mats.append((Bi * (ws * funcs[t])) @ Bj.T)
                    terms.append((1.0, mats))
    return terms


def rhs_tucker(kind: str, amp: float, n: int, p: int, eps: float = 1e-8, bc=(0, 0)):
    """Tucker rhs f~: core W and factors [F_t]_{ij} = int b_i u_{t,j} (App. A)."""
    n_el = bspline.n_el_of(n, p, bc)
    _, om = sample(kind, amp, bc=bc)
    core, U = tucker_of_samples(om, eps)
    xs, ws = bspline.quadrature(n_el, p)
    B0 = bspline.bc_basis(n_el, p, xs, 0, bc)
    F = [(B0 * ws) @ cheb_eval(U[t], xs) for t in range(3)]
    return core, F


def cube_terms(n: int, p: int, bc=(0, 0)):
    """The exact unit-cube operator K(x)M(x)M + M(x)K(x)M + M(x)M(x)K (eq. FD_prec with Q = I)."""
    n_el = bspline.n_el_of(n, p, bc)
    M = bspline.mass(n_el, p, bc)
    K = bspline.stiffness(n_el, p, bc)
    return [(1.0, [K, M, M]), (1.0, [M, K, M]), (1.0, [M, M, K])]
