"""Fast-diagonalization preconditioner: exact (Alg. 3), approximate eigenpairs (App. B),
exponential sums (Prop. 1, eq. estimate_prec_rel) and the low-rank application (Alg. 4).

Oracle module (test infrastructure only).  Dense matrices, direct sums for the sine transforms.

Readings:
  * App. B, U1: the columns of V1 U1 are the B-spline coefficients of the interpolant in V_h,1 of
    the L2-normalised sines sqrt(2) sin(j pi x) at the points x_i (one factor sqrt(2)).
  * App. B, V2: V2 = M^{-1} N with N a basis of null(V1^T), which makes span(V2) the
    M-orthogonal complement of V_h,1; U2, Lambda2 solve the projected pencil with U2^T (V2^T M V2) U2 = I.
  * App. B, Neumann ends (flags bc = (k0, k1), 1 = Neumann): V_h keeps the end function; V_h,1 asks the odd
    derivatives <= p - 1 to vanish there (even ones, from order 2, at a Dirichlet end); the end blocks of
    Phi0 / Phi1 hold twice as many functions as their end has conditions (the paper's n2 when both ends
    agree); the sinusoids sin(omega_j x + k0 pi/2), omega_j = (j - k0/2 - k1/2) pi, carry the same single
    L2-normalising factor as the Dirichlet sines.
  * lambda_min / lambda_max (eq. estimate_prec_rel) are sums over the three directions of the
    extreme entries of Lambda~_i, outliers of Lambda2 included.
  * Exponential sums: the paper takes (omega_j, alpha_j) from Hackbusch's tables, which are not
    available.  This oracle uses the sinc-quadrature sums of 1/lambda = int_R exp(s - lambda e^s) ds
    (trapezoidal rule, step h, nodes s_k = s0 + k h), with (h, s0, R) chosen by a search so that
    E_R(M) <= eps_prec / M on a log grid of [1, M] (selection on 400 points, acceptance on 4000);
    R_P is the smallest such R found.
    The search is not a best approximation, so this R_P is larger than the paper's Table 1 values; the
    bound E_R(M_P) M_P <= eps_prec is pinned.  The best sums, whose R_P reproduces Table 1, are in
    oracle/expsum.py; ApproxFD takes them through its `expsum` argument.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import bspline, tucker


# ---------------------------------------------------------------------------------------------
# Exact FD (Alg. 3)
# ---------------------------------------------------------------------------------------------
def exact_eig(n: int, p: int, bc=(0, 0)):
    """Generalized eigendecomposition K U = M U Lambda, U^T M U = I (eq. factorizations)."""
    n_el = bspline.n_el_of(n, p, bc)
    K = bspline.stiffness(n_el, p, bc)
    M = bspline.mass(n_el, p, bc)
    lam, U = scipy.linalg.eigh(K, M)
    return lam, U


def exact_fd_apply_full(n: int, p: int, s: np.ndarray, bc=(0, 0)) -> np.ndarray:
    """v = P^{-1} s for the exact FD preconditioner (eq. factorized_FD), full vectors, tiny n."""
    lam, U = exact_eig(n, p, bc)
    S = tucker.unvec(s, (n, n, n))
    T = S
    for m in range(3):
        T = tucker.mode_product(T, U.T, m)
    D = lam[:, None, None] + lam[None, :, None] + lam[None, None, :]
    T = T / D
    for m in range(3):
        T = tucker.mode_product(T, U, m)
    return tucker.vec(T)


# ---------------------------------------------------------------------------------------------
# Approximate eigenpairs (App. B)
# ---------------------------------------------------------------------------------------------
def end_orders(p: int, k: int):
    """Derivative orders that vanish at one end for functions of V_h,1 (App. B): the even orders 2, 4, ..
    <= p - 1 at a Dirichlet end (k = 0; order 0 is the space's own condition), the odd orders 1, 3, ..
    <= p - 1 at a Neumann end (k = 1)."""
    first = 2 if k == 0 else 1
    return list(range(first, p, 2))


def split_dims(n_el: int, p: int, bc=(0, 0)):
    """(n1, n2) of the splitting V_h = V_h,1 (+) V_h,2 (App. B): every vanishing derivative at an end removes
    one dimension from V_h (n = n_el + p - 2 + k0 + k1)."""
    n = n_el + p - 2 + bc[0] + bc[1]
    c = len(end_orders(p, bc[0])) + len(end_orders(p, bc[1]))
    return n - c, c


def interpolation_points(n_el: int, p: int, bc=(0, 0)) -> np.ndarray:
    """Breakpoints, without the ends that carry a Dirichlet condition (odd p), or span midpoints (even p)."""
    if p % 2 == 1:
        return np.arange(1 - bc[0], n_el + bc[1]) / n_el
    return (np.arange(1, n_el + 1) - 0.5) / n_el


def sine_frequencies(n1: int, bc=(0, 0)) -> np.ndarray:
    """omega_j = (j - k0/2 - k1/2) pi, j = 1..n1: the sinusoids of App. B (the plain sines j pi when no end
    carries a Neumann condition)."""
    return (np.arange(1, n1 + 1) - 0.5 * (bc[0] + bc[1])) * np.pi


def sine_matrix(x: np.ndarray, n1: int, bc=(0, 0)) -> np.ndarray:
    """U_dft[l, j] = c_j sin(omega_j x_l + k0 pi/2) with c_j the L2 normalisation on [0, 1] (sqrt2, or 1 for
    the constant of two Neumann ends)."""
    w = sine_frequencies(n1, bc)
    c = np.where(w == 0.0, 1.0, np.sqrt(2.0))
    return c * np.sin(np.outer(x, w) + 0.5 * np.pi * bc[0])


def _nullspace(A: np.ndarray) -> np.ndarray:
    if A.shape[0] == 0:
        return np.eye(A.shape[1])
    return scipy.linalg.null_space(A)


def v1_basis(n_el: int, p: int, bc=(0, 0)) -> np.ndarray:
    """V1 (n x n1): columns Phi0 | Phi | Phi1 spanning V_h,1 (eq. Phi0, eq. Phi1).  Phi0 (Phi1) is the part
    of the span of the first (last) 2 c functions that meets the c conditions of its end; the functions in
    between are taken one by one.  With equal ends 2 c = n2, the paper's blocks."""
    n = n_el + p - 2 + bc[0] + bc[1]
    n1, _ = split_dims(n_el, p, bc)
    o0, o1 = end_orders(p, bc[0]), end_orders(p, bc[1])
    a, b = 2 * len(o0), 2 * len(o1)
    V1 = np.zeros((n, n1))
    col = 0
    if o0:
        D0 = np.array([bspline.bc_basis(n_el, p, np.array([0.0]), d, bc)[:a, 0] for d in o0])
        Z0 = _nullspace(D0)
        V1[:a, :Z0.shape[1]] = Z0
        col = Z0.shape[1]
    for i in range(a, n - b):
        V1[i, col] = 1.0
        col += 1
    if o1:
        D1 = np.array([bspline.bc_basis(n_el, p, np.array([1.0]), d, bc)[n - b:, 0] for d in o1])
        Z1 = _nullspace(D1)
        V1[n - b:, col:col + Z1.shape[1]] = Z1
        col += Z1.shape[1]
    assert col == n1
    return V1


def approx_eig(n: int, p: int, bc=(0, 0)):
    """U~ (n x n) and Lambda~ (n) of App. B, built from their definitions with dense matrices."""
    n_el = bspline.n_el_of(n, p, bc)
    n1, n2 = split_dims(n_el, p, bc)
    M = bspline.mass(n_el, p, bc)
    K = bspline.stiffness(n_el, p, bc)
    V1 = v1_basis(n_el, p, bc)
    x = interpolation_points(n_el, p, bc)
    E = bspline.bc_basis(n_el, p, x, 0, bc).T             # E[l, a] = b_a(x_l)
    Cint = E @ V1                                          # Cint[l, i] = v_i(x_l)
    Udft = sine_matrix(x, n1, bc)
    U1 = np.linalg.solve(Cint, Udft)                       # interpolation: Cint c = f(x)
    lam1 = sine_frequencies(n1, bc) ** 2
    parts = [V1 @ U1]
    lams = [lam1]
    if n2 > 0:
        N = _nullspace(V1.T)                               # n x n2
        V2 = np.linalg.solve(M, N)
        lam2, U2 = scipy.linalg.eigh(V2.T @ K @ V2, V2.T @ M @ V2)
        parts.append(V2 @ U2)
        lams.append(lam2)
    return np.concatenate(parts, axis=1), np.concatenate(lams)


def sine_symbol(n_el: int, p: int, bc=(0, 0)) -> np.ndarray:
    """mu_j = sum over the interpolation lattice of B(x_l - c) cos(omega_j (x_l - c)) for a B-spline b with
    centre c whose local knots are uniform: the factor by which collocating the uniform spline with
    coefficients sin(omega_j c_i + phi) multiplies the samples sin(omega_j x_l + phi) (B is symmetric)."""
    n1, _ = split_dims(n_el, p, bc)
    x = interpolation_points(n_el, p, bc)
    kn = bspline.open_uniform_knots(n_el, p)
    f0 = (p + n_el - 1) // 2                     # full index of a function with distinct local knots
    c0 = 0.5 * (kn[f0] + kn[f0 + p + 1])
    vals = bspline.basis(kn, p, x)[f0]
    return np.cos(np.outer(sine_frequencies(n1, bc), x - c0)) @ vals


def sine_factorization(n: int, p: int, bc=(0, 0)):
    """(W, mu) with V1 U1 = W U_dft diag(1/mu): the App. B eigenvector block written as a sparse
    boundary correction W (n x n1) of the scaled sine transform.  Dense construction:
    W = (V1 U1) diag(mu) U_dft^{-1}; entries below 1e-11 max|W| are dropped."""
    n_el = bspline.n_el_of(n, p, bc)
    n1, _ = split_dims(n_el, p, bc)
    U, _ = approx_eig(n, p, bc)
    x = interpolation_points(n_el, p, bc)
    Udft = sine_matrix(x, n1, bc)
    mu = sine_symbol(n_el, p, bc)
    W = np.linalg.solve(Udft.T, (U[:, :n1] * mu).T).T
    W[np.abs(W) < 1e-11 * np.abs(W).max()] = 0.0
    return W, mu, Udft


def mp_value(n: int, p: int, bc=(0, 0)) -> float:
    """M_P = lambda_max / lambda_min (eq. estimate_prec_rel) for the same n, p in all directions."""
    _, lam = approx_eig(n, p, bc)
    return (3.0 * lam.max()) / (3.0 * lam.min())


def mp_value_fast(n_el: int, p: int, bc=(0, 0)) -> float:
    """M_P from Lambda1 = omega_j^2 and the small pencil on V_h,2 only (no dense U1)."""
    n1, n2 = split_dims(n_el, p, bc)
    w = sine_frequencies(n1, bc)
    lam = [w[0] ** 2, w[-1] ** 2]
    if n2 > 0:
        M = bspline.mass(n_el, p, bc)
        K = bspline.stiffness(n_el, p, bc)
        V1 = v1_basis(n_el, p, bc)
        N = _nullspace(V1.T)
        V2 = np.linalg.solve(M, N)
        lam2 = scipy.linalg.eigh(V2.T @ K @ V2, V2.T @ M @ V2, eigvals_only=True)
        lam += list(lam2)
    return max(lam) / min(lam)


# ---------------------------------------------------------------------------------------------
# Exponential sums (Prop. 1)
# ---------------------------------------------------------------------------------------------
def expsum_error(omega, alpha, M: float, npts: int = 4000) -> float:
    """E_R(M) = sup_{lambda in [1, M]} |1/lambda - sum_j omega_j exp(-alpha_j lambda)| on a log grid."""
    lam = np.exp(np.linspace(0.0, np.log(M), npts))
    s = np.exp(-np.outer(lam, alpha)) @ omega
    return float(np.max(np.abs(1.0 / lam - s)))


def sinc_expsum(R: int, h: float, s0: float):
    """Trapezoidal rule for 1/lambda = int exp(s - lambda e^s) ds with nodes s0 + k h, k < R."""
    s = s0 + h * np.arange(R)
    return h * np.exp(s), np.exp(s)


def expsum_for(M: float, eps_prec: float, rmax: int = 80):
    """Smallest R (and its omega, alpha) with E_R(M) <= eps_prec / M found by a grid search of (h, s0)."""
    target = eps_prec / M
    for R in range(1, rmax + 1):
        best = None
        for h in np.linspace(0.15, 1.6, 30):
            top = np.log(np.log(1.0 / target) + 2.0) + 0.5
            for s0 in np.linspace(top - h * (R - 1) - 2.0, top - h * (R - 1) + 1.0, 13):
                om, al = sinc_expsum(R, h, s0)
                e = expsum_error(om, al, M, 400)
                if best is None or e < best[0]:
                    best = (e, om, al)
        if best[0] <= target:
            om, al = best[1], best[2]
            if expsum_error(om, al, M) <= target:
                return R, om, al
    raise RuntimeError("no exponential sum found")


# ---------------------------------------------------------------------------------------------
# Low-rank FD application (Alg. 4)
# ---------------------------------------------------------------------------------------------
class ApproxFD:
    """Setup of Alg. 4 for n dofs, degree p and boundary conditions bc in every direction.  bc = (1, 1) (Neumann
    at both ends of every direction) is rejected: its Kronecker sum has the constant in its kernel."""

    def __init__(self, n: int, p: int, eps_prec: float = 0.1, expsum=None, bc=(0, 0)):
        if tuple(bc) == (1, 1):
            raise ValueError("Neumann at both ends of every direction: singular operator")
        self.n, self.p, self.bc = n, p, tuple(bc)
        self.U, self.lam = approx_eig(n, p, bc)
        self.lmin = 3.0 * self.lam.min()
        self.lmax = 3.0 * self.lam.max()
        self.MP = self.lmax / self.lmin
        if expsum is None:
            self.RP, self.omega, self.alpha = expsum_for(self.MP, eps_prec)
        else:
            self.omega, self.alpha = np.asarray(expsum[0]), np.asarray(expsum[1])
            self.RP = len(self.omega)

    def diag(self, j: int) -> np.ndarray:
        """Diagonal of D_(i,j), eq. diag_factor."""
        return np.exp(-self.alpha[j] / self.lmin * self.lam)

    def apply(self, S):
        """Alg. 4, steps 5-9: core P (x) S (block form) and factors [U~ D_(i,1) U~^T S_i, ..., U~ D_(i,R_P) U~^T S_i]."""
        core, F = S
        V = tucker.superdiag_kron(self.omega / self.lmin, core)
        facs = []
        for m in range(3):
            Z = self.U.T @ F[m]
            facs.append(np.concatenate([self.U @ (self.diag(j)[:, None] * Z) for j in range(self.RP)], axis=1))
        return V, facs
