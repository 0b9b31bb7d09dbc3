"""Compressible linear elasticity in Tucker format (Sec. 5.3): 3 x 3 block operator, block right-hand side,
block-diagonal FD preconditioner, and Alg. 5 on block vectors.

Oracle module (test infrastructure only).

Bilinear form (eq. bil_lin): b(u, v) = 2 mu int eps(u) : eps(v) + lambda int div u div v.  On the parametric
cube with F the geometry map, J[a, b] = dF_a / d eta_b and G = J^-1, the trial function phi e_j and the test
function psi e_i give

    b = sum_{k,l} int C^{ij}_{kl}(eta) d_k phi d_l psi d eta,
    C^{ij}_{kl} = det(J) [ mu delta_ij (G G^T)_{kl} + mu G_{ki} G_{lj} + lambda G_{kj} G_{li} ],

(k: derivative of the trial function, l: derivative of the test function), which for i = j and the identity map
reduces to the Poisson coefficient mu I plus (lambda + mu) e_i e_i^T.  Each C^{ij}_{kl} is approximated and
folded into Kronecker terms exactly as the Poisson coefficient Q_{kl} (App. A, ``lowrank``), so every block
A_ij is a Kronecker sum.  Block vectors are lists of three Tucker tensors; products, sums, scalar products and
truncations act block-wise (Sec. 5.3).

Readings:
  * boundary conditions: homogeneous Dirichlet on every face for every component by default; with the Neumann
    flags bc = (k0, k1) of the Poisson spaces (the same pair in every direction) the faces eta_t = 0 (k0 = 1)
    or eta_t = 1 (k1 = 1) are traction-free for every component (the natural condition of the bilinear form:
    their end functions stay in the space).  The paper's column test mixes Dirichlet and Neumann faces per
    direction on a geometry it does not give;
  * body force: a constant vector f, so component i of the rhs is f_i times the Poisson load of f = 1;
  * preconditioner block i: the parametric-cube diagonal block mu (K M M + M K M + M M K) + (lambda + mu)
    (K in direction i), i.e. fast diagonalization with direction weights c_t = mu + (lambda + mu) delta_ti,
    and the exponential sum of the Poisson preconditioner (the weighted spectrum has the same ratio M_P);
  * block truncation: every component is truncated with the same relative tolerance; Alg. 2 uses block
    scalar products.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import bspline, fd, geometry, lowrank, rounding, tucker


# ------------------------------------------------------------------------------------------- coefficients
def coefficients(kind: str, amp: float, lam: float, mu: float, e1, e2, e3):
    """C[..., i, j, k, l] at the parametric points (shape (...) + (3, 3, 3, 3))."""
    e1, e2, e3 = np.broadcast_arrays(np.asarray(e1, float), np.asarray(e2, float), np.asarray(e3, float))
    if kind == "cube":
        G = np.broadcast_to(np.eye(3), e1.shape + (3, 3))
        det = np.ones(e1.shape)
    elif kind == "twist":
        J = geometry.twist_jacobian(e1, e2, e3, amp)
        det = np.linalg.det(J)
        G = np.linalg.inv(J)
    else:
        raise ValueError(kind)
    GGt = G @ np.swapaxes(G, -1, -2)
    C = np.zeros(e1.shape + (3, 3, 3, 3))
    eye = np.eye(3)
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    C[..., i, j, k, l] = det * (mu * eye[i, j] * GGt[..., k, l] + mu * G[..., k, i] * G[..., l, j]
                                                + lam * G[..., k, j] * G[..., l, i])
    return C


def _terms_of_coefficient(Ckl, n: int, p: int, eps: float, bc=(0, 0)):
    """Kronecker terms of sum_{k,l} int Ckl[k][l](eta) d_k phi d_l psi (the Poisson construction)."""
    n_el = bspline.n_el_of(n, p, bc)
    xs, ws = bspline.quadrature(n_el, p)
    B0 = bspline.bc_basis(n_el, p, xs, 0, bc)
    B1 = bspline.bc_basis(n_el, p, xs, 1, bc)
    norms = np.array([[np.linalg.norm(Ckl[..., k, l]) for l in range(3)] for k in range(3)])
    scale = max(norms.max(), 1e-300)
    terms = []
    for k in range(3):
        for l in range(3):
            if norms[k, l] <= 1e-13 * scale:
                continue
            core, U = lowrank.tucker_of_samples(Ckl[..., k, l], eps)
            R = core.shape
            mstar = max(range(3), key=lambda t: (R[t], t))
            others = [t for t in range(3) if t != mstar]
            g = [lowrank.cheb_eval(U[t], xs) for t in range(3)]
            for a in range(R[others[0]]):
                for b in range(R[others[1]]):
                    idx = [slice(None)] * 3
                    idx[others[0]] = a
                    idx[others[1]] = b
                    h = g[mstar] @ core[tuple(idx)]
                    funcs = {others[0]: g[others[0]][:, a], others[1]: g[others[1]][:, b], mstar: h}
                    mats = []
                    for t in range(3):
                        Bi = B1 if t == l else B0     # derivative l acts on the test function (rows)
                        Bj = B1 if t == k else B0     # derivative k acts on the trial function (columns)
                        mats.append((Bi * (ws * funcs[t])) @ Bj.T)
                    terms.append((1.0, mats))
    return terms


def operator_blocks(kind: str, amp: float, n: int, p: int, lam: float, mu: float, eps: float = 1e-8,
                    bc=(0, 0)):
    """blocks[i][j]: Kronecker terms of A_ij (component i of the test space, j of the trial space)."""
    xc = lowrank.cheb_points()
    e1, e2, e3 = np.meshgrid(xc, xc, xc, indexing="ij")
    C = coefficients(kind, amp, lam, mu, e1, e2, e3)
    return [[_terms_of_coefficient(C[..., i, j, :, :], n, p, eps, bc) for j in range(3)] for i in range(3)]


def rhs(kind: str, amp: float, n: int, p: int, force, eps: float = 1e-8, bc=(0, 0)):
    """Component i: f_i times the load of the unit body force, int det(J) psi (Tucker, App. A)."""
    n_el = bspline.n_el_of(n, p, bc)
    xc = lowrank.cheb_points()
    e1, e2, e3 = np.meshgrid(xc, xc, xc, indexing="ij")
    if kind == "cube":
        om = np.ones(e1.shape)
    else:
        om = np.linalg.det(geometry.twist_jacobian(e1, e2, e3, amp))
    core, U = lowrank.tucker_of_samples(om, eps)
    xs, ws = bspline.quadrature(n_el, p)
    B0 = bspline.bc_basis(n_el, p, xs, 0, bc)
    F = [(B0 * ws) @ lowrank.cheb_eval(U[t], xs) for t in range(3)]
    return [(force[i] * core, [f.copy() for f in F]) for i in range(3)]


# ------------------------------------------------------------------------------------------- block algebra
def assemble(blocks):
    """The 3 n^3 x 3 n^3 sparse matrix [A_ij] (component-major ordering)."""
    rows = []
    for i in range(3):
        from .fullcg import assemble as asm
        rows.append([asm(blocks[i][j]) if blocks[i][j] else None for j in range(3)])
    N = next(b.shape[0] for r in rows for b in r if b is not None)
    return sp.bmat([[b if b is not None else sp.csr_matrix((N, N)) for b in r] for r in rows]).tocsr()


def bvec(X):
    return np.concatenate([tucker.vec(tucker.full(x)) for x in X])


def bmatvec(blocks, X):
    """y_i = sum_j A_ij x_j (unrounded block-diagonal cores)."""
    out = []
    for i in range(3):
        yi = None
        for j in range(3):
            if not blocks[i][j]:
                continue
            t = tucker.matvec(blocks[i][j], X[j])
            yi = t if yi is None else tucker.add(yi, t)
        out.append(yi)
    return out


def badd(X, Y):
    return [tucker.add(x, y) for x, y in zip(X, Y)]


def bscale(X, a):
    return [tucker.scale(x, a) for x in X]


def bdot(X, Y):
    return float(sum(tucker.dot(x, y) for x, y in zip(X, Y)))


def bnorm(X):
    return float(np.sqrt(max(bdot(X, X), 0.0)))


def bround(X, eps, caps=None):
    return [rounding.t_rel(x, eps, caps) for x in X]


def bzero(n):
    return [(np.zeros((0, 0, 0)), [np.zeros((n, 0)) for _ in range(3)]) for _ in range(3)]


# ------------------------------------------------------------------------------------------- preconditioner
def direction_weights(lam: float, mu: float):
    """c[i][t] = mu + (lambda + mu) delta_ti: the parametric diagonal block i as a weighted Kronecker sum."""
    return [[mu + (lam + mu) * (1.0 if t == i else 0.0) for t in range(3)] for i in range(3)]


class BlockFD:
    """Block-diagonal P~^-1: block i is Alg. 4 for sum_t c_t (K in direction t) with the App. B eigenpairs.
    1 / sum_t c_t lam_t ~= (1/l_i) sum_j omega_j prod_t exp(-alpha_j c_t lam_t / l_i), l_i = (sum_t c_t) lam_min."""

    def __init__(self, n: int, p: int, lam: float, mu: float, base: fd.ApproxFD | None = None, bc=(0, 0)):
        self.P = base if base is not None else fd.ApproxFD(n, p, bc=bc)
        self.bc = tuple(bc)
        self.c = direction_weights(lam, mu)
        self.lmin1 = float(self.P.lam.min())
        self.lmin = [sum(ci) * self.lmin1 for ci in self.c]

    def apply_one(self, i, S):
        core, F = S
        P = self.P
        V = tucker.superdiag_kron(P.omega / self.lmin[i], core)
        facs = []
        for t in range(3):
            Z = P.U.T @ F[t]
            cols = [P.U @ (np.exp(-P.alpha[j] * self.c[i][t] * P.lam / self.lmin[i])[:, None] * Z)
                    for j in range(P.RP)]
            facs.append(np.concatenate(cols, axis=1))
        return V, facs

    def apply(self, S):
        return [self.apply_one(i, S[i]) for i in range(3)]

    def exact_block(self, i):
        """Dense inverse of the weighted FD block with exact eigenpairs (reference for tiny n)."""
        lamx, U = fd.exact_eig(self.P.n, self.P.p, self.bc)
        c = self.c[i]
        D = c[0] * lamx[:, None, None] + c[1] * lamx[None, :, None] + c[2] * lamx[None, None, :]
        return U, D


# ------------------------------------------------------------------------------------------- Alg. 5, block form
def tpcg(blocks, f, prec, prm, record=None):
    """Alg. 5 on block vectors (Sec. 5.3); the same steps as ``tpcg.tpcg`` with block operations."""
    A = lambda X: bmatvec(blocks, X)
    nf = bnorm(f)
    eps_min = prm.eps_min if prm.eps_min is not None else prm.tol * nf * 0.1
    n = f[0][1][0].shape[0]
    x = bzero(n)
    r = f
    nr = bnorm(r)
    eta = prm.beta_trunc * prm.tol * nf / nr
    z = bround(prec(r), eta, prm.caps)
    p = z
    q = bround(A(p), eta, prm.caps)
    xi = bdot(p, q)
    eps = prm.eps0
    k = 0
    while nr > prm.tol * nf and k < prm.max_it:
        omega = bdot(r, p) / xi
        x_tilde = badd(x, bscale(p, omega))
        # Alg. 2 with block scalar products
        d_tilde = badd(x_tilde, bscale(x, -1.0))
        dd = bdot(d_tilde, d_tilde)
        while True:
            x_next = bround(x_tilde, eps, prm.caps)
            v = bdot(d_tilde, badd(x_next, bscale(x, -1.0))) / dd if dd > 0 else 1.0
            if abs(v - 1.0) < prm.delta:
                break
            elif prm.alpha * eps > eps_min:
                eps *= prm.alpha
            else:
                break
        x = x_next
        r = bround(badd(f, bscale(A(x), -1.0)), eta, prm.caps)
        nr = bnorm(r)
        eta = prm.beta_trunc * prm.tol * nf / nr
        z = bround(prec(r), eta, prm.caps)
        beta_k = -bdot(z, q) / xi
        p = bround(badd(z, bscale(p, beta_k)), eta, prm.caps)
        q = bround(A(p), eta, prm.caps)
        xi = bdot(p, q)
        k += 1
        if record is not None:
            record.append({"k": k, "res": nr / nf, "eps": eps})
    return x, {"iters": k, "res": nr / nf}
