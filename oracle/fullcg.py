"""Assembled Kronecker-sum matrix and full-vector (P)CG: the exact reference for tiny n.

Oracle module (test infrastructure only).  A~ = sum_j w_j K3^j (x) K2^j (x) K1^j is built as a
sparse matrix with scipy (eq. kron_matrices, eq. kron_vec_multi); the linear system
A~ x = f~ (eq. approx_ls) is then solved directly or by textbook PCG.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def assemble(terms):
    A = None
    for w, (K1, K2, K3) in terms:
        T = w * sp.kron(sp.csr_matrix(K3), sp.kron(sp.csr_matrix(K2), sp.csr_matrix(K1)))
        A = T if A is None else A + T
    return A.tocsr()


def solve_direct(terms, fvec):
    return spla.spsolve(assemble(terms).tocsc(), fvec)


def pcg(A, b, apply_prec, tol=1e-10, max_it=1000):
    """Textbook preconditioned CG on full vectors; returns (x, iterations)."""
    x = np.zeros_like(b)
    r = b.copy()
    z = apply_prec(r)
    p = z.copy()
    rz = r @ z
    nb = np.linalg.norm(b)
    for k in range(1, max_it + 1):
        q = A @ p
        a = rz / (p @ q)
        x += a * p
        r -= a * q
        if np.linalg.norm(r) <= tol * nb:
            return x, k
        z = apply_prec(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, max_it
