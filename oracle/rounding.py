"""Truncation of Tucker tensors: ST-HOSVD, relative truncation (Alg. 1), dynamic truncation (Alg. 2).

Oracle module (test infrastructure only).

Readings:
  * ST-HOSVD (Sec. 2.3, Vannieuwenhoven et al.) processes modes 1, 2, 3 in order; mode m keeps the
    smallest s_m whose discarded squared singular values sum to <= eps^2 ||Z||^2 / 3, so that the
    total error is <= eps ||Z|| (the errors of the three sequential projections add in squares).
    An optional rank cap clips s_m afterwards; the realised error is returned.
  * Alg. 2, step "ElsIf": the test is alpha * eps_new > eps_min (with the current tolerance).
"""
from __future__ import annotations

import numpy as np

from . import tucker


def _unfold(Z: np.ndarray, m: int) -> np.ndarray:
    return np.moveaxis(Z, m, 0).reshape(Z.shape[m], -1)


def sthosvd(Z: np.ndarray, eps: float, caps=None):
    """Sequentially truncated HOSVD of a full tensor.

    Returns (core, [S1, S2, S3], discarded) with Z ~= core x_1 S1 x_2 S2 x_3 S3, orthonormal S_m,
    and discarded = sum over modes of the discarded squared singular values (the exact squared
    error of the sequential truncation).
    """
    nrm2 = float(np.sum(Z * Z))
    budget = eps * eps * nrm2 / 3.0
    S = []
    discarded = 0.0
    for m in range(3):
        U, sig, _ = np.linalg.svd(_unfold(Z, m), full_matrices=False)
        sig2 = sig ** 2
        # tail[s] = sum_{i >= s} sig_i^2
        tail = np.concatenate([np.cumsum(sig2[::-1])[::-1], [0.0]])
        s = int(np.argmax(tail <= budget))
        if s == 0 and Z.shape[m] > 0 and nrm2 > 0.0:
            s = 1 if tail[0] > 0.0 else 0
        if caps is not None:
            s = min(s, caps[m])
        discarded += float(tail[s])
        Sm = U[:, :s]
        S.append(Sm)
        Z = tucker.mode_product(Z, Sm.T, m)
    return Z, S, discarded


def t_rel(Y, eps: float, caps=None, return_info: bool = False):
    """Relative tolerance truncation, Alg. 1.

    1. QR of every factor, Y_t = Q_t R_t;  2. Z = core x_t R_t;  3. ST-HOSVD(Z, eps);
    4. new factors Q_t S_t.
    """
    core, U = Y
    Q, R = [], []
    for m in range(3):
        q, r = np.linalg.qr(U[m], mode="reduced")
        Q.append(q)
        R.append(r)
    Z = tucker.contract(core, R)
    newcore, S, discarded = sthosvd(Z, eps, caps)
    out = (newcore, [Q[m] @ S[m] for m in range(3)])
    if return_info:
        return out, {"discarded": discarded, "norm2": float(np.sum(Z * Z))}
    return out


def t_dt(y_k, y_tilde, eps: float, alpha: float, eps_min: float, delta: float, caps=None):
    """Dynamic truncation, Alg. 2.  Returns (y_{k+1}, eps_new, trials)."""
    eps_new = eps
    d_tilde = tucker.add(y_tilde, tucker.scale(y_k, -1.0))
    dd = tucker.dot(d_tilde, d_tilde)
    trials = 0
    while True:
        trials += 1
        y_next = t_rel(y_tilde, eps_new, caps)
        d = tucker.add(y_next, tucker.scale(y_k, -1.0))
        v = tucker.dot(d_tilde, d) / dd if dd > 0 else 1.0
        if abs(v - 1.0) < delta:
            break
        elif alpha * eps_new > eps_min:
            eps_new = alpha * eps_new
        else:
            break
    return y_next, eps_new, trials
