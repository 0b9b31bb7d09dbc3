"""Tucker vectors and Tucker/Kronecker matrices (Sec. 2.3).

Oracle module (test infrastructure only).  A Tucker tensor is ``(core, [U1, U2, U3])`` with
U_t of shape (n_t, r_t); vec() is column-major (mode 1 fastest).  The core is either a dense
(r1, r2, r3) array, or a ``Blocks`` object: a block-diagonal core kept as its list of
diagonal blocks, each (offsets, dense block).  The block form is the same core as the dense one
with its zero off-diagonal blocks left out (sums and Kronecker cores of Sec. 2.3 are
block-diagonal); ``dense_core`` materialises it, and tests check both forms agree.
"""
from __future__ import annotations

import numpy as np


class Blocks:
    """Block-diagonal core: shape (r1, r2, r3) and blocks [((o1, o2, o3), G)]."""

    def __init__(self, shape, blocks):
        self.shape = tuple(int(s) for s in shape)
        self.blocks = blocks

    def scaled(self, a):
        return Blocks(self.shape, [(o, a * G) for o, G in self.blocks])


def as_blocks(core):
    if isinstance(core, Blocks):
        return core
    return Blocks(core.shape, [((0, 0, 0), core)])


def dense_core(core) -> np.ndarray:
    if not isinstance(core, Blocks):
        return core
    out = np.zeros(core.shape)
    for o, G in core.blocks:
        sl = tuple(slice(o[t], o[t] + G.shape[t]) for t in range(3))
        out[sl] += G
    return out


def mode_product(X: np.ndarray, J: np.ndarray, m: int) -> np.ndarray:
    """[X x_m J]_{..i_m..} = sum_j X_{..j..} J_{i_m, j}  (Sec. 2.3; Kolda-Bader index order)."""
    Xm = np.moveaxis(X, m, 0)
    Y = np.tensordot(J, Xm, axes=(1, 0))
    return np.moveaxis(Y, 0, m)


def contract(core, mats) -> np.ndarray:
    """core x_1 mats[0] x_2 mats[1] x_3 mats[2] (dense result); a block core is contracted block
    by block, sum_b G_b x_t mats[t][:, block columns]."""
    if not isinstance(core, Blocks):
        Z = core
        for m in range(3):
            Z = mode_product(Z, mats[m], m)
        return Z
    Z = np.zeros(tuple(mats[m].shape[0] for m in range(3)))
    for o, G in core.blocks:
        T = G
        for m in range(3):
            T = mode_product(T, mats[m][:, o[m]:o[m] + G.shape[m]], m)
        Z += T
    return Z


def full(T) -> np.ndarray:
    """The full n1 x n2 x n3 array of a Tucker tensor, eq. Tucker."""
    core, U = T
    return contract(core, U)


def vec(X: np.ndarray) -> np.ndarray:
    """Column-major vectorisation (Sec. 2.3)."""
    return X.reshape(-1, order="F")


def unvec(x: np.ndarray, n) -> np.ndarray:
    return x.reshape(tuple(n), order="F")


def kron_core(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Kronecker product of two dense 3-way tensors, eq. kron_tensors: k_l = j_l + i_l n_l."""
    m, nn = A.shape, B.shape
    out = np.zeros(tuple(m[t] * nn[t] for t in range(3)))
    for i in np.ndindex(*m):
        sl = tuple(slice(i[t] * nn[t], (i[t] + 1) * nn[t]) for t in range(3))
        out[sl] = A[i] * B
    return out


def superdiag_kron(w, core):
    """superdiag(w) (x) core as a block core: block j is w_j * core at offsets j * r."""
    c = as_blocks(core)
    r = c.shape
    blocks = []
    for j, wj in enumerate(w):
        for o, G in c.blocks:
            blocks.append(((o[0] + j * r[0], o[1] + j * r[1], o[2] + j * r[2]), wj * G))
    return Blocks(tuple(len(w) * r[t] for t in range(3)), blocks)


def superdiagonal(w) -> np.ndarray:
    """R x R x R tensor with w on the superdiagonal."""
    R = len(w)
    D = np.zeros((R, R, R))
    for j in range(R):
        D[j, j, j] = w[j]
    return D


def matvec(terms, X, dense: bool = False):
    """Kronecker-sum matrix times Tucker vector, eq. tt_product.

    ``terms`` = [(w_j, [K1^j, K2^j, K3^j])]: a Tucker matrix with superdiagonal core w.
    Result factors [K_t^1 X_t, ..., K_t^R X_t]; result core superdiag(w) (x) G_X
    (dense with ``dense=True``, else as blocks).
    """
    core, U = X
    w = [t[0] for t in terms]
    fac = [np.concatenate([t[1][m] @ U[m] for t in terms], axis=1) for m in range(3)]
    if dense:
        return kron_core(superdiagonal(w), dense_core(core)), fac
    return superdiag_kron(w, core), fac


def add(X, Y):
    """Tucker sum: concatenated factors, block-diagonal core (Sec. 2.3)."""
    cx, ux = X
    cy, uy = Y
    bx, by = as_blocks(cx), as_blocks(cy)
    r = bx.shape
    blocks = list(bx.blocks) + [((o[0] + r[0], o[1] + r[1], o[2] + r[2]), G) for o, G in by.blocks]
    core = Blocks(tuple(r[t] + by.shape[t] for t in range(3)), blocks)
    return core, [np.concatenate([ux[m], uy[m]], axis=1) for m in range(3)]


def add_dense(X, Y):
    """Tucker sum with the block-diagonal core materialised (the literal definition)."""
    c, U = add(X, Y)
    return dense_core(c), U


def scale(X, a: float):
    core, U = X
    if isinstance(core, Blocks):
        return core.scaled(a), list(U)
    return a * core, list(U)


def dot(X, Y) -> float:
    """<X, Y> = vec(G_X)^T vec(G_Y x_3 X_3^T Y_3 x_2 X_2^T Y_2 x_1 X_1^T Y_1)  (Sec. 2.3)."""
    gx, ux = X
    gy, uy = Y
    Z = contract(gy, [ux[m].T @ uy[m] for m in range(3)])
    return float(np.sum(dense_core(gx) * Z))


def norm(X) -> float:
    return float(np.sqrt(max(dot(X, X), 0.0)))


def ranks(X):
    return tuple(X[0].shape)


def mem_compression(X, n) -> float:
    """Memory compression percentage, eq. mem_comp."""
    r = X[0].shape
    return (r[0] * r[1] * r[2] + sum(r[t] * n[t] for t in range(3))) / float(n[0] * n[1] * n[2]) * 100.0
