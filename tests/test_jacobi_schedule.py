"""CPU model of the one-CTA FP32 Jacobi eigensolver's step (jacobi_eig_v_kernel): round-robin pairs, the
rotating threads writing their own 2 x 2 diagonal block (a_pp - t a_pq, a_qq + t a_pq, coupling zero), the
off-diagonal blocks (a < b) decoded from a flat index, and V's update for a step applied during the next
step's rotations (rotation parameters double-buffered by step parity, the last step's flushed after the
sweeps).  The model checks what the kernel relies on: the decode enumerates every off-diagonal block once,
the blocks and diagonal writes of a step touch disjoint entries that cover the matrix, the diagonal formula
equals J^T A J with the kernel's sign convention, and the deferred V update yields the eigenvectors."""
import math

import numpy as np
import pytest

NT = 1024   # threads per CTA in the kernel


def _pairs(step, M):
    Mp = M + (M % 2)
    P, half = Mp - 1, Mp // 2
    out = []
    for k in range(half):
        a, b = (P, step) if k == 0 else ((step + k) % P, (step - k) % P)
        p, q = min(a, b), max(a, b)
        out.append((p, q if q < M else -1))
    return out


def _decode(q):
    """Flat index -> off-diagonal block (a, b), a < b, as the kernel decodes it (float sqrt, then fixed up)."""
    bb = int((1.0 + math.sqrt(8.0 * q + 1.0)) * 0.5)
    while bb * (bb - 1) // 2 > q:
        bb -= 1
    while (bb + 1) * bb // 2 <= q:
        bb += 1
    return q - bb * (bb - 1) // 2, bb


@pytest.mark.parametrize("M", [2, 3, 17, 96, 127, 128])
def test_blocks_and_diagonal_writes_partition_the_matrix(M):
    half = (M + (M % 2)) // 2
    nblk = half * (half - 1) // 2
    assert nblk <= 2 * NT                       # two blocks per thread at most
    assert NT - half >= 32                      # at least one warp left for V
    blocks = [_decode(q) for q in range(nblk)]
    assert sorted(blocks) == sorted((a, b) for b in range(half) for a in range(b))
    P = M + (M % 2) - 1
    for step in range(0, P, max(1, P // 7)):
        pr = _pairs(step, M)
        hit = np.zeros((M, M), dtype=int)
        for p, q in pr:                          # the rotating threads' diagonal blocks
            idx = [p] + ([q] if q >= 0 else [])
            for i in idx:
                for j in idx:
                    hit[i, j] += 1
        for a, b in blocks:                      # each off-diagonal block and its mirror
            ra = [x for x in pr[a] if x >= 0]
            rb = [x for x in pr[b] if x >= 0]
            for i in ra:
                for j in rb:
                    hit[i, j] += 1
                    hit[j, i] += 1
        assert (hit == 1).all()


def test_diagonal_block_formula_matches_the_similarity():
    rng = np.random.default_rng(5)
    for _ in range(20):
        X = rng.standard_normal((6, 7))
        A = X @ X.T
        p, q = sorted(rng.choice(6, 2, replace=False))
        app, aqq, apq = A[p, p], A[q, q], A[p, q]
        th = (aqq - app) / (2 * apq)
        t = (1.0 if th >= 0 else -1.0) / (abs(th) + math.sqrt(th * th + 1))
        c = 1 / math.sqrt(t * t + 1)
        s = t * c
        J = np.eye(6)
        J[p, p] = J[q, q] = c
        J[p, q], J[q, p] = s, -s
        B = J.T @ A @ J
        assert abs(B[p, q]) <= 1e-12 * abs(A).max()
        assert np.isclose(B[p, p], app - t * apq) and np.isclose(B[q, q], aqq + t * apq)


def _jacobi_deferred_v(G, tau=1e-12, max_sweeps=30):
    M = G.shape[0]
    A = G.copy()
    V = np.eye(M)
    P = M + (M % 2) - 1
    half = (M + (M % 2)) // 2
    rot = [[(1.0, 0.0, 0, -1)] * half, [(1.0, 0.0, 0, -1)] * half]

    def update_v(buf):
        for c, s, p, q in rot[buf]:
            if s != 0.0 and q >= 0:
                vp, vq = V[:, p].copy(), V[:, q].copy()
                V[:, p] = c * vp - s * vq
                V[:, q] = s * vp + c * vq

    g = 0
    for _ in range(max_sweeps):
        rotated = False
        for step in range(P):
            cur = g & 1
            if g > 0:
                update_v(cur ^ 1)                # V by the previous step, beside this step's rotations
            for k, (p, q) in enumerate(_pairs(step, M)):
                c, s = 1.0, 0.0
                if q >= 0 and abs(A[p, q]) > tau * math.sqrt(abs(A[p, p] * A[q, q])):
                    th = (A[q, q] - A[p, p]) / (2 * A[p, q])
                    t = (1.0 if th >= 0 else -1.0) / (abs(th) + math.sqrt(th * th + 1))
                    c = 1 / math.sqrt(t * t + 1)
                    s = t * c
                    app, aqq, apq = A[p, p], A[q, q], A[p, q]
                    A[p, p], A[q, q], A[p, q], A[q, p] = app - t * apq, aqq + t * apq, 0.0, 0.0
                    rotated = True
                rot[cur][k] = (c, s, p, q)
            B = A.copy()                         # off-diagonal blocks: rows by J_a^T, columns by J_b
            pr = rot[cur]
            for a in range(half):
                for b in range(a + 1, half):
                    ca, sa, pa, qa = pr[a]
                    cb, sb, pb, qb = pr[b]
                    ra = [pa] + ([qa] if qa >= 0 else [])
                    rb = [pb] + ([qb] if qb >= 0 else [])
                    Ja = np.array([[ca, sa], [-sa, ca]])[:len(ra), :len(ra)] if qa >= 0 else np.eye(1)
                    Jb = np.array([[cb, sb], [-sb, cb]])[:len(rb), :len(rb)] if qb >= 0 else np.eye(1)
                    Y = Ja.T @ A[np.ix_(ra, rb)] @ Jb
                    B[np.ix_(ra, rb)] = Y
                    B[np.ix_(rb, ra)] = Y.T
            A = B
            g += 1
        if not rotated:
            break
    if g > 0:
        update_v((g - 1) & 1)                    # flush: V by the last step
    return A, V


@pytest.mark.parametrize("M", [1, 2, 5, 8, 13])
def test_deferred_v_update_gives_the_eigenvectors(M):
    rng = np.random.default_rng(M)
    X = rng.standard_normal((M, M + 2))
    G = X @ X.T
    A, V = _jacobi_deferred_v(G)
    w = np.linalg.eigvalsh(G)
    d = np.diag(A)
    assert np.allclose(np.sort(d), w, rtol=0, atol=1e-10 * w.max())
    assert np.linalg.norm(V.T @ V - np.eye(M)) < 1e-10
    assert np.linalg.norm(G @ V - V * d) < 1e-9 * np.linalg.norm(G)
