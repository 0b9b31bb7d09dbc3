"""CPU model of the pair schedule of the cluster-parallel Jacobi eigensolver (cjacobi_eig_kernel): C CTAs
own consecutive pair slots, the circle method moves every player one slot per step, and only the boundary
columns travel between CTAs.  The model checks what the kernel relies on: every pair of players meets exactly
once per sweep, each CTA's buffers stay a permutation of its slots (no column lost or duplicated), and Jacobi
rotations applied in this order diagonalise a symmetric matrix."""
import numpy as np
import pytest

C = 8   # CTAs per cluster in the kernel


def _padded(M):
    return ((M + 4 * C - 1) // (4 * C)) * (4 * C)


class Ring:
    """Slots top[k], bot[k] (k < h); CTA c owns slots [c ppc, (c+1) ppc) with buffer indices per slot."""

    def __init__(self, Mp):
        self.h = Mp // 2
        self.ppc = self.h // C
        ppc = self.ppc
        self.tix = [list(range(ppc)) for _ in range(C)]
        self.bix = [list(range(ppc, 2 * ppc)) for _ in range(C)]
        self.topP = [[2 * (c * ppc + k) for k in range(ppc)] for c in range(C)]
        self.botP = [[2 * (c * ppc + k) + 1 for k in range(ppc)] for c in range(C)]

    def pairs(self):
        return [(self.topP[c][k], self.botP[c][k]) for c in range(C) for k in range(self.ppc)]

    def move(self, cols):
        """One circle-method step; cols[c][b] is the column held in buffer b of CTA c (moved with players)."""
        ppc = self.ppc
        landing = [[None, None] for _ in range(C)]     # (player, column) arriving as top / bottom
        for c in range(C):
            if c < C - 1:
                landing[c + 1][0] = (self.topP[c][ppc - 1], cols[c][self.tix[c][ppc - 1]])
            if c > 0:
                landing[c - 1][1] = (self.botP[c][0], cols[c][self.bix[c][0]])
        for c in range(C):
            tix, bix, topP, botP = self.tix[c], self.bix[c], self.topP[c], self.botP[c]
            nt, nb, ntp, nbp = [None] * ppc, [None] * ppc, [None] * ppc, [None] * ppc
            for k in range(1, ppc):
                nt[k], ntp[k] = tix[k - 1], topP[k - 1]
            for k in range(ppc - 1):
                nb[k], nbp[k] = bix[k + 1], botP[k + 1]
            if c == 0:
                nt[0], ntp[0] = tix[0], topP[0]
                nt[1], ntp[1] = bix[0], botP[0]
                for k in range(2, ppc):
                    nt[k], ntp[k] = tix[k - 1], topP[k - 1]
            else:
                nt[0], ntp[0] = bix[0], landing[c][0][0]
                cols[c][bix[0]] = landing[c][0][1]
            if c == C - 1:
                nb[ppc - 1], nbp[ppc - 1] = tix[ppc - 1], topP[ppc - 1]
            else:
                nb[ppc - 1], nbp[ppc - 1] = tix[ppc - 1], landing[c][1][0]
                cols[c][tix[ppc - 1]] = landing[c][1][1]
            self.tix[c], self.bix[c], self.topP[c], self.botP[c] = nt, nb, ntp, nbp


@pytest.mark.parametrize("M", [3, 32, 40, 128, 256])
def test_every_pair_meets_once_per_sweep_and_buffers_are_conserved(M):
    Mp = _padded(M)
    ring = Ring(Mp)
    cols = [[("col", c, b) for b in range(2 * ring.ppc)] for c in range(C)]
    owner = {}
    for c in range(C):
        for k in range(ring.ppc):
            owner[ring.topP[c][k]] = cols[c][ring.tix[c][k]]
            owner[ring.botP[c][k]] = cols[c][ring.bix[c][k]]
    met = set()
    for _ in range(Mp - 1):
        for p, q in ring.pairs():
            met.add((min(p, q), max(p, q)))
        ring.move(cols)
        for c in range(C):
            assert sorted(ring.tix[c] + ring.bix[c]) == list(range(2 * ring.ppc))
            for k in range(ring.ppc):   # each player's column travelled with it
                assert cols[c][ring.tix[c][k]] == owner[ring.topP[c][k]]
                assert cols[c][ring.bix[c][k]] == owner[ring.botP[c][k]]
        assert sorted(sum(ring.topP, []) + sum(ring.botP, [])) == list(range(Mp))
    assert len(met) == Mp * (Mp - 1) // 2


def test_jacobi_in_the_ring_order_diagonalises():
    rng = np.random.default_rng(3)
    M = 40
    X = rng.standard_normal((M, M + 5))
    A = X @ X.T
    Mp = _padded(M)
    ring = Ring(Mp)
    V = np.eye(M)
    B = A.copy()
    for _ in range(12):
        for _ in range(Mp - 1):
            for p, q in ring.pairs():
                p, q = min(p, q), max(p, q)
                if q >= M or abs(B[p, q]) <= 1e-15 * np.sqrt(abs(B[p, p] * B[q, q])):
                    continue
                th = (B[q, q] - B[p, p]) / (2 * B[p, q])
                t = np.sign(th) / (abs(th) + np.hypot(th, 1.0)) if th != 0 else 1.0
                c = 1 / np.hypot(t, 1.0)
                s = t * c
                J = np.eye(M)
                J[p, p] = J[q, q] = c
                J[p, q], J[q, p] = s, -s
                B = J.T @ B @ J
                V = V @ J
            ring.move([[None] * (2 * ring.ppc) for _ in range(C)])
    w = np.linalg.eigvalsh(A)
    assert np.allclose(np.sort(np.diag(B)), w, rtol=0, atol=1e-12 * w.max())
    assert np.linalg.norm(V.T @ V - np.eye(M)) < 1e-12
    assert np.linalg.norm(A @ V - V * np.diag(B)) < 1e-10 * np.linalg.norm(A)
