"""Operator pieces at the large size (twisted annulus, p = 3, n = 512 dofs per direction): the banded apply,
a truncation and the FD preconditioner, checked on sampled entries that the oracle computes one by one (the
full 512^3 tensors are never formed on the host)."""
import numpy as np
import pytest

import synth
from oracle import fd, rounding, tucker

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N, P = 512, 3


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_00632_gb300 import api, lib
    lib.load()
    pb = api.tpcg_setup(lib.GEOM_TWIST, synth.amp_from_seed(11), P, N, lib.F64)
    ex = pb.export()
    return api, lib, pb, ex


def _entries(T, idx):
    """Entries (i, j, k) of a Tucker tensor with a dense or block core, computed one by one."""
    core, U = T
    blocks = tucker.as_blocks(core).blocks
    out = np.zeros(len(idx))
    for o, G in blocks:
        sl = [slice(o[t], o[t] + G.shape[t]) for t in range(3)]
        A = U[0][idx[:, 0], sl[0]]
        B = U[1][idx[:, 1], sl[1]]
        C = U[2][idx[:, 2], sl[2]]
        out += np.einsum("abc,qa,qb,qc->q", G, A, B, C)
    return out


def _band_terms(ex, R):
    bw = 2 * P + 1
    bands = np.asarray(ex["bands"]).reshape(R, 3, bw, N)
    terms = []
    for j in range(R):
        mats = []
        for t in range(3):
            K = np.zeros((N, N))
            for d in range(bw):
                i = np.arange(N)
                jj = i + d - P
                ok = (jj >= 0) & (jj < N)
                K[i[ok], jj[ok]] = bands[j, t, d, ok]
            mats.append(K)
        terms.append((float(ex["w"][j]), mats))
    return terms


def test_apply_round_and_preconditioner_at_n512(setup):
    api, lib, pb, ex = setup
    info = pb.info
    R = info.R
    X = synth.random_tucker((N, N, N), (8, 6, 5), seed=12, decay=0.5)
    x = api.Tucker.from_numpy(X[0], X[1])
    rng = np.random.default_rng(13)
    idx = rng.integers(0, N, size=(300, 3))
    # apply: y = A x (block core), sampled against the oracle's matvec with the exported operator
    terms = _band_terms(ex, R)
    y = api.Tucker(N, cap=R * 8, core_cap=(R * 8) ** 3)
    api.tucker_apply(pb, x, y)
    Y = y.to_numpy(others=[x])
    Yo = tucker.matvec(terms, X)
    ref = _entries(Yo, idx)
    got = _entries(Y, idx)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    # truncation of y (k = R r < n: the QR path, FP64 Grams on the cluster eigensolver): error bound of Alg. 1,
    # sampled entries within it, and ranks within one of the oracle's own truncation
    ctx = api.Ctx(N, R * 8, min(R * 8, 256))
    info_dev = torch.zeros(6, dtype=torch.float64, device="cuda")
    api.tucker_round(ctx, y, 1e-6, info=info_dev)
    Yr = y.to_numpy()
    h = info_dev.cpu().numpy()
    assert h[5] == 0.0                                              # the core fitted
    assert np.sqrt(h[1]) <= 1e-6 * np.sqrt(h[0]) * (1 + 1e-9)       # Alg. 1 error bound, exact accounting
    # every entry of the error is bounded by its Frobenius norm
    assert np.max(np.abs(_entries(Yr, idx) - ref)) <= 1e-6 * np.sqrt(h[0]) * (1 + 1e-6)
    Yor = rounding.t_rel(Yo, 1e-6)
    assert all(abs(a - b) <= 1 for a, b in zip(Yr[0].shape, Yor[0].shape))
    # FD preconditioner (Alg. 4 with App. B eigenpairs) on a plain input, against the oracle's Alg. 4
    Pf = fd.ApproxFD(N, P, expsum=(np.asarray(ex["omega"]), np.asarray(ex["alpha"])))
    s = api.Tucker.from_numpy(X[0], X[1])
    v = api.Tucker(N, cap=info.RP * 8, core_cap=1)
    ctx2 = api.Ctx(N, info.RP * 8, 8)
    api.fd_precond_apply(pb, ctx2, s, v)
    V = v.to_numpy(others=[s])
    ref_v = _entries(Pf.apply(X), idx)
    got_v = _entries(V, idx)
    assert np.max(np.abs(got_v - ref_v)) <= 1e-9 * np.max(np.abs(ref_v))
