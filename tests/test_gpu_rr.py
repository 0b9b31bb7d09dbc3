"""Alg. 1 step 3 on Grams larger than the one-CTA eigensolvers take (n' > 128 in FP32, n' > 256 in FP64), reduced
before the eigensolver to the Rayleigh-Ritz matrix Q^T G Q of an orthonormal basis Q of at most 128 pivoted-Cholesky
columns of G: the rank decision, the discarded energy and the error bound of Alg. 1 against the FP64 oracle, on
plain tensors whose every mode Gram is a dense n x n matrix with geometric eigenvalues d_i^2 (superdiagonal core
d_i behind random orthonormal factors of full rank, stored as five diagonal blocks like an operator product, so
Alg. 1 forms Z = the whole n^3 tensor).  eps puts the mode-1 budget between two consecutive tails of the
spectrum, far from both, so the oracle's ranks are the only right answer.  An operator product on the QR path
(Gram order 152) is rounded against the oracle.  A mixed-precision solve at n = 192, where the FP32
inner truncations meet Grams of order R r > 128, converges to the FP64 residual."""
import numpy as np
import pytest

from oracle import rounding
from tests.gpu_helpers import rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_00632_gb300 import api, lib
    lib.load()
    return api, lib


def _upload_block_diagonal(api, T, d, U, nb):
    """T <- the superdiagonal core d (length n) behind factors U, stored as nb diagonal blocks (the block
    layout of an operator product, each block within the context's rank cap)."""
    import struct
    n = len(d)
    b = n // nb
    dt = T.core.dtype
    for t in range(3):
        T.U[t][:n].copy_(torch.as_tensor(np.ascontiguousarray(U[t].T), dtype=dt))
    raw = bytearray(T.desc.numel())
    struct.pack_into("4i", raw, 0, nb, n, n, n)
    base = T.core.data_ptr()
    for k in range(nb):
        g = np.zeros((b, b, b))
        g[np.arange(b), np.arange(b), np.arange(b)] = d[k * b:(k + 1) * b]
        T.core[k * b ** 3:(k + 1) * b ** 3].copy_(torch.as_tensor(g.reshape(-1, order="F"), dtype=dt))
        o = 32 + 40 * k
        struct.pack_into("3i", raw, o, k * b, k * b, k * b)
        struct.pack_into("3i", raw, o + 12, b, b, b)
        struct.pack_into("Q", raw, o + 24, base + k * b ** 3 * T.core.element_size())
        struct.pack_into("d", raw, o + 32, 1.0)
    T.desc.copy_(torch.frombuffer(raw, dtype=torch.uint8))
    torch.cuda.synchronize()


def _case(n, decades_per_index, cut, seed):
    g = np.random.default_rng(seed)
    d = 10.0 ** (-np.arange(n) * decades_per_index)
    G = np.zeros((n, n, n))
    G[np.arange(n), np.arange(n), np.arange(n)] = d
    U = [np.linalg.qr(g.standard_normal((n, n)))[0] for _ in range(3)]
    tail = np.cumsum((d ** 2)[::-1])[::-1]
    budget = np.sqrt(tail[cut] * tail[cut - 1])     # between the mode-1 tails at s = cut - 1 and s = cut
    eps = float(np.sqrt(3.0 * budget / np.sum(d ** 2)))
    return (G, U), eps


@pytest.mark.parametrize("n,dtype_name,step,cut,cap", [(200, "F32", 0.1, 10, 64), (300, "F64", 1.0 / 12, 41, 96)])
def test_large_gram_rank_discarded_and_bound(mods, n, dtype_name, step, cut, cap):
    api, lib = mods
    dt = getattr(lib, dtype_name)
    Y, eps = _case(n, step, cut, seed=23)
    (G0, U0), inf0 = rounding.t_rel(Y, eps, return_info=True)
    assert G0.shape[0] == cut and max(G0.shape) <= cap      # the oracle's decision (margins set on the CPU)
    # five diagonal blocks of order n / 5 <= cap: the Z-formation workspace of a rank-cap-`cap` context holds them
    y = api.Tucker(n, cap=n, core_cap=5 * (n // 5) ** 3, dtype=dt)
    _upload_block_diagonal(api, y, Y[0][np.arange(n), np.arange(n), np.arange(n)], Y[1], 5)
    ctx = api.Ctx(n, n, cap, dtype=dt)
    info = torch.zeros(6, dtype=torch.float64, device="cuda")
    api.tucker_round(ctx, y, eps, info=info)
    torch.cuda.synchronize()
    h = info.cpu().numpy()
    G, U = y.to_numpy()
    assert h[5] == 0.0                                          # the workspace and the core fitted
    assert G.shape == G0.shape and tuple(int(v) for v in h[2:5]) == G0.shape
    tol = 1e-6 if dt == lib.F32 else 1e-12
    assert abs(h[0] - inf0["norm2"]) <= tol * inf0["norm2"]
    # discarded energy: the oracle's, to the accuracy of the Gram (FP32: a few 1e-6 of ||Z||^2 over three modes)
    assert abs(h[1] - inf0["discarded"]) <= (1e-2 * inf0["discarded"] + (5e-6 if dt == lib.F32 else 1e-14)
                                             * inf0["norm2"])
    # the tensor itself: the oracle's truncation, and Alg. 1's bound against Y
    from oracle import tucker
    full_y = tucker.full(Y)
    full_g = tucker.full((G, U))
    ny = np.linalg.norm(full_y)
    floor = 3e-6 if dt == lib.F32 else 1e-20
    assert np.linalg.norm(full_g - full_y) <= np.sqrt(eps ** 2 + floor) * ny * (1 + 1e-6)
    assert rel(full_g, tucker.full((G0, U0))) <= (1e-3 if dt == lib.F32 else 1e-9)
    # orthonormal factors
    for t in range(3):
        assert np.abs(U[t].T @ U[t] - np.eye(U[t].shape[1])).max() <= (2e-5 if dt == lib.F32 else 1e-12)


def test_operator_product_round_qr_path(mods):
    """An unrounded operator product at n = 192 (19 Kronecker terms, k = 19 r = 152 columns per mode: the QR
    path, Gram order 152 > 128) rounded in FP32 through the Rayleigh-Ritz step, against the oracle."""
    api, lib = mods
    import synth
    from oracle import tucker
    from tests.gpu_helpers import identity_tables, random_banded_terms
    n, p, R, cap, eps = 192, 3, 19, 96, 1e-2
    terms = random_banded_terms(n, p, R, seed=61)
    f = synth.random_tucker((n, n, n), (1, 1, 1), seed=62)
    X = synth.random_tucker((n, n, n), (8, 8, 8), seed=63, decay=0.3)
    Yo = tucker.matvec(terms, X)
    Go, Uo = rounding.t_rel(Yo, eps)
    assert max(Go.shape) <= cap                                 # (67, 56, 70): the cap does not bind
    full_o = tucker.full(Yo)
    ny = np.linalg.norm(full_o)
    pb = api.tpcg_problem_create(n, p, terms, f[0], f[1], identity_tables(n), dtype=1)
    x = api.Tucker.from_numpy(X[0], X[1], dtype=1)
    y = api.Tucker(n, cap=R * 8, core_cap=(R * 8) ** 3, dtype=1)
    api.tucker_apply(pb, x, y)
    ctx = api.Ctx(n, R * 8, cap, dtype=1)
    info = torch.zeros(6, dtype=torch.float64, device="cuda")
    api.tucker_round(ctx, y, eps, info=info)
    torch.cuda.synchronize()
    h = info.cpu().numpy()
    G, U = y.to_numpy()
    assert h[5] == 0.0
    # Alg. 1's bound against the exact product, with the FP32 Gram's resolution; the reported discarded energy
    # is the realised one
    err = np.linalg.norm(tucker.full((G, U)) - full_o)
    assert err <= np.sqrt(eps ** 2 + 3e-6) * ny * 1.01
    assert abs(err ** 2 - h[1]) <= 1e-2 * err ** 2 + 3e-6 * ny ** 2
    # the Ritz values of the pivoted-Cholesky basis miss at most 1% of the budget: the oracle's ranks up to an
    # FP32 near-tie
    assert all(abs(a - o) <= 1 for a, o in zip(G.shape, Go.shape))
    for t in range(3):
        assert np.abs(U[t].T @ U[t] - np.eye(U[t].shape[1])).max() <= 2e-5


def test_mixed_solve_n192_large_grams(mods):
    api, lib = mods
    import synth
    n, rc = 192, 64
    pb = api.tpcg_setup(lib.GEOM_TWIST, synth.amp_from_seed(7), 3, n, lib.MIXED)
    ctx = api.Ctx(n, api.max_cols_for(pb.info, rc, lib.MIXED), rc, lib.MIXED)
    x = api.Tucker(n, cap=rc, core_cap=rc ** 3, dtype=lib.MIXED)
    st = api.tpcg_solve(pb, ctx, x, tol=1e-6, rank_cap=rc)
    torch.cuda.synchronize()
    assert st.status == 0 and st.true_rel_res <= 1e-6
