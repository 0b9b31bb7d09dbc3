"""Parity of the CUDA library (through the C ABI) with the FP64 oracle, element by element on seeded
inputs.  Sizes span several 64-wide GEMM tiles with ragged tails.  FP64 bar: 1e-10 relative (1e-12 where
the path has no truncation decision)."""
import numpy as np
import pytest

import synth
from oracle import fd, rounding, tucker
from tests.gpu_helpers import gpu_problem, identity_tables, oracle_problem, random_banded_terms, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_00632_gb300 import api as a
    from paper_2306_00632_gb300 import lib
    lib.load()
    return a


def _plain(api, T, cap=None, core_cap=None, dtype=0):
    return api.Tucker.from_numpy(T[0], T[1], cap=cap, core_cap=core_cap, dtype=dtype)


# ------------------------------------------------------------------------------------ apply / residual
@pytest.mark.parametrize("n,p,R,ranks", [(23, 2, 3, (3, 4, 2)), (70, 3, 5, (7, 5, 9)), (131, 5, 2, (1, 1, 1))])
def test_apply_matches_oracle(api, n, p, R, ranks):
    terms = random_banded_terms(n, p, R, seed=5)
    f = synth.random_tucker((n, n, n), (2, 1, 3), seed=8)
    pb = api.tpcg_problem_create(n, p, terms, f[0], f[1], identity_tables(n))
    X = synth.random_tucker((n, n, n), ranks, seed=3)
    x = _plain(api, X)
    y = api.Tucker(n, cap=R * max(ranks) + 3, core_cap=1)
    api.tucker_apply(pb, x, y)
    core, fac = y.to_numpy(others=[x])
    ref = tucker.matvec(terms, X, dense=True)
    for t in range(3):                                    # factors [K_t^1 X_t, ..., K_t^R X_t]
        assert rel(fac[t], ref[1][t]) < 1e-13
    assert rel(core, ref[0]) < 1e-15
    # residual f - A x: factors [F_t, K X_t...], block core (f core, -w_j G_x)
    yr = api.Tucker(n, cap=R * max(ranks) + 3, core_cap=1)
    api.tucker_residual(pb, x, yr)
    pbf = pb.info
    ex = pb.export()
    fcore = ex["f_core"].reshape(tuple(pbf.rf), order="F")     # the library's f (orthonormal factors)
    core_r, fac_r = yr.to_numpy(others=[x], fallback=lambda shape: fcore)
    nblk, ranks_r, blocks = yr.read_desc()
    assert nblk == 1 + R and ranks_r == tuple(pbf.rf[t] + R * ranks[t] for t in range(3))
    for t in range(3):                                    # leading columns: the library's F_t
        assert rel(fac_r[t][:, :pbf.rf[t]], ex[f"f_U{t}"].reshape((n, pbf.rf[t]), order="F")) < 1e-15
        assert rel(fac_r[t][:, pbf.rf[t]:], ref[1][t]) < 1e-13
    if n <= 70:                                           # full tensors: f - A x
        assert rel(tucker.full((core_r, fac_r)), tucker.full(f) - tucker.full(ref)) < 1e-12
    assert pbf.R == R


def test_axpby_and_dot(api):
    n = 67
    A = synth.random_tucker((n, n, n), (3, 5, 4), seed=1)
    B = synth.random_tucker((n, n, n), (4, 2, 6), seed=2)
    a, b = _plain(api, A), _plain(api, B)
    z = api.Tucker(n, cap=12, core_cap=1)
    coef = torch.tensor([-0.75], dtype=torch.float64, device="cuda")
    api.tucker_axpby(1.5, a, coef, b, z)
    core, fac = z.to_numpy(others=[a, b])
    ref = tucker.add_dense(tucker.scale(A, 1.5), tucker.scale(B, -0.75))
    assert rel(core, ref[0]) < 1e-15
    for t in range(3):
        assert rel(fac[t], ref[1][t]) < 1e-15
    ctx = api.Ctx(n, 64, 32)
    d = api.tucker_dot(ctx, a, b).item()
    assert abs(d - tucker.dot(A, B)) <= 1e-12 * tucker.norm(A) * tucker.norm(B)
    dd = api.tucker_dot(ctx, a, a).item()
    assert abs(dd - tucker.dot(A, A)) <= 1e-12 * tucker.dot(A, A)


# ------------------------------------------------------------------------------------ rounding (Alg. 1)
def _rotated_superdiagonal(d, n, seed):
    g = np.random.default_rng(seed)
    Qs = [np.linalg.qr(g.standard_normal((n, len(d))))[0] for _ in range(3)]
    return tucker.superdiagonal(d), Qs


@pytest.mark.parametrize("eps", [2e-3, 1e-6])
def test_round_rank_rule_and_tensor(api, eps):
    # Q path (k < n) with a spectrum whose truncation decisions are clear-cut
    n = 45
    d = np.array([1.0, 0.5, 0.1, 3e-3, 1e-3, 2e-4, 1e-5])
    Y = _rotated_superdiagonal(d, n, seed=5)
    ctx = api.Ctx(n, 64, 32)
    y = _plain(api, Y, cap=16, core_cap=16 ** 3)
    info = torch.zeros(8, dtype=torch.float64, device="cuda")
    api.tucker_round(ctx, y, eps, info=info)
    G, U = y.to_numpy()
    (G0, U0), oinfo = rounding.t_rel(Y, eps, return_info=True)
    assert G.shape == G0.shape
    assert rel(tucker.full((G, U)), tucker.full((G0, U0))) < 1e-10
    inf = info.cpu().numpy()
    assert abs(inf[1] - oinfo["discarded"]) <= 1e-10 * oinfo["norm2"]
    for t in range(3):
        assert np.abs(U[t].T @ U[t] - np.eye(U[t].shape[1])).max() < 1e-12


@pytest.mark.parametrize("n,ranks", [(19, (12, 25, 9)), (70, (40, 71, 66))])
def test_round_wide_factors_lossless(api, n, ranks):
    # k >= n in some modes (Q = I path) and k < n in others; eps = 0 keeps everything
    Y = synth.random_tucker((n, n, n), ranks, seed=4)
    ctx = api.Ctx(n, 80, min(n, 80))
    y = _plain(api, Y, cap=80, core_cap=80 ** 3)
    api.tucker_round(ctx, y, 0.0)
    G, U = y.to_numpy()
    G0, U0 = rounding.t_rel(Y, 0.0)
    assert G.shape == G0.shape
    assert rel(tucker.full((G, U)), tucker.full(Y)) < 1e-11


def test_round_block_tensor_and_cap(api):
    # rounding an unrounded apply output (block core), exact rank of a sum, and a rank cap
    n, p, R = 37, 3, 4
    terms = random_banded_terms(n, p, R, seed=9)
    f = synth.random_tucker((n, n, n), (1, 1, 1), seed=8)
    pb = api.tpcg_problem_create(n, p, terms, f[0], f[1], identity_tables(n))
    X = synth.random_tucker((n, n, n), (2, 3, 2), seed=6)
    x = _plain(api, X)
    y = api.Tucker(n, cap=16, core_cap=16 ** 3)
    api.tucker_apply(pb, x, y)
    ctx = api.Ctx(n, 16, 16)
    api.tucker_round(ctx, y, 1e-12)
    G, U = y.to_numpy()
    ref = tucker.matvec(terms, X)
    G0, U0 = rounding.t_rel(ref, 1e-12)
    assert G.shape == G0.shape
    assert rel(tucker.full((G, U)), tucker.full(ref)) < 1e-10
    # cap
    y2 = api.Tucker(n, cap=16, core_cap=16 ** 3)
    api.tucker_apply(pb, x, y2)
    api.tucker_round(ctx, y2, 1e-12, rank_cap=3)
    G2, U2 = y2.to_numpy()
    G3, U3 = rounding.t_rel(ref, 1e-12, caps=(3, 3, 3))
    assert G2.shape == G3.shape == (3, 3, 3)
    assert rel(tucker.full((G2, U2)), tucker.full((G3, U3))) < 1e-9


def test_round_zero_tensor(api):
    n = 20
    Y = (np.zeros((2, 2, 2)), [np.zeros((n, 2))] * 3)
    ctx = api.Ctx(n, 8, 8)
    y = _plain(api, Y, cap=8, core_cap=512)
    api.tucker_round(ctx, y, 1e-8)
    nblk, ranks, _ = y.read_desc()
    assert ranks == (0, 0, 0)


# ------------------------------------------------------------------------------------ FD preconditioner
@pytest.mark.parametrize("n,p", [(20, 2), (24, 3), (21, 4), (70, 5)])
def test_fd_matches_oracle(api, n, p):
    pb = gpu_problem("cube", 0.0, n, p)
    _, _, P, _ = oracle_problem("cube", 0.0, n, p)
    S = synth.random_tucker((n, n, n), (2, 3, 2), seed=21)
    s = _plain(api, S)
    ctx = api.Ctx(n, P.RP * 3 + 8, 8)
    v = api.Tucker(n, cap=P.RP * 3 + 8, core_cap=1)
    api.fd_precond_apply(pb, ctx, s, v)
    core, fac = v.to_numpy(others=[s])
    ref = P.apply(S)
    for t in range(3):
        assert rel(fac[t], ref[1][t]) < 1e-11
    assert rel(core, tucker.dense_core(ref[0])) < 1e-14


# ------------------------------------------------------------------------------------ setup (App. A, B)
@pytest.mark.parametrize("kind,amp,n,p", [("cube", 0.0, 12, 2), ("twist", 0.2, 14, 3), ("twist", 0.13, 13, 4),
                                          ("twist", 0.3, 15, 5)])
def test_setup_matches_oracle(api, kind, amp, n, p):
    kid = 0 if kind == "cube" else 1
    pb = api.tpcg_setup(kid, amp, p, n)
    terms, f, P, tables = oracle_problem(kind, amp, n, p)
    assert pb.info.R == len(terms)
    ex = pb.export()
    assert np.allclose(np.sort(ex["lam"]), np.sort(P.lam), rtol=1e-10)
    assert np.allclose(ex["mu"], tables["mu"], rtol=1e-11)
    assert abs(pb.info.MP - P.MP) <= 1e-10 * P.MP
    # the setup's default sums are the best sums of Prop. 1: equal to the oracle's Remez exchange
    from oracle import expsum
    R, om, al, _, _ = expsum.rp_best(P.MP, 0.1)
    assert pb.info.RP == R
    a, b = np.argsort(np.asarray(ex["alpha"])), np.argsort(al)
    assert np.allclose(np.asarray(ex["alpha"])[a], al[b], rtol=1e-8)
    assert np.allclose(np.asarray(ex["omega"])[a], om[b], rtol=1e-8)
    # operator: same action on a random Tucker vector (the Kronecker terms themselves are not unique)
    X = synth.random_tucker((n, n, n), (3, 2, 3), seed=2)
    x = _plain(api, X)
    y = api.Tucker(n, cap=pb.info.R * 3, core_cap=1)
    api.tucker_apply(pb, x, y)
    got = tucker.full(y.to_numpy(others=[x]))
    assert rel(got, tucker.full(tucker.matvec(terms, X))) < 1e-9
    # rhs
    rf = tuple(pb.info.rf)
    Fg = (ex["f_core"].reshape(rf, order="F"), [ex[f"f_U{t}"].reshape((n, rf[t]), order="F") for t in range(3)])
    assert rel(tucker.full(Fg), tucker.full(f)) < 1e-9


# ------------------------------------------------------------------------------------ TPCG (Alg. 5)
def test_tpcg_cube_one_step(api):
    n, p = 14, 2
    pb = gpu_problem("cube", 0.0, n, p)
    terms, f, P, _ = oracle_problem("cube", 0.0, n, p)
    from oracle import tpcg as otp
    xo, info = otp.tpcg(terms, f, P.apply, otp.Params(tol=1e-6))
    ctx = api.Ctx(n, max(P.RP, 4) * 14 + 4, 14)
    x = api.Tucker(n, cap=14, core_cap=14 ** 3)
    st = api.tpcg_solve(pb, ctx, x, tol=1e-6)
    assert st.status == 0 and st.iters == info["iters"] == 1
    assert rel(tucker.full(x.to_numpy()), tucker.full(xo)) < 1e-10


def test_tpcg_twist_against_oracle_and_direct(api):
    n, p = 12, 3
    amp = synth.amp_from_seed(7)
    pb = gpu_problem("twist", amp, n, p)
    terms, f, P, _ = oracle_problem("twist", amp, n, p)
    from oracle import fullcg
    from oracle import tpcg as otp
    xo, info = otp.tpcg(terms, f, P.apply, otp.Params(tol=1e-6))
    ctx = api.Ctx(n, max(len(terms) * 12 + 2, P.RP * 12), 12)
    x = api.Tucker(n, cap=12, core_cap=12 ** 3)
    st = api.tpcg_solve(pb, ctx, x, tol=1e-6)
    assert st.status == 0
    assert abs(st.iters - info["iters"]) <= 2
    xg = tucker.vec(tucker.full(x.to_numpy()))
    A = fullcg.assemble(terms)
    fv = tucker.vec(tucker.full(f))
    assert np.linalg.norm(fv - A @ xg) <= 2e-6 * np.linalg.norm(fv)
    assert rel(xg, tucker.vec(tucker.full(xo))) < 1e-4


# ------------------------------------------------------------------------------------ FP32 form
# Bar: 1e-4 relative (single-precision storage and products; the Gram of ST-HOSVD squares the FP32 rounding).
F32_TOL = 1e-4


def test_f32_apply_fd_dot(api):
    n, p = 40, 3
    pb = gpu_problem("cube", 0.0, n, p, dtype=1)
    terms, _, P, _ = oracle_problem("cube", 0.0, n, p)
    X = synth.random_tucker((n, n, n), (3, 2, 4), seed=31)
    x = _plain(api, X, dtype=1)
    y = api.Tucker(n, cap=3 * 4 + 1, core_cap=1, dtype=1)
    api.tucker_apply(pb, x, y)
    core, fac = y.to_numpy(others=[x])
    ref = tucker.matvec(terms, X, dense=True)
    assert rel(tucker.full((core, fac)), tucker.full(ref)) < F32_TOL
    ctx = api.Ctx(n, P.RP * 4 + 8, 8, dtype=1)
    v = api.Tucker(n, cap=P.RP * 4 + 8, core_cap=1, dtype=1)
    api.fd_precond_apply(pb, ctx, x, v)
    got = tucker.full(v.to_numpy(others=[x]))
    assert rel(got, tucker.full(P.apply(X))) < F32_TOL
    Y = synth.random_tucker((n, n, n), (2, 5, 3), seed=32)
    yy = _plain(api, Y, dtype=1)
    d = api.tucker_dot(ctx, x, yy).item()
    assert abs(d - tucker.dot(X, Y)) <= 1e-5 * tucker.norm(X) * tucker.norm(Y)


@pytest.mark.parametrize("eps", [2e-3, 3e-2])
def test_f32_round_rank_rule_and_tensor(api, eps):
    n = 45
    d = np.array([1.0, 0.5, 0.1, 3e-3, 1e-3, 2e-4, 1e-5])
    Y = _rotated_superdiagonal(d, n, seed=5)
    ctx = api.Ctx(n, 64, 32, dtype=1)
    y = _plain(api, Y, cap=16, core_cap=16 ** 3, dtype=1)
    api.tucker_round(ctx, y, eps)
    G, U = y.to_numpy()
    G0, U0 = rounding.t_rel(Y, eps)
    assert G.shape == G0.shape
    assert rel(tucker.full((G, U)), tucker.full((G0, U0))) < F32_TOL


def test_f32_round_block_tensor(api):
    n, p, R = 37, 3, 4
    terms = random_banded_terms(n, p, R, seed=9)
    f = synth.random_tucker((n, n, n), (1, 1, 1), seed=8)
    pb = api.tpcg_problem_create(n, p, terms, f[0], f[1], identity_tables(n), dtype=1)
    X = synth.random_tucker((n, n, n), (2, 3, 2), seed=6)
    x = _plain(api, X, dtype=1)
    y = api.Tucker(n, cap=16, core_cap=16 ** 3, dtype=1)
    api.tucker_apply(pb, x, y)
    ctx = api.Ctx(n, 16, 16, dtype=1)
    api.tucker_round(ctx, y, 1e-4)
    G, U = y.to_numpy()
    ref = tucker.matvec(terms, X)
    G0, U0 = rounding.t_rel(ref, 1e-4)
    assert G.shape == G0.shape
    assert rel(tucker.full((G, U)), tucker.full(ref)) < 1e-4
