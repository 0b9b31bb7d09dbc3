"""Alg. 1 below the resolution of one FP64 mode Gram.  A Gram carries rounding errors of about eps_machine ||Y||^2,
so at eps ~ 1e-8 its smallest eigenvalues, the energies the budget eps^2 ||Y||^2 / 3 is about, are noise.  The
resolved rule (TPCG_OPT_ROUND_RULE 2; the default of FP64 solves below 1e-8) rounds the resolved part first and
the remainder against the absolute budget: the result meets ||Y - Y~|| <= eps ||Y|| as the oracle's SVD-based
truncation does.  The input is a rank-20 tensor with singular values down to 1e-6 plus a rank-6 tensor of relative
size 1e-8, which an eps of 3e-9 must mostly keep."""
import numpy as np
import pytest

from oracle import rounding, tucker

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_00632_gb300 import api, lib
    lib.load()
    yield api, lib
    api.set_option(lib.OPT_ROUND_RULE, -1)


def _input(n=40, seed=11):
    g = np.random.default_rng(seed)
    d = np.logspace(0, -6, 20)
    Qx = [np.linalg.qr(g.standard_normal((n, 20)))[0] for _ in range(3)]
    X = (tucker.superdiagonal(d), Qx)
    Gd = g.standard_normal((6, 6, 6))
    Ud = [np.linalg.qr(g.standard_normal((n, 6)))[0] for _ in range(3)]
    scale = 1e-8 * np.linalg.norm(d) / np.linalg.norm(Gd)
    core = np.zeros((26, 26, 26))
    core[:20, :20, :20] = X[0]
    core[20:, 20:, 20:] = scale * Gd
    return core, [np.concatenate([Qx[t], Ud[t]], axis=1) for t in range(3)]


def test_resolved_rule_meets_the_bound_below_gram_resolution(mods):
    api, lib = mods
    n = 40
    core, U = _input(n)
    Y = tucker.full((core, U))
    ny = np.linalg.norm(Y)
    eps = 3e-9
    ref = rounding.t_rel((core, U), eps)
    assert np.linalg.norm(tucker.full(ref) - Y) <= eps * ny          # the oracle meets it
    api.set_option(lib.OPT_ROUND_RULE, 2)
    # the two parts are merged losslessly, so the result may carry more columns than the input's 26
    y = api.Tucker.from_numpy(core, U, cap=n, core_cap=n ** 3)
    ctx = api.Ctx(n, 3 * n, n, lib.F64)
    api.tucker_round(ctx, y, eps)
    torch.cuda.synchronize()
    c, f = y.to_numpy()
    err = np.linalg.norm(tucker.full((c, f)) - Y)
    assert err <= eps * ny * (1 + 1e-6)
    # close to the SVD's ranks (measured 28, 27, 26 against 25, 25, 25): the lossless merge keeps a few
    # directions the two parts share
    for t in range(3):
        assert f[t].shape[1] <= ref[1][t].shape[1] + 6
    # most of the small component survives: its removal alone would cost 1e-8 ||Y||
    assert err <= 0.5e-8 * ny
    # and at a tolerance one pass resolves, the rule is the plain one: same ranks as the oracle
    y2 = api.Tucker.from_numpy(core, U, cap=26, core_cap=26 ** 3)
    api.tucker_round(ctx, y2, 1e-5)
    torch.cuda.synchronize()
    assert [u.shape[1] for u in y2.to_numpy()[1]] == [u.shape[1] for u in rounding.t_rel((core, U), 1e-5)[1]]
