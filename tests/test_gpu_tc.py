"""FP32 contractions on the tensor cores (tcgen05, 3xTF32 with FP32 accumulation; TPCG_OPT_TC = 1) against
the FP32 SIMT path and the FP64 oracle: Alg. 1 on plain and block tensors whose contractions span several
128 x 128 output tiles, K chunks with ragged tails and strided batches, the Tucker scalar product, and a
mixed-precision solve whose inner FP32 solves run every contraction on the tensor cores."""
import numpy as np
import pytest

import synth
from oracle import rounding, tucker
from tests.gpu_helpers import identity_tables, random_banded_terms, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_00632_gb300 import api as a
    from paper_2306_00632_gb300 import lib
    lib.load()
    yield a
    a.set_option(lib.OPT_TC, 0)


def _tc(api, on):
    from paper_2306_00632_gb300 import lib
    api.set_option(lib.OPT_TC, 1 if on else 0)


def _round(api, Y, n, eps, cap, dt, on):
    _tc(api, on)
    y = api.Tucker.from_numpy(Y[0], Y[1], cap=cap, core_cap=cap ** 3, dtype=dt)
    ctx = api.Ctx(n, cap, cap, dtype=dt)
    info = torch.zeros(6, dtype=torch.float64, device="cuda")
    api.tucker_round(ctx, y, eps, info=info)
    torch.cuda.synchronize()
    return y.to_numpy(), info.cpu().numpy()


@pytest.mark.parametrize("n,ranks,eps", [(45, (7, 9, 5), 1e-3), (130, (70, 40, 66), 1e-2), (128, (128, 100, 90), 3e-3)])
def test_tc_round_matches_simt_and_oracle(api, n, ranks, eps):
    Y = synth.random_tucker((n, n, n), ranks, seed=51, decay=0.8)
    cap = max(ranks)
    (G1, U1), h1 = _round(api, Y, n, eps, cap, 1, True)
    (G0, U0), h0 = _round(api, Y, n, eps, cap, 1, False)
    _tc(api, False)
    full = tucker.full(Y)
    nf = np.linalg.norm(full)
    assert rel(h1[0], h0[0]) < 1e-5                              # ||Z||^2 of the same Z formation
    # both are truncations of Y within the bound of Alg. 1 plus the FP32 Gram's resolution of the discarded
    # energy (about 1e-6 ||Z||^2 per mode); with geometric spectra a rank decision can sit at a near-tie, so
    # the two FP32 paths (and the oracle) may differ by one in a mode and by up to eps in norm
    Go, Uo = rounding.t_rel(Y, eps)
    for G, U in ((G1, U1), (G0, U0)):
        assert np.linalg.norm(tucker.full((G, U)) - full) <= np.sqrt(eps ** 2 + 3e-6) * nf * 1.01
        assert all(abs(a - b) <= 1 for a, b in zip(G.shape, Go.shape))
    assert rel(tucker.full((G1, U1)), tucker.full((G0, U0))) < 2 * eps
    if G1.shape == G0.shape:
        assert rel(tucker.full((G1, U1)), tucker.full((G0, U0))) < 0.1 * eps


def test_tc_block_round_and_dot(api):
    # an unrounded operator product (block core, 5 Kronecker terms, k = 5 r columns) rounded with the tensor
    # cores, and the scalar product of two plain tensors
    n, p, R = 93, 3, 5
    terms = random_banded_terms(n, p, R, seed=53)
    f = synth.random_tucker((n, n, n), (1, 1, 1), seed=54)
    X = synth.random_tucker((n, n, n), (9, 11, 7), seed=55)
    ref = tucker.matvec(terms, X)
    outs = []
    for on in (True, False):
        _tc(api, on)
        pb = api.tpcg_problem_create(n, p, terms, f[0], f[1], identity_tables(n), dtype=1)
        x = api.Tucker.from_numpy(X[0], X[1], dtype=1)
        y = api.Tucker(n, cap=R * 11, core_cap=64 ** 3, dtype=1)
        api.tucker_apply(pb, x, y)
        ctx = api.Ctx(n, R * 11, 64, dtype=1)
        api.tucker_round(ctx, y, 1e-5)
        outs.append(tucker.full(y.to_numpy()))
        Y2 = synth.random_tucker((n, n, n), (13, 6, 10), seed=56)
        y2 = api.Tucker.from_numpy(Y2[0], Y2[1], dtype=1)
        d = api.tucker_dot(ctx, x, y2).item()
        assert abs(d - tucker.dot(X, Y2)) <= 1e-5 * tucker.norm(X) * tucker.norm(Y2)
    _tc(api, False)
    assert rel(outs[0], outs[1]) < 5e-5
    assert rel(outs[0], tucker.full(ref)) < 2e-5


def test_tc_mixed_solve_converges(api):
    from paper_2306_00632_gb300 import lib
    n = 48
    sts = []
    for on in (True, False):
        _tc(api, on)
        pb = api.tpcg_setup(lib.GEOM_TWIST, synth.amp_from_seed(7), 3, n, lib.MIXED)
        ctx = api.Ctx(n, api.max_cols_for(pb.info, n, lib.MIXED), n, lib.MIXED)
        x = api.Tucker(n, cap=n, core_cap=n ** 3, dtype=lib.MIXED)
        sts.append(api.tpcg_solve(pb, ctx, x, tol=1e-6))
        torch.cuda.synchronize()
    _tc(api, False)
    for st in sts:
        assert st.status == 0 and st.true_rel_res <= 1e-6
    assert abs(sts[0].iters - sts[1].iters) <= max(3, sts[1].iters // 5)
