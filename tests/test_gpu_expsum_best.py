"""The setup's best exponential sums (the default, tpcg_set_option(TPCG_OPT_EXPSUM_BEST, 1)): R_P and the sums
equal the oracle's Remez exchange, the FD preconditioner built from them equals the oracle's Alg. 4 with the
same sums, TPCG converges with it, and the sinc-search setup (option 0) needs more terms."""
import numpy as np
import pytest

import synth
from oracle import expsum, fd, tucker
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


def test_setup_with_best_sums(mods):
    api, lib = mods
    n, p, amp = 20, 3, 0.2
    pb = api.tpcg_setup(lib.GEOM_TWIST, amp, p, n)
    info = pb.info
    ex = pb.export()
    R, om, al, E, E_prev = expsum.rp_best(info.MP, 0.1)
    assert info.RP == R and E * info.MP <= 0.1 < E_prev * info.MP
    a, b = np.argsort(np.asarray(ex["alpha"])), np.argsort(al)
    assert np.allclose(np.asarray(ex["alpha"])[a], al[b], rtol=1e-8)
    assert np.allclose(np.asarray(ex["omega"])[a], om[b], rtol=1e-8)
    # fewer terms than the sinc-search setup of the same problem
    api.set_option(lib.OPT_EXPSUM_BEST, 0)
    try:
        rp_sinc = api.tpcg_setup(lib.GEOM_TWIST, amp, p, n).info.RP
    finally:
        api.set_option(lib.OPT_EXPSUM_BEST, 1)
    assert info.RP < rp_sinc
    # Alg. 4 on the GPU with these sums against the oracle's Alg. 4 with the same sums
    P = fd.ApproxFD(n, p, expsum=(np.asarray(ex["omega"]), np.asarray(ex["alpha"])))
    S = synth.random_tucker((n, n, n), (2, 3, 2), seed=31)
    s = api.Tucker.from_numpy(S[0], S[1])
    ctx = api.Ctx(n, info.RP * 3 + 8, 8)
    v = api.Tucker(n, cap=info.RP * 3 + 8, core_cap=1)
    api.fd_precond_apply(pb, ctx, s, v)
    got = tucker.full(v.to_numpy(others=[s]))
    ref = tucker.full(P.apply(S))
    assert rel(got, ref) < 1e-10
    # TPCG (FP64, ranks uncapped) converges with the best-sum preconditioner, in as many iterations as the
    # oracle's Alg. 5 with the same sums on the oracle's own setup of the problem
    from oracle import tpcg as otp
    from tests.gpu_helpers import oracle_problem
    terms, f, _, _ = oracle_problem("twist", amp, n, p)
    _, info_o = otp.tpcg(terms, f, P.apply, otp.Params(tol=1e-6))
    rc = n
    ctx2 = api.Ctx(n, api.max_cols_for(info, rc, lib.F64), rc)
    x = api.Tucker(n, cap=rc, core_cap=rc ** 3)
    st = api.tpcg_solve(pb, ctx2, x, tol=1e-6, rank_cap=rc)
    torch.cuda.synchronize()
    assert st.status == 0 and st.true_rel_res <= 1e-6
    assert abs(st.iters - info_o["iters"]) <= 2
