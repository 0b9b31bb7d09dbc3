"""Many solves at once (tpcg_solve_batch): each result equals the same solve run alone, and the batch
matches the oracle's Alg. 5.  Problems of different n, p and geometry share the device."""
import numpy as np
import pytest

from oracle import fullcg
from oracle import tpcg as otp
from oracle import tucker
from tests.gpu_helpers import gpu_problem, oracle_problem, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [("cube", 0.0, 12, 2), ("twist", 0.21, 14, 3), ("cube", 0.0, 18, 3), ("twist", 0.05, 16, 2)]


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_00632_gb300 import api as a
    from paper_2306_00632_gb300 import lib
    lib.load()
    return a


def _setup(api, case, dtype=0):
    kind, amp, n, p = case
    pb = gpu_problem(kind, amp, n, p, dtype=dtype)
    rc = n
    mc = max(pb.info.R * rc + max(pb.info.rf), pb.info.RP * rc, 2 * rc)
    ctx = api.Ctx(n, mc, rc, dtype)
    x = api.Tucker(n, cap=rc, core_cap=rc ** 3, dtype=dtype)
    return pb, ctx, x


def test_batch_equals_alone_and_oracle(api):
    kw = dict(tol=1e-8)
    alone = []
    for case in CASES:
        pb, ctx, x = _setup(api, case)
        st = api.tpcg_solve(pb, ctx, x, **kw)
        torch.cuda.synchronize()
        alone.append((x.to_numpy(), st.iters, tuple(st.rank), st.status))
    objs = [_setup(api, case) for case in CASES]
    streams = [torch.cuda.Stream() for _ in CASES]
    codes, sts = api.tpcg_solve_batch([o[0] for o in objs], [o[1] for o in objs], [o[2] for o in objs], streams,
                                      **kw)
    torch.cuda.synchronize()
    for i, case in enumerate(CASES):
        (core_a, fac_a), it_a, rk_a, code_a = alone[i]
        core_b, fac_b = objs[i][2].to_numpy()
        assert codes[i] == code_a == 0
        assert sts[i].iters == it_a and tuple(sts[i].rank) == rk_a
        # same kernels on the same inputs: the tensors agree to rounding (in practice bit for bit)
        assert rel(tucker.full((core_b, fac_b)), tucker.full((core_a, fac_a))) < 1e-13
        # and the solve is Alg. 5's: true residual on the assembled system, and the oracle's solution
        kind, amp, n, p = case
        terms, f, P, _ = oracle_problem(kind, amp, n, p)
        xg = tucker.vec(tucker.full((core_b, fac_b)))
        fv = tucker.vec(tucker.full(f))
        assert np.linalg.norm(fv - fullcg.assemble(terms) @ xg) <= 2e-8 * np.linalg.norm(fv)
        xo, _ = otp.tpcg(terms, f, P.apply, otp.Params(tol=1e-8))
        assert rel(xg, tucker.vec(tucker.full(xo))) < 1e-6


def test_batch_rejects_shared_context(api):
    from paper_2306_00632_gb300 import lib
    pb, ctx, x = _setup(api, CASES[0])
    s = [torch.cuda.Stream(), torch.cuda.Stream()]
    with pytest.raises(lib.TpcgError, match="its own context"):
        api.tpcg_solve_batch([pb, pb], [ctx, ctx], [x, x], s)
