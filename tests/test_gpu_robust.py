"""Failure paths of the solver and the public scalar product, and isolation of concurrent solves that share
one problem.  Every failure here is made on the host side (an iteration cap, an indefinite operator, a
block tensor passed where a plain one is required, an undersized output); no kernel is given data it could
read or write out of bounds."""
import threading

import numpy as np
import pytest

import synth
from oracle import tucker
from tests.gpu_helpers import gpu_problem, oracle_problem, rel

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


def _twist(api, n=12, p=3):
    amp = synth.amp_from_seed(7)
    terms, f, P, tables = oracle_problem("twist", amp, n, p)
    pb = gpu_problem("twist", amp, n, p)
    ctx = api.Ctx(n, max(len(terms) * n + max(f[0].shape), P.RP * n, 2 * n), n)
    return pb, ctx, terms, f, P, tables


def test_not_converged_at_iteration_cap(api):
    from paper_2306_00632_gb300 import lib
    n = 12
    pb, ctx, *_ = _twist(api, n)
    x = api.Tucker(n, cap=n, core_cap=n ** 3)
    st = api.tpcg_solve(pb, ctx, x, tol=1e-6, max_it=1)
    assert st.status == lib.STATUS_CODES["E_NOT_CONVERGED"] and st.iters == 1
    assert st.rel_res > 1e-6


def test_breakdown_on_indefinite_operator(api):
    # -A is negative definite: the first curvature xi_0 = p_0 . q_0 of Alg. 5 is negative, which the scalar
    # update reports as a breakdown before any step is taken
    from paper_2306_00632_gb300 import lib
    n, p = 12, 3
    amp = synth.amp_from_seed(7)
    terms, f, P, tables = oracle_problem("twist", amp, n, p)
    neg = [(-w, mats) for w, mats in terms]
    pb = api.tpcg_problem_create(n, p, neg, f[0], f[1], tables)
    ctx = api.Ctx(n, max(len(terms) * n + max(f[0].shape), P.RP * n, 2 * n), n)
    x = api.Tucker(n, cap=n, core_cap=n ** 3)
    with pytest.raises(lib.TpcgError) as e:
        api.tpcg_solve(pb, ctx, x, tol=1e-6)
    assert e.value.code == lib.STATUS_CODES["E_BREAKDOWN"]
    assert api.ctx_history(ctx)[0]["xi"] < 0


def test_dot_refuses_block_tensor(api):
    from paper_2306_00632_gb300 import lib
    n = 12
    pb, ctx, terms, f, P, _ = _twist(api, n)
    X = synth.random_tucker((n, n, n), (2, 2, 2), seed=5)
    x = api.Tucker.from_numpy(X[0], X[1], cap=4)
    y = api.Tucker(n, cap=len(terms) * 2, core_cap=1)
    api.tucker_apply(pb, x, y)
    for fn in (lambda: api.tucker_dot(ctx, x, y), lambda: api.tucker_dot_static(y, x)):
        with pytest.raises(lib.TpcgError, match="not a plain tensor") as e:
            fn()
        assert e.value.code == lib.STATUS_CODES["E_INVALID"]
    assert np.isfinite(api.tucker_dot(ctx, x, x).item())


def test_shared_problem_capacity_flags_are_per_solve(api):
    # one solve runs while another stream keeps overflowing standalone products of the same problem (each
    # leaves an empty result and raises the problem's own flag): the solve keeps its own flags and its result
    # equals the same solve run alone
    n = 12
    pb, ctx, terms, f, P, _ = _twist(api, n)
    alone = api.Tucker(n, cap=n, core_cap=n ** 3)
    st0 = api.tpcg_solve(pb, ctx, alone, tol=1e-6)
    torch.cuda.synchronize()
    assert st0.status == 0
    X = synth.random_tucker((n, n, n), (3, 3, 3), seed=6)
    xs = api.Tucker.from_numpy(X[0], X[1], cap=3)
    small = api.Tucker(n, cap=len(terms) * 3 - 1, core_cap=1)     # one column short of R rank(x)
    side = torch.cuda.Stream()
    stop = threading.Event()
    calls = [0]

    def overflow_loop():
        while not stop.is_set():
            api.tucker_apply(pb, xs, small, stream=side)
            calls[0] += 1
            side.synchronize()

    th = threading.Thread(target=overflow_loop)
    th.start()
    try:
        ctx2 = api.Ctx(n, ctx.max_cols, n)
        shared = api.Tucker(n, cap=n, core_cap=n ** 3)
        st = api.tpcg_solve(pb, ctx2, shared, tol=1e-6, stream=torch.cuda.Stream())
        torch.cuda.synchronize()
    finally:
        stop.set()
        th.join()
    assert calls[0] > 0
    assert small.read_desc()[0] == 0                  # the overflowing product really was refused
    assert st.status == 0 and st.iters == st0.iters
    assert rel(tucker.full(shared.to_numpy()), tucker.full(alone.to_numpy())) < 1e-13
