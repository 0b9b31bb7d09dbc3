"""Continuous-batching server: requests of different n, degree, geometry and rank budget overlap on the device,
and each result is the same as when the request runs alone."""
import numpy as np
import pytest

from oracle import tucker
from tests.gpu_helpers import rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_00632_gb300 import lib, serve
    lib.load()
    return lib, serve


def _requests(lib, serve, dtype):
    import synth
    arr = synth.poisson_arrivals(200.0, 10, seed=5)
    shapes = [(lib.GEOM_TWIST, 0.12, 3, 24, 20), (lib.GEOM_CUBE, 0.0, 2, 20, 12), (lib.GEOM_TWIST, 0.27, 2, 32, 24),
              (lib.GEOM_CUBE, 0.0, 3, 28, 16), (lib.GEOM_TWIST, 0.05, 3, 16, 16)]
    return [serve.Request(*shapes[i % len(shapes)], tol=1e-6, dtype=dtype, arrival=float(arr[i]))
            for i in range(len(arr))]


@pytest.mark.parametrize("dtype_name", ["MIXED", "F64"])
def test_results_same_alone_and_in_the_mix(mods, dtype_name):
    lib, serve = mods
    dtype = getattr(lib, dtype_name)
    reqs = _requests(lib, serve, dtype)
    free, _ = torch.cuda.mem_get_info()
    alone = serve.Server(free // 4, max_slots=1, keep_solutions=True).run(reqs)
    mixed_srv = serve.Server(free // 4, max_slots=8, keep_solutions=True)
    mix = mixed_srv.run(reqs)
    for a, b in zip(alone, mix):
        assert a.request == b.request
        assert a.status == b.status == 0
        # the mixed form stops on the true FP64 residual; FP64 Alg. 5 stops on the truncated residual, which
        # the true one may exceed by the last truncations (eta_k of eq. rel_tol_iterates)
        assert b.true_rel_res <= (1e-6 if dtype == lib.MIXED else 2e-6)
        assert (a.iters, a.outer_iters, a.rank) == (b.iters, b.outer_iters, b.rank)
        assert rel(tucker.full((b.core, b.factors)), tucker.full((a.core, a.factors))) < 1e-13
    # in the mix requests overlapped: some were admitted before an earlier one had finished
    overlapped = sum(1 for i in range(1, len(mix)) if mix[i].admitted < max(m.finished for m in mix[:i]))
    assert overlapped >= 1
    p = serve.percentiles(mix)
    assert 0 < p["p50"] <= p["p99"]


def test_admission_respects_memory_budget(mods):
    lib, serve = mods
    reqs = _requests(lib, serve, lib.F64)[:4]
    srv = serve.Server(1 << 40, max_slots=8)
    fp = [srv.footprint(r, srv.problem(r)) for r in reqs]
    budget = max(fp)
    res = serve.Server(budget, max_slots=8).run(reqs)
    # two requests whose footprints do not fit together never overlap in time
    for i in range(len(res)):
        for j in range(i + 1, len(res)):
            if fp[i] + fp[j] > budget:
                a, b = res[i], res[j]
                assert a.finished <= b.admitted + 1e-3 or b.finished <= a.admitted + 1e-3
    need = budget
    with pytest.raises(ValueError, match="more than the whole budget"):
        serve.Server(need // 2, max_slots=8).run(reqs)


def test_poisson_and_elasticity_requests_share_the_device(mods):
    # the serving mix of Poisson and elasticity requests: each result equals the request alone
    lib, serve = mods
    import synth
    arr = synth.poisson_arrivals(300.0, 6, seed=9)
    reqs = []
    for i in range(6):
        if i % 2:
            reqs.append(serve.Request(lib.GEOM_TWIST, 0.1 + 0.02 * i, 2, 12, 12, tol=1e-6, dtype=lib.F64,
                                      arrival=float(arr[i]), problem="elasticity", lame_mu=0.3 + 0.1 * i,
                                      lame_lambda=1.0, force=(0.0, 0.1, -1.0)))
        else:
            reqs.append(serve.Request(lib.GEOM_TWIST, 0.1 + 0.02 * i, 3, 16, 16, tol=1e-6, dtype=lib.MIXED,
                                      arrival=float(arr[i])))
    free, _ = torch.cuda.mem_get_info()
    alone = serve.Server(free // 4, max_slots=1, keep_solutions=True).run(reqs)
    mix = serve.Server(free // 4, max_slots=6, keep_solutions=True).run(reqs)
    for a, b in zip(alone, mix):
        assert a.status == b.status == 0 and b.true_rel_res <= 1e-6
        if a.request.problem == "elasticity":
            for i in range(3):
                assert rel(tucker.full((b.core[i], b.factors[i])), tucker.full((a.core[i], a.factors[i]))) < 1e-13
        else:
            assert rel(tucker.full((b.core, b.factors)), tucker.full((a.core, a.factors))) < 1e-13


def test_setup_in_latency_builds_each_operator_once_and_matches(mods):
    # operators built after their requests arrive: one build per description, the build time inside the latency
    # of the requests that waited for it, and the same results as with operators built beforehand
    lib, serve = mods
    reqs = _requests(lib, serve, lib.MIXED)
    free, _ = torch.cuda.mem_get_info()
    ref = serve.Server(free // 4, max_slots=8, keep_solutions=True).run(reqs)
    srv = serve.Server(free // 4, max_slots=8, keep_solutions=True, setup_in_latency=True)
    res = srv.run(reqs)
    assert len(srv._problems) == 5                       # five descriptions among the ten requests
    for a, b in zip(ref, res):
        assert a.request == b.request and a.status == b.status == 0
        assert (a.iters, a.outer_iters, a.rank) == (b.iters, b.outer_iters, b.rank)
        assert rel(tucker.full((b.core, b.factors)), tucker.full((a.core, a.factors))) < 1e-13
        assert b.admitted >= b.request.arrival + b.setup_s - 1e-3
    assert not res[0].cache_hit and res[0].setup_s > 0.0
    assert sum(1 for r in res if not r.cache_hit) >= 5
