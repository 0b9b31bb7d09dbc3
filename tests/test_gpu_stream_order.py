"""Set-up writes are complete before the library returns: a context and a problem created while the legacy default
stream is still busy with other work (here a queue of large matrix products on torch's default stream) give a
solve on the context's own non-blocking stream exactly the result of a solve on an idle device.  (A device memset
or a pageable upload issued on the legacy stream returns before it lands and is not ordered with non-blocking
streams: the late zero fill of the context's scalars would overwrite the solver's first scalars.)"""
import numpy as np
import pytest

from oracle import tucker

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_00632_gb300 import api, lib
    lib.load()
    return api, lib


def _solve(api, lib, busy):
    n, rc = 16, 16
    a = b = None
    if busy:   # about a second of queued work on the legacy default stream
        a = torch.randn(4096, 4096, device="cuda")
        b = torch.randn(4096, 4096, device="cuda")
        for _ in range(40):
            a = a @ b * 1e-3
    pb = api.tpcg_setup(lib.GEOM_TWIST, 0.05, 3, n, lib.F64)
    ctx = api.Ctx(n, api.max_cols_for(pb.info, rc, lib.F64), rc, lib.F64)
    s = api.ctx_stream(ctx)
    with torch.cuda.stream(s):
        x = api.Tucker(n, cap=rc, core_cap=rc ** 3, dtype=lib.F64)
        st = api.tpcg_solve(pb, ctx, x, stream=s, tol=1e-6, rank_cap=rc)
        s.synchronize()
        out = (int(st.status), int(st.iters), x.to_numpy())
    torch.cuda.synchronize()
    return out


def test_setup_writes_are_ordered_before_the_solve(mods):
    api, lib = mods
    ref = _solve(api, lib, busy=False)
    got = _solve(api, lib, busy=True)
    assert ref[0] == got[0] == 0 and ref[1] == got[1]
    R, G = tucker.full(ref[2]), tucker.full(got[2])
    assert np.linalg.norm(G - R) <= 1e-13 * np.linalg.norm(R)
