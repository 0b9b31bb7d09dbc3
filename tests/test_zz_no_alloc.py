"""The allocation-free Tucker dot (tucker_dot_static) against the context-based tucker_dot and the oracle.

Collected last on purpose: it must also pass after every other GPU test has run in the same process."""
import numpy as np
import pytest

import synth
from oracle import tucker

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


@pytest.mark.parametrize("dtype,tol", [(0, 1e-12), (1, 1e-5)])
def test_dot_static_matches_dot(api, dtype, tol):
    n = 97
    # ranks span several 64-wide GEMM tiles of the contraction up to the fixed limit of 64
    X = synth.random_tucker((n, n, n), (64, 33, 17), seed=41)
    Y = synth.random_tucker((n, n, n), (5, 64, 40), seed=42)
    x = api.Tucker.from_numpy(X[0], X[1], cap=64, dtype=dtype)
    y = api.Tucker.from_numpy(Y[0], Y[1], cap=64, dtype=dtype)
    ctx = api.Ctx(n, 128, 64, dtype=dtype)
    ref = api.tucker_dot(ctx, x, y).item()
    scale = tucker.norm(X) * tucker.norm(Y)
    assert abs(ref - tucker.dot(X, Y)) <= tol * scale
    # two calls in a row through the fixed scratch, then the self dot
    out = torch.full((2,), np.nan, dtype=torch.float64, device="cuda")
    api.tucker_dot_static(x, y, out=out[0:1])
    api.tucker_dot_static(x, y, out=out[1:2])
    got = out.cpu().numpy()
    assert np.all(np.abs(got - ref) <= tol * scale)
    xx = api.tucker_dot_static(x, x).item()
    assert abs(xx - api.tucker_dot(ctx, x, x).item()) <= tol * tucker.norm(X) ** 2
    # nothing is allocated on the device by further calls: free device memory is unchanged across them
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for q in range(2):
        api.tucker_dot_static(x, y, out=out[q:q + 1])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.all(np.abs(out.cpu().numpy() - ref) <= tol * scale)


def test_dot_static_rejects_ranks_above_limit(api):
    n = 16
    X = synth.random_tucker((n, n, n), (2, 2, 2), seed=43)
    x = api.Tucker.from_numpy(X[0], X[1], cap=65)
    y = api.Tucker.from_numpy(X[0], X[1], cap=8)
    from paper_2306_00632_gb300 import lib
    with pytest.raises(lib.TpcgError, match="exceeds the fixed scratch limit"):
        api.tucker_dot_static(x, y)
