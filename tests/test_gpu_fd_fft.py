"""The FFT sine transforms of the preconditioner (Alg. 4 with App. B, chirp-z FFTs of any length) against the
oracle and against the library's dense sine product.

n1 (the sine-transform length) covers DST-I (odd p, length n1 = n - p + 1) and DST-II/III (even p, n1 =
n - p + 2) with FFT sizes 32 to 1024, including lengths whose doubled DFT size has a large prime factor
(n1 = 126: DFT length 254 = 2 127) and the n = 512 benchmark-family size."""
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
    yield a
    a.set_option(lib.OPT_DST, 1)


def _fd(api, pb, ctx, s, cap, kind):
    from paper_2306_00632_gb300 import lib
    api.set_option(lib.OPT_DST, kind)
    v = api.Tucker(s.n, cap=cap, core_cap=1, dtype=s.dtype)
    api.fd_precond_apply(pb, ctx, s, v)
    return v.to_numpy(others=[s])


@pytest.mark.parametrize("n,p", [(17, 2), (24, 3), (33, 4), (128, 3), (66, 4), (40, 5)])
def test_fft_sine_transforms_match_oracle_and_dense(api, n, p):
    pb = gpu_problem("cube", 0.0, n, p)
    _, _, P, _ = oracle_problem("cube", 0.0, n, p)
    S = synth.random_tucker((n, n, n), (3, 2, 4), seed=23)
    s = api.Tucker.from_numpy(S[0], S[1])
    cap = P.RP * 4 + 4
    ctx = api.Ctx(n, cap, 8)
    core_f, fac_f = _fd(api, pb, ctx, s, cap, 1)
    core_d, fac_d = _fd(api, pb, ctx, s, cap, 0)
    for t in range(3):
        assert rel(fac_f[t], fac_d[t]) < 1e-12
    assert rel(core_f, core_d) == 0.0
    if n <= 70:   # the oracle's dense Alg. 4 (App. B eigenvectors by interpolation)
        ref = P.apply(S)
        for t in range(3):
            assert rel(fac_f[t], ref[1][t]) < 1e-11


def test_fft_sine_transforms_fp32_and_n512(api):
    # FP32 at the benchmark size, and the n = 512 family size (n1 = 510, FFT size 1024) in FP64
    from paper_2306_00632_gb300 import lib
    for n, p, dt, tol in ((128, 3, lib.F32, 2e-6), (512, 3, lib.F64, 1e-12)):
        pb = api.tpcg_setup(lib.GEOM_TWIST, 0.1, p, n, dt)
        S = synth.random_tucker((n, n, n), (2, 3, 2), seed=29)
        s = api.Tucker.from_numpy(S[0], S[1], dtype=dt)
        cap = pb.info.RP * 3 + 2
        ctx = api.Ctx(n, cap, 4, dt)
        _, fac_f = _fd(api, pb, ctx, s, cap, 1)
        _, fac_d = _fd(api, pb, ctx, s, cap, 0)
        for t in range(3):
            assert rel(fac_f[t], fac_d[t]) < tol
