"""The FP32 ST-HOSVD eigensolver at the size the benchmark runs it: 128 x 128 mode Grams (Alg. 1 step 3).

The input is a plain FP32 Tucker tensor with n = 128, full factor rank 128 (so Alg. 1 forms Z = the whole
128^3 tensor, no QR) and a superdiagonal core d_i = 10^(-i/8) behind random orthonormal factors: every mode
Gram is a dense 128 x 128 matrix with eigenvalues d_i^2 spread over 32 decades (most of them far below FP32
resolution).  eps is placed so that the budget eps^2 ||Z||^2 / 3 of each mode sits between two consecutive
tails of the spectrum with margins of at least 1.6e-4 ||Z||^2, over ten times the FP32 resolution of the
rule (trace minus kept eigenvalues: 1e-6 to 1e-5 ||Z||^2 over three modes, the rounding of the FP32 Gram and
of its factorisation included).  The rounding must then make the oracle's rank decision in all three modes,
report the oracle's discarded energy to FP32 accuracy, keep the dominant subspaces, and return the same
tensor."""
import numpy as np
import pytest

from oracle import rounding, tucker
from tests.gpu_helpers import rel

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


def _case(n=128, seed=11):
    g = np.random.default_rng(seed)
    d = 10.0 ** (-np.arange(n) / 8.0)
    G = np.zeros((n, n, n))
    G[np.arange(n), np.arange(n), np.arange(n)] = d
    U = [np.linalg.qr(g.standard_normal((n, n)))[0] for _ in range(3)]
    tail = np.cumsum((d ** 2)[::-1])[::-1]
    budget = np.sqrt(tail[10] * tail[9])           # between the mode-1 tails at s = 9 and s = 10
    eps = float(np.sqrt(3.0 * budget / np.sum(d ** 2)))
    return (G, U), eps


def test_f32_gram_128_rank_discarded_subspace(api):
    n = 128
    Y, eps = _case(n)
    (G0, U0), inf0 = rounding.t_rel(Y, eps, return_info=True)
    assert G0.shape == (10, 9, 9)                   # the oracle's decisions (margins checked on the CPU)
    y = api.Tucker.from_numpy(Y[0], Y[1], cap=n, core_cap=n ** 3, dtype=1)
    ctx = api.Ctx(n, n, n, dtype=1)
    info = torch.zeros(6, dtype=torch.float64, device="cuda")
    api.tucker_round(ctx, y, eps, info=info)
    torch.cuda.synchronize()
    h = info.cpu().numpy()
    G, U = y.to_numpy()
    # rank decision of every mode
    assert G.shape == G0.shape and tuple(int(v) for v in h[2:5]) == G0.shape
    # ||Z||^2 and the discarded energy (trace minus kept eigenvalues in FP32)
    assert abs(h[0] - inf0["norm2"]) <= 1e-6 * inf0["norm2"]
    assert abs(h[1] - inf0["discarded"]) <= 1e-5 * inf0["norm2"]
    # kept subspaces: the oracle's 6 leading singular vectors of each mode (eigenvalue gaps >= 1e-2 of the
    # largest) lie in the span of the GPU factor; the GPU factors are orthonormal to FP32 accuracy
    for t in range(3):
        assert np.abs(U[t].T @ U[t] - np.eye(U[t].shape[1])).max() < 1e-5
        lead = U0[t][:, :6]
        resid = lead - U[t] @ (U[t].T @ lead)
        assert np.linalg.norm(resid, 2) < 1e-3
    # the truncated tensors agree within the truncation tolerance, and the error bound of Alg. 1 holds
    full = tucker.full(Y)
    assert rel(tucker.full((G, U)), tucker.full((G0, U0))) < 2 * eps
    assert np.linalg.norm(tucker.full((G, U)) - full) <= eps * np.linalg.norm(full) * (1 + 1e-3)
