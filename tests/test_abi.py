"""The C-ABI library builds for sm_103a, loads, and exports every function include/tpcg.h declares
(no compute calls: this runs without a GPU)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tpcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b((?:tpcg|tucker|fd)_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_builds_loads_and_exports_all_symbols():
    from paper_2306_00632_gb300 import build, lib
    path = build.build()
    assert os.path.exists(path)
    L = lib.load(build_if_missing=False)
    declared = _declared()
    assert len(declared) >= 19
    for name in declared:
        assert hasattr(L, name), name
    assert set(declared) == set(lib.SYMBOLS)
    assert L.tpcg_version().decode().startswith("tpcg-gb300")


def test_ctx_bytes_is_host_only_and_monotone():
    from paper_2306_00632_gb300 import lib
    L = lib.load()
    a = L.tpcg_ctx_bytes(128, 1024, 64, 0)
    b = L.tpcg_ctx_bytes(128, 2048, 64, 0)
    c = L.tpcg_ctx_bytes(128, 2048, 64, 1)
    assert 0 < a < b and c < b


def test_expsum_best_is_host_only_and_matches_the_oracle():
    # tpcg_expsum_best (the setup's best sums, no GPU call) against the oracle's Remez exchange and Table 1:
    # the best approximation is unique, so the two independent implementations agree to rounding
    import json
    import numpy as np
    from oracle import expsum
    from paper_2306_00632_gb300 import api
    t1 = json.load(open(os.path.join(ROOT, "tests", "golden", "table1.json")))
    for p in ("2", "3"):
        M, want = t1["M_P"][p][0], t1["R_P"][p][0]
        om, al, E = api.expsum_best(M, 0.1)
        R, om_o, al_o, E_o, _ = expsum.rp_best(M, 0.1)
        assert len(om) == R == want
        a, b = np.argsort(al), np.argsort(al_o)
        assert np.allclose(al[a], al_o[b], rtol=1e-8) and np.allclose(om[a], om_o[b], rtol=1e-8)
        assert abs(E - E_o) <= 1e-8 * E_o and E * M <= 0.1
        om2, al2, E2 = api.expsum_best(M, 0.1)   # served from the per-M cache: the same sums
        assert np.array_equal(om, om2) and np.array_equal(al, al2) and E2 == E
    # small M (few terms): the same best sums from both implementations
    for M in (3.0, 40.0, 700.0, 5.0e3):
        om, al, E = api.expsum_best(M, 0.1)
        R, om_o, al_o, E_o, _ = expsum.rp_best(M, 0.1)
        assert len(om) == R
        a, b = np.argsort(al), np.argsort(al_o)
        assert np.allclose(al[a], al_o[b], rtol=1e-7) and np.allclose(om[a], om_o[b], rtol=1e-7)
    # invalid arguments are rejected before any work
    import ctypes as C
    from paper_2306_00632_gb300 import lib
    L = lib.load()
    buf = (C.c_double * 4)()
    R = C.c_int(0)
    assert L.tpcg_expsum_best(0.5, 0.1, 4, buf, buf, C.byref(R), None) == 1    # M < 1
    assert L.tpcg_expsum_best(2.3e4, 0.1, 4, buf, buf, C.byref(R), None) == 1  # no R <= 4 meets the bound


def test_problem_create_refuses_non_finite_tables_on_the_host():
    # a NaN in the right-hand side (or an Inf in a band) is refused by the host-side check of
    # tpcg_problem_create before any device call, so this runs without a GPU
    import numpy as np
    import pytest
    from paper_2306_00632_gb300 import api, lib
    from tests.gpu_helpers import oracle_problem
    n, p = 8, 2
    terms, f, P, tables = oracle_problem("cube", 0.0, n, p)
    core = np.array(f[0], dtype=float)
    core.flat[0] = np.nan
    with pytest.raises(lib.TpcgError, match="NaN or an Inf") as e:
        api.tpcg_problem_create(n, p, terms, core, f[1], tables)
    assert e.value.code == lib.STATUS_CODES["E_INVALID"]
    bad = [(w, [m.copy() for m in mats]) for w, mats in terms]
    bad[1][1][2][3, 3] = np.inf
    with pytest.raises(lib.TpcgError, match="NaN or an Inf"):
        api.tpcg_problem_create(n, p, bad, f[0], f[1], tables)
