"""Host logic of the server's set-up-in-latency mode, on the CPU: the operator of a description is built once
however many requests wait for it, concurrently across descriptions; requests record whether their operator was
cached when they arrived and how long they waited for its build; a request whose set-up fails reports status -1
without stopping the others.  The device work (set-up upload, solve) is replaced by stand-ins."""
import threading
import time

import pytest

torch = pytest.importorskip("torch")


def _server(monkeypatch, build_s=0.2, fail_n=None):
    from paper_2306_00632_gb300 import serve
    builds = []
    lock = threading.Lock()

    def build(r):
        with lock:
            builds.append((r.n, time.perf_counter()))
        time.sleep(build_s)
        if fail_n is not None and r.n == fail_n:
            raise RuntimeError("set-up failed")
        return object()

    def solve_in_slot(self, r, pb, t0, admitted, out, idx, setup_s, hit):
        time.sleep(0.05)
        out[idx] = serve.Result(r, 0, 1, 0, 0.0, (1, 1, 1), admitted, time.perf_counter() - t0, None, None,
                                setup_s, hit)

    monkeypatch.setattr(serve.Server, "_build", staticmethod(build))
    monkeypatch.setattr(serve.Server, "footprint", lambda self, r, pb: 1)
    monkeypatch.setattr(serve.Server, "_solve_in_slot", solve_in_slot)
    return serve, serve.Server(10, max_slots=4, setup_in_latency=True), builds


def _req(serve, n, t):
    return serve.Request(1, 0.1, 3, n, 8, arrival=t)


def test_one_build_per_description_and_cache_hits(monkeypatch):
    serve, srv, builds = _server(monkeypatch)
    reqs = [_req(serve, 16, 0.0), _req(serve, 16, 0.01), _req(serve, 24, 0.02), _req(serve, 16, 0.5)]
    res = srv.run(reqs)
    assert sorted(n for n, _ in builds) == [16, 24]                  # one build per description
    assert [r.cache_hit for r in res] == [False, False, False, True]  # the last arrives after the build
    assert res[1].setup_s > 0.1                                        # waited for the first request's build
    assert res[3].setup_s < 0.05
    # the two descriptions built concurrently, not one after the other
    t16 = next(t for n, t in builds if n == 16)
    t24 = next(t for n, t in builds if n == 24)
    assert abs(t24 - t16) < 0.15
    for r in res:
        assert r.status == 0 and r.admitted >= r.request.arrival + r.setup_s - 1e-3


def test_failed_setup_fails_only_its_requests(monkeypatch):
    serve, srv, _ = _server(monkeypatch, build_s=0.05, fail_n=24)
    res = srv.run([_req(serve, 16, 0.0), _req(serve, 24, 0.0), _req(serve, 32, 0.01)])
    assert [r.status for r in res] == [0, -1, 0]
    assert res[1].error
