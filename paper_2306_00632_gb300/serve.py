"""Continuous-batching TPCG server on one GPU.

Requests (geometry, amplitude, degree, n, rank cap, tolerance) arrive over time.  Each admitted request gets
a slot: its own solver context, solution buffers, CUDA stream and host thread, which calls ``tpcg_solve``
(the solver's kernels are the library's; this module only schedules).  Admission is by device memory: a
request is admitted when the bytes of its context (``tpcg_ctx_bytes``) and solution fit in the budget left by
the requests in flight and a slot is free.  Requests that arrive while others are on the GPU are admitted as
soon as memory and a slot free up, so their kernels overlap on the device with the running solves.

Requests are scalar Poisson problems (``tpcg_solve``) or linear elasticity block systems (Sec. 5.3,
``tpcg_elast_solve``).  Operators and preconditioner tables are cached per problem description: they are
read-only during solves and shared by all requests on that geometry.  By default they are built before the
clock starts; with ``setup_in_latency`` a request whose operator is not cached builds it after it arrives
(host setup of App. A and B, then upload, on the request's own thread, one build per description however many
requests wait for it), and that time counts in its latency; results record the build time and whether the
operator was already cached when the request arrived.

Results do not depend on what else runs: every solve has its own workspace and the kernels are deterministic.
Set CUDA_DEVICE_MAX_CONNECTIONS=32 before the CUDA context is created: with the default of 8 hardware queues,
solves beyond the eighth share queues and wait on each other's kernels.
"""
from __future__ import annotations

import dataclasses
import threading
import time

import torch

from . import api
from . import lib as L


@dataclasses.dataclass(frozen=True)
class Request:
    kind: int                 # L.GEOM_CUBE or L.GEOM_TWIST
    amp: float
    degree: int
    n: int
    rank_cap: int
    tol: float = 1e-6
    dtype: int = L.MIXED      # elasticity requests run L.F64 or L.F32
    arrival: float = 0.0      # seconds after the start of the run
    problem: str = "poisson"  # "poisson" or "elasticity" (Sec. 5.3)
    lame_lambda: float = 0.3 / 0.52
    lame_mu: float = 1.0 / 2.6
    force: tuple = (0.0, 0.0, -1.0)


@dataclasses.dataclass
class Result:
    request: Request
    status: int
    iters: int
    outer_iters: int
    true_rel_res: float
    rank: tuple
    admitted: float           # seconds after start
    finished: float
    core: object = None       # host copies of the solution (when keep_solutions)
    factors: object = None
    setup_s: float = 0.0      # operator build time this request waited for (setup_in_latency)
    cache_hit: bool = True    # operator already built when the request arrived
    error: str = ""           # why a request failed (status -1: set-up or budget, -2: solve)

    @property
    def latency(self) -> float:
        return self.finished - self.request.arrival


class Server:
    def __init__(self, mem_budget_bytes: int, max_slots: int = 16, keep_solutions: bool = False,
                 setup_in_latency: bool = False):
        self.budget = int(mem_budget_bytes)
        self.max_slots = int(max_slots)
        self.keep = keep_solutions
        self.setup_in_latency = bool(setup_in_latency)
        self._problems = {}
        self._klocks = {}
        self._plock = threading.Lock()
        self._cv = threading.Condition()
        self._used = 0
        self._running = 0

    # ------------------------------------------------------------------ per-request resources
    @staticmethod
    def _key(r: Request):
        return (r.problem, r.kind, float(r.amp), r.degree, r.n, r.dtype, r.lame_lambda, r.lame_mu, tuple(r.force))

    @staticmethod
    def _build(r: Request):
        if r.problem == "elasticity":
            return api.tpcg_elast_setup(r.kind, r.amp, r.degree, r.n, r.lame_lambda, r.lame_mu, r.force, r.dtype)
        return api.tpcg_setup(r.kind, r.amp, r.degree, r.n, r.dtype)

    def cached(self, r: Request) -> bool:
        with self._plock:
            return self._key(r) in self._problems

    def problem(self, r: Request):
        """The operator of r's description, built on first use; different descriptions build concurrently."""
        key = self._key(r)
        with self._plock:
            pb = self._problems.get(key)
            if pb is not None:
                return pb
            lk = self._klocks.setdefault(key, threading.Lock())
        with lk:
            with self._plock:
                pb = self._problems.get(key)
            if pb is None:
                pb = self._build(r)
                with self._plock:
                    self._problems[key] = pb
            return pb

    @staticmethod
    def _shape(r: Request, pb):
        rc = min(r.rank_cap, r.n)
        if r.problem == "elasticity":
            rows = [sum(pb.R[3 * i:3 * i + 3]) * rc + 8 for i in range(3)]
            return rc, max(max(rows), pb.RP * rc, 2 * rc)
        return rc, api.max_cols_for(pb.info, rc, r.dtype)

    def footprint(self, r: Request, pb) -> int:
        """Device bytes a request holds while in flight: its context (with the solver tensors it allocates)
        and its solution buffers."""
        rc, max_cols = self._shape(r, pb)
        elt = 4 if r.dtype == L.F32 else 8
        ncomp = 3 if r.problem == "elasticity" else 1
        sol = ncomp * (elt * (3 * r.n * rc + rc ** 3) + 8192)
        ctx = int(L.load().tpcg_ctx_bytes(r.n, max_cols, rc, r.dtype))
        if r.problem == "elasticity":   # 21 solver tensors instead of the 10 counted by tpcg_ctx_bytes
            ctx += 11 * (elt * (3 * r.n * max_cols + rc ** 3) + 8192)
        return ctx + sol

    # ------------------------------------------------------------------ serving loop
    def _solve(self, r: Request, pb, t0: float, admitted: float, need: int, out: list, idx: int,
               setup_s: float = 0.0, hit: bool = True):
        try:
            self._solve_in_slot(r, pb, t0, admitted, out, idx, setup_s, hit)
        except Exception as e:   # a failed request reports status -2 and its error; the others carry on
            now = time.perf_counter() - t0
            out[idx] = Result(r, -2, 0, 0, float("inf"), (0, 0, 0), admitted, now, None, None, setup_s, hit, str(e))
        finally:
            with self._cv:
                self._used -= need
                self._running -= 1
                self._cv.notify_all()

    def _solve_in_slot(self, r: Request, pb, t0: float, admitted: float, out: list, idx: int, setup_s: float,
                       hit: bool):
        rc, max_cols = self._shape(r, pb)
        ctx = api.Ctx(r.n, max_cols, rc, r.dtype)
        # the context's own stream: torch's pool recycles 32 streams, and two solves on one stream would
        # interleave with each other's graph captures
        stream = api.ctx_stream(ctx)
        with torch.cuda.stream(stream):
            core = fac = None
            if r.problem == "elasticity":
                x = [api.Tucker(r.n, cap=rc, core_cap=rc ** 3, dtype=r.dtype) for _ in range(3)]
                st = api.elast_solve(pb, ctx, x, stream=stream, tol=r.tol, rank_cap=rc)
                if self.keep:
                    parts = [xi.to_numpy() for xi in x]
                    core, fac = [c for c, _ in parts], [f for _, f in parts]
            else:
                x = api.Tucker(r.n, cap=rc, core_cap=rc ** 3, dtype=r.dtype)
                st = api.tpcg_solve(pb, ctx, x, stream=stream, tol=r.tol, rank_cap=rc)
                if self.keep:
                    core, fac = x.to_numpy()
            stream.synchronize()
        out[idx] = Result(r, int(st.status), int(st.iters), int(st.outer_iters), float(st.true_rel_res),
                          tuple(st.rank), admitted, time.perf_counter() - t0, core, fac, setup_s, hit)
        del ctx, x

    def prepare(self, requests, workers: int = 8):
        """Build the operators of `requests` on `workers` host threads (the host setup of App. A and B is
        independent per problem); later calls of problem() find them in the cache."""
        from concurrent.futures import ThreadPoolExecutor
        todo = {}
        with self._plock:
            for r in requests:
                if self._key(r) not in self._problems:
                    todo.setdefault(self._key(r), r)
        with ThreadPoolExecutor(max_workers=max(1, workers)) as ex:
            built = list(ex.map(self._build, todo.values()))
        with self._plock:
            for key, pb in zip(todo.keys(), built):
                self._problems.setdefault(key, pb)

    def _admit(self, need: int):
        with self._cv:
            while self._running >= self.max_slots or self._used + need > self.budget:
                self._cv.wait()
            self._used += need
            self._running += 1

    def _arrive(self, r: Request, t0: float, out: list, idx: int, hit: bool):
        """One request with its operator setup in its latency: build (or wait for) the operator, then admission
        by memory and slot, then the solve."""
        ts = time.perf_counter()
        setup_s = 0.0
        try:
            pb = self.problem(r)
            setup_s = time.perf_counter() - ts
            need = self.footprint(r, pb)
            if need > self.budget:
                raise ValueError(f"request {idx} needs {need} bytes, more than the whole budget {self.budget}")
        except Exception:   # a request that cannot be set up or never fits fails alone (status -1)
            now = time.perf_counter() - t0
            out[idx] = Result(r, -1, 0, 0, float("inf"), (0, 0, 0), now, now, None, None, setup_s, hit,
                              "set-up failed or the request never fits the memory budget")
            return
        self._admit(need)
        self._solve(r, pb, t0, time.perf_counter() - t0, need, out, idx, setup_s, hit)

    def run(self, requests):
        """Serve `requests` (sorted by arrival time) and return their results in the same order."""
        requests = sorted(requests, key=lambda q: q.arrival)
        if self.setup_in_latency:
            out = [None] * len(requests)
            threads = []
            t0 = time.perf_counter()
            for i, r in enumerate(requests):
                wait = r.arrival - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
                th = threading.Thread(target=self._arrive, args=(r, t0, out, i, self.cached(r)))
                th.start()
                threads.append(th)
            for th in threads:
                th.join()
            return out
        # operators are built before the clock starts (a cache warm-up, not part of a request)
        needs = [self.footprint(r, self.problem(r)) for r in requests]
        for i, need in enumerate(needs):
            if need > self.budget:
                raise ValueError(f"request {i} needs {need} bytes, more than the whole budget {self.budget}")
        out = [None] * len(requests)
        threads = []
        t0 = time.perf_counter()
        for i, r in enumerate(requests):
            wait = r.arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            need = needs[i]
            self._admit(need)
            admitted = time.perf_counter() - t0
            th = threading.Thread(target=self._solve, args=(r, self.problem(r), t0, admitted, need, out, i))
            th.start()
            threads.append(th)
        for th in threads:
            th.join()
        return out


def percentiles(results, qs=(50, 99)):
    import numpy as np
    lat = np.array([r.latency for r in results])
    return {f"p{q}": float(np.percentile(lat, q)) for q in qs}
