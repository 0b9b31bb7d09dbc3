#!/usr/bin/env python
"""TPCG benchmark on GB300: solves/sec to relative residual 1e-6 (plus p50/p99 latency) for the
single deformed-geometry Poisson workload (twisted quarter annulus, p = 3, n = 128 dofs per direction).

One step = ``--concurrent`` (default 32) complete TPCG solves (Alg. 5 with Alg. 1, 2, 4; every hot-path
kernel) of resident problems of the same family (one seed each), run at once; the single-solve latency is
measured separately.  ``python bench.py --gpus N --steps K --warmup W`` prints one JSON line on rank 0.
``--impl reference`` times the FP64 CPU oracle on the host cores instead (a bounded sample).
Multi-GPU: independent replicas (one solve stream per GPU, no collective), weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
# concurrent solves run on separate streams: give the device as many hardware work queues as it has
# (the default of 8 makes streams beyond the eighth share queues and wait on each other's kernels); this must
# be set before the CUDA context exists
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

N_DOF, DEGREE, SEED = 128, 3, 7
AMP = synth.amp_from_seed(SEED)
TOL = 1e-6
WORKLOAD = f"twisted quarter annulus Poisson, p={DEGREE}, n={N_DOF}/direction, amp={AMP:.4f} (seed {SEED})"
METRIC = "TPCG solves/sec to rel-residual 1e-6"
# iterations of the FP64 Alg. 5 on this workload (the FP64 GPU form takes 30 for seed 7): the CPU oracle's
# per-iteration time is scaled by this count
ORACLE_ITERS = 30


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--dtype", default="mixed", choices=["mixed", "f64", "f32"])
    ap.add_argument("--concurrent", type=int, default=32, help="solves per step, run at once")
    ap.add_argument("--rank-cap", type=int, default=96)
    ap.add_argument("--inner-tol", type=float, default=2e-2, help="mixed form: inner FP32 solve tolerance")
    ap.add_argument("--refine-keep", type=float, default=3e-2, help="mixed form: accuracy kept of each correction")
    ap.add_argument("--gemm-ctas-per-sm", type=int, default=2, help="grouped-GEMM CTA budget per SM (0: uncapped)")
    ap.add_argument("--torch-streams", action="store_true", help="give each solve a torch stream (<= 32)")
    ap.add_argument("--serve", type=float, default=0.0,
                    help="instead of the batch benchmark: serve a Poisson-arrival stream at this rate (requests/s)")
    ap.add_argument("--requests", type=int, default=48, help="requests in the --serve stream")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------- CPU oracle
def oracle_sample(iters_for_scale: int, n=N_DOF, p=DEGREE, sample_iters=20):
    """Time `sample_iters` iterations of the oracle's Alg. 5 on the same workload (setup excluded) and
    scale to solves/sec with the iteration count of a full solve."""
    from oracle import expsum, fd, lowrank, tpcg as otp
    terms = lowrank.operator_terms("twist", AMP, n, p)
    f = lowrank.rhs_tucker("twist", AMP, n, p)
    # the preconditioner with the best exponential sums for this M_P, as the library's setup builds it
    _, om, al, _, _ = expsum.rp_best(fd.mp_value(n, p), 0.1)
    P = fd.ApproxFD(n, p, expsum=(om, al))
    t0 = time.perf_counter()
    _, info = otp.tpcg(terms, f, P.apply, otp.Params(tol=TOL, max_it=sample_iters))
    dt = time.perf_counter() - t0
    per_iter = dt / max(info["iters"], 1)
    iters = max(iters_for_scale, 1)
    return {"value": 1.0 / (per_iter * iters), "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{info['iters']} TPCG iterations of the {n}^3 p={p} twisted-annulus solve in {dt:.1f}s "
                      f"(setup excluded), scaled to a {iters}-iteration solve"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    K = max(args.steps, 1)
    vals = []
    for _ in range(K):
        vals.append(oracle_sample(ORACLE_ITERS, sample_iters=2)["value"])
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": K, "warmup": args.warmup, "ms_per_step": 1000.0 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "tol": TOL},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"2 TPCG iterations per step, scaled to a {ORACLE_ITERS}-iteration solve"},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------- replicas
def max_over_ranks(x: float, device: str) -> float:
    """The slowest rank's time: replicas finish when the last one does."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, solves_per_step: int, steps: int, total_ms: float) -> float:
    """Whole-job solves/s: every rank solved `solves_per_step` problems per step (weak scaling)."""
    return world * solves_per_step * steps / (total_ms * 1e-3)


def rank_seeds(rank: int, solves_per_step: int):
    """Seeds of the problems one rank solves: replicas take disjoint seed ranges."""
    return [SEED + rank * solves_per_step + i for i in range(solves_per_step)]


# ------------------------------------------------------------------------------------------- GPU arm
def _profile(L, lib):
    import ctypes as C
    prof = {}
    for name, kind in lib.PROF_KINDS.items():
        ms, cnt, fl, by = C.c_double(), C.c_longlong(), C.c_double(), C.c_double()
        L.tpcg_profile_get(kind, C.byref(ms), C.byref(cnt), C.byref(fl), C.byref(by))
        prof[name] = {"ms": ms.value, "launches": cnt.value, "flops": fl.value, "bytes": by.value}
    return prof


def _roofline(prof, dt_name, lib, step_ms_total):
    """Roofline of the dominant kernel class: algorithmic work per launch / measured launch time."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    bf16 = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0))
    src = "of measured" if peaks else "of fallback"
    # FP32/FP64 SIMT peaks derived from the measured sustained bf16 rate and the nominal ratios
    # (bf16 2250, FP32 75, FP64 1.25 TFLOP/s dense nominal)
    alu = {"f64": bf16 * 1.25 / 2250.0, "f32": bf16 * 75.0 / 2250.0}
    classes = ["zgemm", "zblk", "gram", "eig", "proj", "qr", "apply", "fd"]
    # DRAM bytes per launch of the FP32 eigensolver from one ncu capture of this workload (dram__bytes_read.sum +
    # dram__bytes_write.sum, mean of 3 launches); other kernels: no capture, traffic null
    ncu_traffic = {"eig": 105216.0} if dt_name == "mixed" else {}
    dom = max(classes, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    per_launch_ms = d["ms"] / max(d["launches"], 1)
    roof = {"kernel": dom, "share_of_step": d["ms"] / max(step_ms_total, 1e-9), "launches": d["launches"],
            "ms_per_launch": per_launch_ms}
    if dom in ("apply", "fd"):
        ach = d["bytes"] / (d["ms"] * 1e-3) / 1e9 if d["ms"] > 0 else 0.0
        roof.update({"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                     "traffic": None, "peak_source": f"hbm_gbs {src}"})
    else:
        # the eigensolver's algorithmic work is the dense symmetric eigen-decomposition count 9 n'^3 per Gram
        # (the mixed form's eigensolver launches are FP32 apart from the FP64 truncations of x)
        prec = "f32" if (dom == "eig" and dt_name == "mixed") or dt_name == "f32" else "f64"
        pk = alu[prec]
        ach = d["flops"] / (d["ms"] * 1e-3) / 1e12 if d["ms"] > 0 else 0.0
        roof.update({"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                     "traffic": ncu_traffic.get(dom),
                     "peak_source": f"{prec.upper()} SIMT peak = bf16_tflops_sustained {src} x nominal "
                                    f"{'75' if prec == 'f32' else '1.25'}/2250"})
    return roof


def _make_problem(api, lib, dt, seed):
    return api.tpcg_setup(lib.GEOM_TWIST, synth.amp_from_seed(seed), DEGREE, N_DOF, dt)


def _ctx_for(api, info, dt, rc):
    return api.Ctx(N_DOF, api.max_cols_for(info, rc, dt), rc, dt)


def run_gpu(args):
    import torch
    from paper_2306_00632_gb300 import api, lib

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    L = lib.load()
    dt = {"f64": lib.F64, "f32": lib.F32, "mixed": lib.MIXED}[args.dtype]
    B = max(args.concurrent, 1)
    rc = min(args.rank_cap, N_DOF)
    # B problems of the same family (seeds SEED .. SEED+B-1), one context, solution and stream each
    seeds = rank_seeds(rank, B)
    pbs = [_make_problem(api, lib, dt, sd) for sd in seeds]
    ctxs = [_ctx_for(api, p.info, dt, rc) for p in pbs]
    xs = [api.Tucker(N_DOF, cap=rc, core_cap=rc ** 3, dtype=dt) for _ in range(B)]
    # by default the library gives each solve a stream of its own (torch's pool holds 32 streams per priority)
    if args.torch_streams and B > 32:
        raise SystemExit("--torch-streams: torch's pool has 32 streams per priority; concurrent solves need their own")
    streams = [torch.cuda.Stream() for _ in range(B)] if args.torch_streams else [None] * B
    lib.check(L.tpcg_set_option(1, args.gemm_ctas_per_sm), "tpcg_set_option")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 256 MB > L2
    main = torch.cuda.current_stream()

    kw = dict(tol=TOL, rank_cap=rc, inner_tol=args.inner_tol, refine_keep=args.refine_keep)

    # (1) single-solve latency and the per-kernel profile (problem 0 on the main stream)
    for _ in range(max(args.warmup, 0)):
        api.tpcg_solve(pbs[0], ctxs[0], xs[0], **kw)
    torch.cuda.synchronize()
    L.tpcg_profile_reset()
    L.tpcg_profile_enable(1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    single = []
    torch.cuda.profiler.start()   # an external profiler started with --profile-from-start off sees this region
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(main)
        st = api.tpcg_solve(pbs[0], ctxs[0], xs[0], **kw)
        ev[k][1].record(main)
        single.append(st)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    L.tpcg_profile_enable(0)
    lat_ms = [a.elapsed_time(b) for a, b in ev]
    prof = _profile(L, lib)

    # (2) throughput: K steps of B concurrent solves (tpcg_solve_batch), timed on the device
    def batch():
        return api.tpcg_solve_batch(pbs, ctxs, xs, streams, **kw)

    for _ in range(max(args.warmup, 0)):
        batch()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = L.tpcg_launch_count()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    results = []
    torch.cuda.synchronize()
    g0.record(main)
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()   # the flush completes before the solve streams start
        codes, sts = batch()
        results.append((codes, sts))
    g1.record(main)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    launches = L.tpcg_launch_count() - launches0
    clk = clocks.stop()
    total_ms = g0.elapsed_time(g1)
    if ws > 1:
        total_ms = max_over_ranks(total_ms, "cuda")

    roof = _roofline(prof, args.dtype, lib, sum(lat_ms))
    value = job_throughput(ws, B, args.steps, total_ms)
    last = results[-1][1]
    out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
           "config": {"workload": WORKLOAD, "solves_per_step": B, "inner_tol": args.inner_tol,
                      "gemm_ctas_per_sm": args.gemm_ctas_per_sm,
                      "refine_keep": args.refine_keep,
                      "seeds": f"{seeds[0]}..{seeds[-1]} on rank 0, disjoint ranges per rank (amp from seed)",
                      "tol": TOL, "rank_cap": rc,
                      "R": [p.info.R for p in pbs], "RP": pbs[0].info.RP, "parallelism": f"replicas x{ws}",
                      "l2": "256 MB buffer written between timed steps"},
           "latency_ms": {"p50": float(np.percentile(lat_ms, 50)), "p99": float(np.percentile(lat_ms, 99)),
                          "what": "single solve alone on the device (CUDA events)"},
           "solve": {"status": [int(c) for c in results[-1][0]],
                     "true_rel_res": [float(s.true_rel_res) for s in last],
                     "inner_iters": [int(s.iters) for s in last], "outer_iters": [int(s.outer_iters) for s in last],
                     "rank": [list(s.rank) for s in last]},
           "single": {"iters": [int(s.iters) for s in single], "true_rel_res": [float(s.true_rel_res) for s in single]},
           "gpu_launches": int(launches), "roofline": roof,
           "kernel_ms_single": {k: round(v["ms"], 3) for k, v in prof.items()},
           "clocks": clk}

    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e(api, lib, pbs, dt, ctxs, xs, streams, kw, args)
    if rank == 0 and not args.no_cpu and ws == 1:
        try:
            out["cpu_baseline"] = oracle_sample(ORACLE_ITERS)
        except Exception as e:   # the baseline must not hide the GPU line
            out["cpu_baseline"] = {"value": None, "error": str(e)[:200]}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def e2e(api, lib, pbs, dt, ctxs, xs, streams, kw, args):
    """Same metric through the public API with host inputs: every step re-creates the B problems from pinned
    host arrays (host -> device copies inside tpcg_problem_create), solves them at once and reads the
    solutions back to the host."""
    import torch
    exs = []
    for pb in pbs:
        ex = pb.export()
        ex["v2u2"] = ex["v2u2"][: pb.info.n * pb.info.n2]
        exs.append((ex, pb.info))
    h2d = 0
    for ex, _ in exs:
        h2d += 8 * sum(int(np.asarray(ex[k]).size) for k in ("w", "bands", "f_core", "f_U0", "f_U1", "f_U2", "lam",
                                                            "mu", "w_val", "v2u2", "omega", "alpha"))
        h2d += 4 * (int(ex["w_rowptr"].size) + int(ex["w_col"].size))
    K = max(2, min(args.steps, 3))
    times = []
    d2h = 0
    for k in range(K + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pb2 = [api.problem_from_export(ex, info, dtype=dt, pinned=True) for ex, info in exs]
        api.tpcg_solve_batch(pb2, ctxs, xs, streams, **kw)
        d2h = 0
        for x in xs:
            core, fac = x.to_numpy()
            d2h += (core.size + sum(f.size for f in fac)) * (4 if dt == lib.F32 else 8)
        torch.cuda.synchronize()
        if k > 0:
            times.append(time.perf_counter() - t0)
        del pb2
    return {"value": len(pbs) / statistics.median(times), "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": K}


def run_serve(args):
    """Continuous-batching server under a Poisson-arrival stream: half scalar Poisson requests (mixed form,
    n in {32, 64, 96, 128}, p in {2, 3}), half elasticity requests (FP64, n in {16, 24, 32}, lambda = 1,
    mu in [0.3, 1], body force (0, 0.1, -1)), seeded.  Prints p50/p99 latency and throughput."""
    import torch
    from paper_2306_00632_gb300 import lib, serve
    lib.load()
    arr = synth.poisson_arrivals(args.serve, args.requests, seed=SEED)
    reqs = []
    for i, t in enumerate(arr):
        sd = SEED + 1000 + i
        if i % 2 == 0:
            n = (32, 64, 96, 128)[int(synth.unit_from_seed(sd, 2) * 4)]
            p = 2 + int(synth.unit_from_seed(sd, 3) * 2)
            reqs.append(serve.Request(lib.GEOM_TWIST, synth.amp_from_seed(sd), p, n, min(n, 96), tol=TOL,
                                      dtype=lib.MIXED, arrival=float(t)))
        else:
            n = (16, 24, 32)[int(synth.unit_from_seed(sd, 2) * 3)]
            mu = 0.3 + 0.7 * synth.unit_from_seed(sd, 5)
            reqs.append(serve.Request(lib.GEOM_TWIST, synth.amp_from_seed(sd), 2, n, n, tol=TOL, dtype=lib.F64,
                                      arrival=float(t), problem="elasticity", lame_lambda=1.0, lame_mu=mu,
                                      force=(0.0, 0.1, -1.0)))
    free, _ = torch.cuda.mem_get_info()
    srv = serve.Server(int(free * 0.6), max_slots=32)
    srv.run(reqs[:4])   # warm-up: operators cached, contexts and graphs exercised
    t0 = time.perf_counter()
    res = srv.run(reqs)
    wall = time.perf_counter() - t0
    lat = serve.percentiles(res)
    ok = sum(1 for r in res if r.status == 0 and r.true_rel_res <= TOL)
    line = {"metric": "served TPCG requests: p50/p99 latency and solves/s", "unit": "s",
            "rate_hz": args.serve, "requests": len(res), "converged": ok,
            "latency_s": {"p50": lat["p50"], "p99": lat["p99"]},
            "solves_per_s": len(res) / max(max(r.finished for r in res), 1e-9), "wall_s": wall,
            "mix": "50/50 Poisson (mixed form, n 32-128) / elasticity (FP64, n 16-32), seeded twisted annuli",
            "max_slots": 32}
    by = {}
    for r in res:
        k = r.request.problem
        d = by.setdefault(k, {"requests": 0, "status": {}, "iters": [], "latency_s": [], "n": []})
        d["requests"] += 1
        d["status"][str(r.status)] = d["status"].get(str(r.status), 0) + 1
        d["iters"].append(r.iters)
        d["latency_s"].append(round(r.latency, 2))
        d["n"].append(r.request.n)
    line["by_problem"] = by
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.serve > 0:
        run_serve(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
