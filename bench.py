#!/usr/bin/env python3
"""KKT solves/s and p50/p99 latency of the Schur-complement solve of a
multiperiod storage OPF system on GB300, mixed precision against FP64.

Default workload (the precision configuration): the synthetic 9,241-bus grid
(16,049 lines, 1,445 generators, 400 storage units) over 168 periods; blocks
A_i of order 41,054, coupling S of order 67,200 (input recipe in
gen/mpopf.py).  One step = one KKT solve: the numeric factorization (block
factors, Schur assembly, dense factor of S) plus the solve with FP64
iterative refinement to eta <= 1e-10.  The timed path factors S in TF32 on the
tensor cores (256-wide outer panels) and the top of every block's elimination
tree in emulated FP64 on the tensor cores; the legs beside it are the
FP64-accurate variants and BF16, each with its accuracy.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   # the CPU oracle, timed on the host

Multi-GPU (torchrun, one rank per GPU): independent replicas, one system per
rank, no data-path collective; value = solves of all ranks / max rank time.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "KKT solves/s & p50/p99 latency, mixed-prec vs plain FP64 GPU at resid≤1e-10"
WORKLOAD = "grid9241_n168"
L2_FLUSH_BYTES = 256 << 20
TIGHT_TOL = 1e-12  # the FP64 paths' level on the 9,241-bus system (eta ~ 5e-13 after one step)
# TF32 runs at about half the BF16 tensor rate (nominal 1.1 against 2.25 PFLOP/s dense)
TF32_RATIO = 1.1 / 2.25
# the emulated-FP64 update issues 28 BF16 digit products per FP64 multiply-add
EMU_PRODUCTS = 28.0
# DRAM bytes per launch of the dominant kernel, from an ncu capture of the same
# kernel code (profiles/); None where no capture of the current kernel exists.
# k_tc_update_emu_wide on the 9,241-bus grid: all 56 launches of one factor of
# the 8-period system read 25.99 GB and wrote 14.85 GB; every launch updates the
# same tail in each of its blocks (each tail, 439 MB, exceeds L2), so a launch
# over 168 blocks moves 168 / 8 times as much: 40.84 GB * 21 / 56 per launch.
TRAFFIC = {("grid9241_n168", "k_tc_update_emu_wide"): 40.395244032e9 * 21 / 56}


def workload_desc(name):
    """The config.workload string: the named instance and its sizes."""
    from gen import describe_workload

    return describe_workload(name)


def workload_defaults(name):
    """Tail ratio and autotuning per workload: the 9,241-bus grids take the
    ratio the autotuner chose there (r = 1.25; each candidate costs seconds),
    the others autotune."""
    if name.startswith("grid9241"):
        return {"tail_ratio": 1.25, "autotune": 0}
    return {"tail_ratio": 0.0, "autotune": 1}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [ln.strip().split(",") for ln in self.tmp.read().splitlines() if ln.strip()]
        self.tmp.close()
        os.unlink(self.tmp.name)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [c.strip() for c in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                power.append(float(r[3]))
            except ValueError:
                continue
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count()


# ---------------------------------------------------------------- CPU baseline

def block_flops_host(prob):
    """Flops of one block factor, sum_j c_j (c_j + 3) over the column counts of
    the ordering kkt_analyze chooses (the host-only symbolic library; no GPU).
    It sizes the work of a system for scaling a sampled oracle time."""
    import numpy as np

    from paper_1907_05420_gb300 import build as lib_build

    L = ctypes.CDLL(lib_build.build_symbolic())
    L.kkt_symbolic_create.restype = ctypes.c_void_p
    L.kkt_symbolic_get.restype = ctypes.c_int64
    L.kkt_symbolic_get.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_void_p]
    L.kkt_symbolic_destroy.argtypes = [ctypes.c_void_p]
    rp = np.ascontiguousarray(prob.a_rowptr, dtype=np.int32)
    col = np.ascontiguousarray(prob.a_col, dtype=np.int32)
    hint = np.ascontiguousarray(np.asarray(prob.a_vals).reshape(prob.N, -1)[0], dtype=np.float64)
    zero = np.zeros(2, dtype=np.int32)
    p = ctypes.c_void_p
    h = L.kkt_symbolic_create(ctypes.c_int32(prob.nA), ctypes.c_int32(prob.nP), p(rp.ctypes.data),
                              p(col.ctypes.data), p(hint.ctypes.data), ctypes.c_int32(1), ctypes.c_int32(0),
                              p(zero.ctypes.data), p(zero.ctypes.data), p(zero.ctypes.data), ctypes.c_int32(0))
    if not h:
        raise RuntimeError("symbolic analysis failed")
    try:
        n = L.kkt_symbolic_get(h, b"colcount", None)
        cc = np.zeros(n, dtype=np.int64)
        L.kkt_symbolic_get(h, b"colcount", p(cc.ctypes.data))
    finally:
        L.kkt_symbolic_destroy(h)
    cc = cc.astype(np.float64)
    return float(np.sum(cc * (cc + 3.0)))


def _est(N, nC, block_flops):
    """Estimated oracle work of a system: its block factors and the dense factor of S."""
    return N * block_flops + nC ** 3 / 3.0


# oracle work per sample, in estimated flops (the oracle runs the 2,383-bus,
# 96-period solve, about 3e11 flops, in about 14 s on 16 Grace cores)
CPU_SAMPLE_FLOPS = 6e11
# the largest grid whose blocks the oracle's plain minimum-degree ordering
# handles within seconds (the 9,241-bus blocks do not finish in minutes)
ORACLE_MAX_BUS = 3000


def cpu_sample_plan(workload, prob, block_flops, budget=None):
    """(sample problem, its description, scale to the full workload) for a
    bounded oracle run.  The full workload if its estimated work fits the
    budget; else its first N' periods; else, for grids beyond the oracle's
    ordering, the same generator recipe on the 2,383-bus grid over N' periods,
    scaled by the estimated work of the two systems."""
    import dataclasses

    from gen import CONFIGS, make_problem
    from gen.workloads import workload_spec

    budget = CPU_SAMPLE_FLOPS if budget is None else budget
    ns = prob.nC // prob.N if prob.N else 0
    full = _est(prob.N, prob.nC, block_flops)
    if full <= budget:
        return prob, f"1 full solve of {workload}", 1.0
    kind, spec, _ = workload_spec(workload)
    if kind == "mpopf" and spec.n_bus <= ORACLE_MAX_BUS:
        fit = [k for k in range(1, prob.N + 1) if _est(k, k * ns, block_flops) <= budget]
        n = fit[-1] if fit else 1
        sub = make_problem(dataclasses.replace(spec, n_per=n, name=f"{workload}_first{n}"))
        scale = full / _est(n, n * ns, block_flops)
        return sub, f"1 solve of {workload} over its first {n} of {prob.N} periods", scale
    base = CONFIGS["grid2383_n96"]
    one = make_problem(dataclasses.replace(base, n_per=1, name="grid2383_n1"))
    bf = block_flops_host(one)
    fit = [k for k in range(1, base.n_per + 1) if _est(k, k * base.n_stor, bf) <= budget]
    n = fit[-1] if fit else 1
    sub = make_problem(dataclasses.replace(base, n_per=n, name=f"grid2383_n{n}"))
    scale = full / _est(n, n * base.n_stor, bf)
    return sub, (f"1 solve of the same recipe on the 2,383-bus grid over {n} periods (the oracle's "
                 f"minimum-degree ordering of one {workload} block does not finish in minutes)"), scale


def cpu_reference_solve(prob, perm=None):
    """One oracle solve on the host cores; the ordering is analysis (once per
    pattern, like kkt_analyze) and is computed outside the timed region."""
    import oracle

    if perm is None:
        perm = oracle.min_degree(prob.nA, prob.a_rowptr, prob.a_col, prob.nP)
    t0 = time.perf_counter()
    out = oracle.kkt_solve(prob, perm)
    return out, time.perf_counter() - t0


def cpu_baseline_sample(workload, prob, block_flops, budget=None):
    """The oracle timed on a bounded sample of the workload: (line fields,
    oracle output of the full system or None)."""
    import oracle

    sub, desc, scale = cpu_sample_plan(workload, prob, block_flops, budget)
    out, dt = cpu_reference_solve(sub)
    fields = {"unit": "solves/s", "cores": oracle.max_threads(), "host_cores": host_cores(), "kind": "oracle",
              "value": 1.0 / (dt * scale)}
    if scale == 1.0:
        fields["sample"] = f"{desc} (FP64 oracle, OpenMP; ordering computed once, untimed; {dt:.1f} s)"
        return fields, out
    fields["sample"] = (f"{desc} (FP64 oracle, OpenMP; ordering untimed; {dt:.1f} s), scaled to the full "
                        f"system by the estimated work N*block_flops + nC^3/3 (x{scale:.1f})")
    return fields, None


def run_reference(args):
    """--impl reference: the CPU oracle, timed as it stands on the host cores,
    one bounded sample of the workload per step, rate scaled to the workload."""
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from gen import CONFIGS, build_workload, make_problem

    prob = build_workload(args.workload)
    bf = block_flops_host(prob)
    sub, desc, scale = cpu_sample_plan(args.workload, prob, bf, args.ref_sample_flops)
    small = make_problem(CONFIGS["grid30_n24"])
    for _ in range(args.warmup):  # warm-up on the small instance (loads the library, threads)
        oracle.kkt_solve(small)
    perm = oracle.min_degree(sub.nA, sub.a_rowptr, sub.a_col, sub.nP)  # analysis, untimed
    times = []
    for _ in range(args.steps):
        _, dt = cpu_reference_solve(sub, perm)
        times.append(dt * scale)
    total = sum(times)
    value = args.steps / total
    threads = oracle.max_threads()
    sample = (f"{args.steps} x {desc}" + (f", each scaled by the estimated work (x{scale:.1f})" if scale != 1.0
                                          else "") + f"; ordering computed once untimed (warm-up: {args.warmup} "
              "solves of grid30_n24)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(args.workload), "precision": "fp64", "parallelism": "none (host)"},
        "latency_ms": {"p50": 1e3 * statistics.median(times),
                       "p99": 1e3 * max(times) if len(times) < 100 else
                       1e3 * sorted(times)[int(0.99 * len(times))]},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ batching, serving

def _mix_problems(count, prec):
    import numpy as np
    import torch

    from gen import make_problem, mix_spec
    from paper_1907_05420_gb300 import binding as B

    probs = [make_problem(mix_spec(k)) for k in range(count)]
    dev = torch.device("cuda:0")
    hs = [B.kkt_analyze(p, B.kkt_default_options(prec)) for p in probs]
    up = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(dev)  # noqa: E731
    vals = [(up(p.a_vals), up(p.b_vals), up(p.c_vals), up(p.rhs)) for p in probs]
    xs = [torch.empty_like(v[3]) for v in vals]
    return probs, hs, vals, xs


def run_batch(args):
    """The 64-instance size mix: one batched call against 64 sequential solves."""
    import torch

    import oracle
    from paper_1907_05420_gb300 import binding as B

    count = 64
    out = {"metric": "KKT solves/s, 64-instance size mix, batched vs sequential", "unit": "solves/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
           "data": "synthetic", "config": {"workload": "mix64: 64 seeded grids, 118-3000 buses, "
                                                       "N in {12,24,48,96}, 5-10% storage buses"}}
    for prec in args.batch_precs.split(","):
        probs, hs, vals, xs = _mix_problems(count, prec)
        A = [v[0] for v in vals]
        Bv = [v[1] for v in vals]
        Cv = [v[2] for v in vals]
        R = [v[3] for v in vals]
        for _ in range(args.warmup):
            B.kkt_batch_factor_solve(hs, A, Bv, Cv, R, xs, streams=args.batch_streams)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            B.kkt_batch_factor_solve(hs, A, Bv, Cv, R, xs, streams=args.batch_streams)
        torch.cuda.synchronize()
        t_batch = (time.perf_counter() - t0) / args.steps
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for h, (a, b, c, r), x in zip(hs, vals, xs):
                B.kkt_factor(h, a, b, c)
                B.kkt_solve(h, r, x, allow_not_converged=True)
        torch.cuda.synchronize()
        t_seq = (time.perf_counter() - t0) / args.steps
        etas = [oracle.backward_error(p, x.cpu().numpy()) for p, x in zip(probs, xs)]
        out[prec] = {"batched": count / t_batch, "sequential": count / t_seq,
                     "ms_per_batch": 1e3 * t_batch, "ms_sequential": 1e3 * t_seq,
                     "eta_max": max(etas), "streams": args.batch_streams}
        for h in hs:
            B.kkt_destroy(h)
    out["value"] = out[args.batch_precs.split(",")[0]]["batched"]
    print(json.dumps(out), flush=True)
    return 0


def serve_sweep(args, precs, rates, seconds, pool=64):
    """A Poisson stream of KKT solve requests over the 64-instance size mix
    (configs[3]'s recipe) through the server's pattern cache: each request
    names a mix pattern; with probability resolve_frac it re-solves a pattern
    already seen with fresh barrier diagonals and right-hand side, else it
    solves the instance as drawn.  A pattern is analysed at its first request
    (inside that request's latency) and stays resident; admission of a new
    pattern is by free device memory.  Latency: submit to completion of the
    refined solve; requests arriving while `backlog` are outstanding are shed.
    Returns per precision and rate: offered, served, shed, solves/s, p50/p99."""
    import numpy as np
    import torch

    from gen import make_problem, mix_spec, reseed_barrier
    from paper_1907_05420_gb300 import binding as B

    dev = torch.device("cuda:0")
    up = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(dev)  # noqa: E731
    probs = [make_problem(mix_spec(k)) for k in range(pool)]
    fresh = [reseed_barrier(p, 4242 + k) for k, p in enumerate(probs)]
    vals = [[(up(q.a_vals), up(q.b_vals), up(q.c_vals), up(q.rhs)) for q in (p, f)] for p, f in zip(probs, fresh)]
    pats = [B.make_pattern(p) for p in probs]
    backlog = args.serve_backlog or 4 * args.serve_slots
    out = {"workload": f"{pool}-instance size mix (118-3,000 buses, N in {{12,24,48,96}}); Poisson arrivals; "
                       f"{int(100 * args.resolve_frac)}% re-solves of a seen pattern with fresh barrier diagonals; "
                       "patterns analysed at first request, resident after, admitted by free HBM",
           "slots": args.serve_slots, "seconds_per_rate": seconds, "backlog": backlog,
           "refinement": ["iterative", "gmres"][args.refine_mode]}
    for mode in precs:
        prec, opts, tol = parse_leg(mode)
        if tol is not None:
            opts["refine_tol"] = tol
        srv = B.KKTServer(slots=args.serve_slots)
        srv.set_cache(B.kkt_default_options(prec, refine_mode=args.refine_mode, **opts), reserve_bytes=8 << 30)
        rng = np.random.default_rng(4242)
        seen = set()
        res = {}
        for rate in rates:
            lats, outstanding = [], {}
            shed = offered = 0
            t0 = time.perf_counter()
            t_measure, t_end = t0 + 0.5, t0 + 0.5 + seconds
            t_next = t0

            def reap(block):
                for rid in list(outstanding):
                    got = srv.wait(rid) if block else srv.poll(rid)
                    if got is None:
                        continue
                    st, lat = got
                    if outstanding.pop(rid) and st in (0, 6):
                        lats.append(lat)

            while time.perf_counter() < t_end:
                now = time.perf_counter()
                if now < t_next:
                    time.sleep(min(t_next - now, 0.0005))
                    continue
                t_next += rng.exponential(1.0 / rate)
                in_window = now >= t_measure
                offered += in_window
                reap(False)
                if len(outstanding) >= backlog:
                    shed += in_window
                    continue
                if seen and rng.random() < args.resolve_frac:
                    k, v = int(rng.choice(sorted(seen))), 1
                else:
                    k, v = int(rng.integers(0, pool)), 0
                seen.add(k)
                a, b, c, r = vals[k][v]
                x = torch.empty_like(r)
                outstanding[srv.submit_pattern(k, probs[k], a, b, c, r, x, pattern=pats[k])] = in_window
            reap(True)
            t_done = time.perf_counter()
            n = len(lats)
            res[str(int(rate))] = {"offered": offered, "served": n, "shed": shed,
                                   "solves_per_s": n / max(1e-9, t_done - t_measure),
                                   "p50_ms": float(np.percentile(lats, 50)) if n else None,
                                   "p99_ms": float(np.percentile(lats, 99)) if n else None}
        res["cache"] = srv.cache_info()
        srv.close()
        out[mode] = res
    return out


def run_serve(args):
    """Poisson request stream over the size mix; p50/p99 latency and solves/s per rate."""
    rates = [float(q) for q in args.rates.split(",")]
    sw = serve_sweep(args, args.batch_precs.split(","), rates, args.serve_seconds)
    first = sw[args.batch_precs.split(",")[0]]
    line = {"metric": "KKT solves/s and p50/p99 latency under a Poisson request stream", "unit": "solves/s",
            "n_gpus": 1, "higher_is_better": True, "data": "synthetic", "config": {"workload": sw["workload"]},
            "value": max(v["solves_per_s"] for k, v in first.items() if k != "cache"), "serving": sw}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- main path

def parse_leg(mode):
    """'prec[+tcg|+band][@tol]' -> (prec, options, refine_tol or None)."""
    head, _, tol = mode.partition("@")
    prec, _, extra = head.partition("+")
    opts = {"reduced_contraction": int(extra == "tcg"), "structured_s": int(extra == "band")}
    return prec, opts, (float(tol) if tol else None)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="tf32", choices=["fp64", "tf32", "bf16", "f64emu"],
                    help="arithmetic of the dense factor of S on the timed path (default: the "
                         "mixed path, TF32 tensor cores with FP64 refinement)")
    ap.add_argument("--legs", default=f"fp64+band,f64emu,tf32@{TIGHT_TOL:g},bf16",
                    help="other modes measured beside the timed path ('' for none): prec[+tcg|+band][@tol]")
    ap.add_argument("--leg-steps", type=int, default=2)
    ap.add_argument("--leg-warmup", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=5,
                    help="steps of the end-to-end leg through host buffers (at most --steps)")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-sample-flops", type=float, default=6e10,
                    help="estimated oracle work of one reference-arm step")
    ap.add_argument("--batch-precs", default="tf32,fp64")
    ap.add_argument("--serve-modes", default="tf32,tf32+band,fp64+band",
                    help="modes of the serving sweep in the default run: prec[+band][@tol] (the mix uses the "
                         "adjacent coupling, whose S is banded: +band is its envelope-limited factor)")
    ap.add_argument("--batch-streams", type=int, default=8)
    ap.add_argument("--serve-pool", type=int, default=32)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--rates", default="50,100,200,500,1000,2000")
    ap.add_argument("--resolve-frac", type=float, default=0.2)
    ap.add_argument("--serve-backlog", type=int, default=0,
                    help="requests outstanding before new arrivals are shed (default 4 x slots)")
    ap.add_argument("--refine-mode", type=int, default=1, choices=[0, 1],
                    help="FP64 refinement on K: 0 iterative refinement, 1 GMRES preconditioned by the factorization")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-slack", action="store_true", help="skip the slack-elimination measurement")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving sweep of the default run")
    ap.add_argument("--no-paper", action="store_true",
                    help="skip the structured-S leg on the paper's cumulative coupling")
    ap.add_argument("--serve-seconds-default", type=float, default=2.0,
                    help="measured seconds per rate of the serving sweep inside the default run")
    ap.add_argument("--autotune", type=int, default=-1,
                    help="dense-tail autotuning at analysis: 1 on, 0 off, -1 the workload's default")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "mix64":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    return run_single(args)


def slack_timing(args, dev, stream, torch, np, B, reps=20):
    """The slack elimination (Sec. 2) around one interior-point step on the
    2,383-bus grid over 96 periods with a flow-limit inequality row for every
    line (blocks of 13,386 rows): the in-place reduction and the recovery
    timed alone (CUDA events, `reps` launches each, HBM bytes they must move),
    and one whole step (reduce, factor, refined TF32 solve, recover)."""
    from gen import CONFIGS, make_ipm_state, make_problem

    spec = CONFIGS["grid2383_n96"]
    p = make_problem(spec, flow_limits=spec.n_line)
    st = make_ipm_state(p, 2383)
    up = lambda v: torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).to(dev)  # noqa: E731
    dst = {k: up(getattr(st, k)) for k in B.Slack.FIELDS}
    h = B.kkt_analyze(p, B.kkt_default_options("tf32", tail_ratio=1.25, early_solve=1))
    sl = B.Slack(h, p.ineq_rows)
    try:
        a_base, c_base, b = up(st.a_base), up(st.c_base), up(p.b_vals)
        a, c = a_base.clone(), c_base.clone()
        rhs = torch.empty(p.nK, dtype=torch.float64, device=dev)
        x = torch.empty_like(rhs)
        L, N, nP, nA, nC = len(p.ineq_rows), p.N, p.nP, p.nA, p.nC
        ds, dy = (torch.empty(N * L, dtype=torch.float64, device=dev) for _ in range(2))
        dz = torch.empty(N * nP + nC, dtype=torch.float64, device=dev)

        def timed(fn):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        ms_red = timed(lambda: sl.reduce(dst, a, c, a, c, rhs, stream))
        ms_rec = timed(lambda: sl.recover(dst, x, ds, dz, dy, stream))
        # bytes each must move: per row of K its diagonal (read + write), its
        # right-hand side and its state entries; per unknown recovered its inputs and output
        nx, ni, ne = N * nP + nC, N * L, N * (nA - nP) - N * L
        red_bytes = 8.0 * (nx * (2 + 1 + 4) + ni * (2 + 1 + 5) + ne * 2)
        rec_bytes = 8.0 * (nx * 5 + ni * 7)

        def step():
            a.copy_(a_base)
            sl.reduce(dst, a, c, a, c, rhs, stream)
            B.kkt_factor(h, a, b, c, stream)
            B.kkt_solve(h, rhs, x, 1, stream, allow_not_converged=True)
            sl.recover(dst, x, ds, dz, dy, stream)

        ms_step = timed(step) if reps else None
        info = B.kkt_get_info(h)
        peaks, _ = _peaks()
        return {"workload": f"grid2383_n96 with {spec.n_line:,} flow-limit rows per period (nA={nA:,})",
                "reduce_ms": ms_red, "reduce_gbs": red_bytes / ms_red / 1e6,
                "reduce_hbm_frac": red_bytes / ms_red / 1e6 / peaks["hbm_gbs"],
                "recover_ms": ms_rec, "recover_gbs": rec_bytes / ms_rec / 1e6,
                "recover_hbm_frac": rec_bytes / ms_rec / 1e6 / peaks["hbm_gbs"],
                "ipm_step_ms": ms_step, "ipm_steps_per_s": 1e3 / ms_step if ms_step else None,
                "eta": info["rel_residual"], "refine_steps": info["refine_steps"]}
    finally:
        sl.close()
        B.kkt_destroy(h)


def structured_paper_timing(args, dev, stream, torch, np, B, steps=5, warmup=2):
    """The paper's own MPOPF coupling on the 2,383-bus grid over 96 periods
    (n_C = 9,600: 100 storage multipliers per period, Sec. 4.1 eq. B12N) with
    the structured S of Sec. 4.3 (structured_s = 2): factor + refined solve per
    step, device-resident inputs, FP64 and TF32 block tails.  The dense-S
    analysis of this pattern would need one gather record per pair of B
    entries of a block (reported), far beyond host memory."""
    from gen import CONFIGS, make_problem

    p = make_problem(CONFIGS["grid2383_n96"], coupling="paper")
    N, nC = p.N, p.nC
    ns = nC // N
    up = lambda v: torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).to(dev)  # noqa: E731
    a, b, c, r = up(p.a_vals), up(p.b_vals), up(p.c_vals), up(p.rhs)
    x = torch.empty_like(r)
    bp = np.asarray(p.b_blockptr, dtype=np.int64)
    records = int(np.sum((bp[1:] - bp[:-1]) ** 2))
    # partial LDL^T of order 2 n_s with n_s pivots per period (the last: n_s of order n_s)
    chain_flops = (N - 1) * 7.0 * ns ** 3 / 3.0 + ns ** 3 / 3.0
    fp64_gflops = B.kkt_measure_fp64_peak()
    out = {"workload": f"grid2383_n96_paper: the 2,383-bus grid over 96 periods with the paper's cumulative "
                       f"coupling (C = 0), n_C = {nC:,} ({ns} per period), blocks nA={p.nA:,}",
           "dense_s_gather_records": records, "dense_s_factor_flops": nC ** 3 / 3.0,
           "dense_s_factor_ms_at_fp64_peak": nC ** 3 / 3.0 / (fp64_gflops * 1e6),
           "structured_factor_flops": chain_flops}
    for prec in ("fp64", "tf32"):
        t0 = time.perf_counter()
        h = B.kkt_analyze(p, B.kkt_default_options(prec, structured_s=2, refine_mode=args.refine_mode))
        ana_ms = (time.perf_counter() - t0) * 1e3
        try:
            def step():
                B.kkt_factor(h, a, b, c, stream)
                B.kkt_solve(h, r, x, 1, stream)

            for _ in range(warmup):
                step()
            torch.cuda.synchronize()
            ms, ph = [], {"a_block_factor": [], "b_schur_assembly": [], "c_structured_factor": [], "d_solve": []}
            for _ in range(steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step()
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
                info = B.kkt_get_info(h)
                ph["a_block_factor"].append(info["ms_block_factor"])
                ph["b_schur_assembly"].append(info["ms_schur_assembly"])
                ph["c_structured_factor"].append(info["ms_dense_factor"])
                ph["d_solve"].append(info["ms_solve_device"])
            expect = [N * p.nP, N * (p.nA - p.nP) + nC, 0]
            cms = statistics.mean(ph["c_structured_factor"])
            out[prec] = {"value": 1e3 / statistics.mean(ms), "unit": "solves/s", "ms_per_step": statistics.mean(ms),
                         "analyze_ms": ana_ms, "phases_ms": {k: statistics.mean(v) for k, v in ph.items()},
                         "structured_factor": {"bound": "alu", "gflops": chain_flops / cms / 1e6,
                                               "frac_of_fp64_peak": chain_flops / cms / 1e6 / fp64_gflops},
                         "eta": info["rel_residual"], "refine_steps": info["refine_steps"],
                         "fell_back_fp64": info["fell_back_fp64"],
                         "inertia_ok": [info["n_pos"], info["n_neg"], info["n_zero"]] == expect,
                         "device_bytes": info["device_bytes"]}
        finally:
            B.kkt_destroy(h)
    return out


def _accuracy(B, h, prob, r, x, stream, torch):
    """eta (device), ||r - Kx||_2 / ||r||_2 from the handle's residual kernel,
    and the solution on the host."""
    import numpy as np

    rho = torch.empty_like(x)
    B.kkt_residual(h, r, x, rho, stream)
    torch.cuda.synchronize()
    rh, xh = rho.cpu().numpy(), x.cpu().numpy()
    info = B.kkt_get_info(h)
    return {"eta": info["rel_residual"], "resid2": float(np.linalg.norm(rh) / np.linalg.norm(prob.rhs)),
            "refine_steps": info["refine_steps"], "fell_back_fp64": info["fell_back_fp64"]}, xh


def run_single(args):
    import numpy as np
    import torch

    from gen import build_workload
    from paper_1907_05420_gb300 import binding as B

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    def max_over_ranks(v):
        if world > 1:
            import torch.distributed as dist

            t = torch.tensor([v], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            return float(t.item())
        return v

    prob = build_workload(args.workload)
    wd = workload_defaults(args.workload)
    autotune = wd["autotune"] if args.autotune < 0 else args.autotune
    stream = torch.cuda.current_stream()
    up = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(dev)  # noqa: E731
    a, b, c, r = up(prob.a_vals), up(prob.b_vals), up(prob.c_vals), up(prob.rhs)
    x = torch.empty_like(r)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def analyze(mode, time_kernels=0):
        prec, opts, tol = parse_leg(mode)
        kw = dict(opts, autotune=autotune, early_solve=1, time_kernels=time_kernels,
                  tail_ratio=0.0 if autotune else wd["tail_ratio"], refine_mode=args.refine_mode)
        if tol is not None:
            kw["refine_tol"] = tol
        return B.kkt_analyze(prob, B.kkt_default_options(prec, **kw))

    def time_mode(h, steps, warmup, sample_clocks=False, kernel_stats=False):
        """Factor + refined solve, `steps` timed repetitions with CUDA events."""
        def step():
            B.kkt_factor(h, a, b, c, stream)
            B.kkt_solve(h, r, x, 1, stream, allow_not_converged=True)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        launches0 = B.kkt_get_info(h)["n_launches"]
        clocks = ClockSampler(local) if sample_clocks else None
        if clocks:
            clocks.start()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        phases = {"a_block_factor": [], "b_schur_assembly": [], "c_dense_factor": [], "d_solve": []}
        etas, steps_ir, fallback = [], [], []
        kstats = {}
        t_wall0 = time.perf_counter()
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
            inf = B.kkt_get_info(h)  # synchronizes; the per-step device figures of this step
            phases["a_block_factor"].append(inf["ms_block_factor"])
            phases["b_schur_assembly"].append(inf["ms_schur_assembly"])
            phases["c_dense_factor"].append(inf["ms_dense_factor"])
            phases["d_solve"].append(inf["ms_solve_device"])
            etas.append(inf["rel_residual"])
            steps_ir.append(inf["refine_steps"])
            fallback.append(inf["fell_back_fp64"])
            if kernel_stats:
                for name, st in B.kkt_kernel_stats(h).items():
                    acc = kstats.setdefault(name, {"launches": 0, "ms_total": 0.0, "flops": 0.0})
                    for kk in acc:
                        acc[kk] += st[kk]
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
        clk = clocks.stop() if clocks else None
        info = B.kkt_get_info(h)
        step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
        return {"info": info, "step_ms": step_ms, "total_s": max_over_ranks(sum(step_ms) / 1e3),
                "phases": phases, "etas": etas, "steps_ir": steps_ir, "fallback": fallback, "clocks": clk,
                "launches": info["n_launches"] - launches0, "wall_s": t_wall, "kstats": kstats}

    # ---- the timed path
    h = analyze(args.prec, time_kernels=1)
    info0 = B.kkt_get_info(h)
    main_run = time_mode(h, args.steps, args.warmup, sample_clocks=True, kernel_stats=True)
    value = world * args.steps / main_run["total_s"]
    step_ms, phases = main_run["step_ms"], main_run["phases"]
    acc_main, x_main = _accuracy(B, h, prob, r, x, stream, torch)
    acc_main.update(eta_max_timed=max(main_run["etas"]), refine_steps_mean=statistics.mean(main_run["steps_ir"]))

    # ---- end to end through the public API with host buffers: H2D of the
    # step's inputs and D2H of the solution inside the timed region
    e2e = None
    if not args.no_e2e:
        ksteps = max(1, min(args.steps, args.e2e_steps))
        pin = lambda arr: torch.from_numpy(np.ascontiguousarray(arr)).pin_memory()  # noqa: E731
        ha, hb, hc, hr = pin(prob.a_vals), pin(prob.b_vals), pin(prob.c_vals), pin(prob.rhs)
        hx = torch.empty_like(hr).pin_memory()
        B.kkt_factor(h, ha, hb, hc, stream)
        B.kkt_solve(h, hr, hx, 1, stream, allow_not_converged=True)
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ksteps):
            flush.zero_()
            B.kkt_factor(h, ha, hb, hc, stream)
            B.kkt_solve(h, hr, hx, 1, stream, allow_not_converged=True)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        e2e_s = max_over_ranks(e0.elapsed_time(e1) / 1e3)
        h2d = sum(t.numel() * t.element_size() for t in (ha, hb, hc, hr))
        e2e = {"value": world * ksteps / e2e_s, "unit": "solves/s", "steps": ksteps,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(hx.numel() * 8)}
        del ha, hb, hc, hr, hx
    B.kkt_destroy(h)  # every leg below needs the device memory

    # ---- the other modes, one handle at a time
    legs, xs = {}, {}
    for leg in [m for m in args.legs.split(",") if m and m != args.prec]:
        hl = analyze(leg)
        lr = time_mode(hl, args.leg_steps, args.leg_warmup)
        acc, xs[leg] = _accuracy(B, hl, prob, r, x, stream, torch)
        B.kkt_destroy(hl)
        legs[leg] = {"value": world * args.leg_steps / lr["total_s"], "unit": "solves/s",
                     "ms_per_step": statistics.mean(lr["step_ms"]),
                     "latency_ms": {"p50": float(np.percentile(lr["step_ms"], 50)),
                                    "p99": float(np.percentile(lr["step_ms"], 99))},
                     "accuracy": acc, "phases_ms": {kk: statistics.mean(v) for kk, v in lr["phases"].items()}}

    slack = None if args.no_slack else slack_timing(args, dev, stream, torch, np, B)
    paper = None if args.no_paper else structured_paper_timing(args, dev, stream, torch, np, B)
    serving = None
    if not args.no_serve and world == 1:
        serving = serve_sweep(args, args.serve_modes.split(","), [float(q) for q in args.rates.split(",")],
                              args.serve_seconds_default)

    # ---- forward errors against the FP64-accurate solutions of this run
    ref_leg = next((m for m in ("fp64+band", "fp64", "f64emu") if m in xs), None)
    err = lambda xv, xr: float(np.max(np.abs(xv - xr)) / np.max(np.abs(xr)))  # noqa: E731
    if ref_leg:
        acc_main["fwd_err_vs_" + ref_leg] = err(x_main, xs[ref_leg])
        for leg, xv in xs.items():
            if leg != ref_leg:
                legs[leg]["accuracy"]["fwd_err_vs_" + ref_leg] = err(xv, xs[ref_leg])

    # ---- roofline of the dominant kernel (per-launch CUDA events inside the timed region)
    peaks, peak_kind = _peaks()
    fp64_gflops = B.kkt_measure_fp64_peak()
    ks = main_run["kstats"]
    timed = {kk: v for kk, v in ks.items() if v["launches"] > 0}
    dom = max(timed, key=lambda kk: timed[kk]["ms_total"]) if timed else None
    roofline = None
    if dom:
        st = timed[dom]
        sec = st["ms_total"] / 1e3
        sustained = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        if dom in ("k_tc_update_emu", "k_tc_update_emu_wide"):
            bound, unit, peak = "tensor", "TFLOP/s", sustained
            achieved = EMU_PRODUCTS * st["flops"] / sec / 1e12
            src = (f"bf16_tflops_sustained of {peak_kind} peaks; achieved counts the {EMU_PRODUCTS:.0f} BF16 "
                   "digit products of every FP64 multiply-add")
        elif dom in ("k_tc_update_wide", "k_tc_update"):
            bound, unit, peak = "tensor", "TFLOP/s", sustained * TF32_RATIO
            achieved = st["flops"] / sec / 1e12
            src = f"bf16_tflops_sustained of {peak_kind} peaks x {TF32_RATIO:.3f} (TF32 / BF16 nominal)"
        else:
            bound, unit, peak = "alu", "TFLOP/s", fp64_gflops / 1e3
            achieved = st["flops"] / sec / 1e12
            src = "FP64 FMA throughput measured by kkt_measure_fp64_peak in this run"
        roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                    "traffic": TRAFFIC.get((args.workload, dom)), "kernel": dom,
                    "launches_per_step": st["launches"] / args.steps,
                    "ms_per_launch": st["ms_total"] / st["launches"],
                    "flops_per_launch": st["flops"] / st["launches"], "peak_source": src}
    kernels = {}
    step_total = sum(step_ms)
    for kk, v in timed.items():
        kernels[kk] = {"launches_per_step": v["launches"] / args.steps, "ms_per_step": v["ms_total"] / args.steps,
                       "share_of_step": v["ms_total"] / step_total if step_total else None,
                       "tflops": v["flops"] / (v["ms_total"] / 1e3) / 1e12 if v["flops"] else None}

    # ---- phases against their bounds (algorithmic work per solve)
    info = main_run["info"]
    N, nA, nC = prob.N, prob.nA, prob.nC
    k, nw = info["k_coupling_rows"], info["w_rows"]
    mean = {kk: statistics.mean(v) for kk, v in phases.items()}
    ir = acc_main["refine_steps_mean"]
    # algorithmic work per solve (2 flops per multiply-add): (a) reads A and
    # writes L and D once; (b) the contraction W^T D^-1 W, its symmetric half;
    # (c) the dense LDL^T of S, n^3/3 flops; (d) each application reads the
    # block factors twice and S once
    work = {
        "a_block_factor": ("hbm", 8.0 * N * (prob.nnzA + info["nnz_l"] + nA)),
        "b_schur_assembly": ("tensor", float(N) * nw * k * k),
        "c_dense_factor": ("tensor", nC ** 3 / 3.0),
        "d_solve": ("hbm", (1 + ir) * (8.0 * N * (2 * info["panel_doubles"] + 2 * nA) + 8.0 * nC * nC)),
    }
    sustained = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
    s_peak = sustained * ({"tf32": TF32_RATIO, "bf16": 1.0}.get(args.prec, 1.0))
    phase_report = {}
    for kk, ms in mean.items():
        s = ms / 1e3
        kind, w = work[kk]
        if s <= 0:
            phase_report[kk] = {"ms": ms}
        elif kind == "hbm":
            phase_report[kk] = {"ms": ms, "bound": "hbm", "bytes": w, "gbs": w / s / 1e9,
                                "frac": w / s / 1e9 / peaks["hbm_gbs"]}
        else:
            phase_report[kk] = {"ms": ms, "bound": "tensor", "flops": w, "tflops": w / s / 1e12,
                                "frac": w / s / 1e12 / s_peak}

    mixed_vs_fp64 = None
    if "fp64+band" in legs:
        fp = legs["fp64+band"]
        mixed_vs_fp64 = {"fp64_path": "fp64+band (FP64 on the CUDA cores, FP64 tails, banded factor of S)",
                         "fp64_value": fp["value"], "fp64_eta": fp["accuracy"]["eta"],
                         "at_1e-10": {"mixed": value, "ratio": value / fp["value"]}}
        tight = f"tf32@{TIGHT_TOL:g}"
        if tight in legs:
            mixed_vs_fp64[f"at_{TIGHT_TOL:g}"] = {
                "mixed": legs[tight]["value"], "ratio": legs[tight]["value"] / fp["value"],
                "mixed_eta": legs[tight]["accuracy"]["eta"]}

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "tf32": "f64+tf32", "bf16": "f64+bf16", "f64emu": "f64+bf16x7"}[args.prec],
        "data": "synthetic",
        "config": {"workload": workload_desc(args.workload), "precision": args.prec,
                   "refinement": ["iterative", "gmres"][args.refine_mode],
                   "l2": "256 MB buffer written before every timed step (inputs also exceed L2)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "accuracy": acc_main, "mixed_vs_fp64": mixed_vs_fp64,
        "roofline": roofline, "kernels": kernels, "phases": phase_report,
        "fp64_peak_gflops_measured": fp64_gflops,
        "e2e": e2e, "clocks": main_run["clocks"], "gpu_launches": int(main_run["launches"]),
        "wall_s_timed": main_run["wall_s"], "analyze_ms": info0["ms_analyze"],
        "dense_tail": {"cols": info0["dense_tail_cols"], "ratio": info0["tail_ratio"],
                       "augmented": bool(info0["tail_augmented"]),
                       "autotune_candidates": info0["autotune_candidates"]},
        "device_bytes": info0["device_bytes"], "other_precisions": legs, "slack_elimination": slack,
        "structured_paper": paper, "serving": serving,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], out = cpu_baseline_sample(args.workload, prob, info0["factor_flops"])
        if out is not None:
            xo = out["x"]
            acc_main["fwd_err_vs_oracle"] = err(x_main, xo)
            for leg, xv in xs.items():
                legs[leg]["accuracy"]["fwd_err_vs_oracle"] = err(xv, xo)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
