#!/usr/bin/env python3
"""KKT solves/s of the Schur-complement solve of a multiperiod storage OPF
system on GB300.

Workload: the synthetic 2,383-bus grid (2,900 lines, 327 generators, 100
storage units) over 96 periods; blocks A_i of size 10,486, coupling S of
size 9,600 (input recipe in gen/mpopf.py).  One step = one KKT solve: the
numeric factorization (block factors, Schur assembly, dense factor of S) plus
the solve with FP64 iterative refinement to eta <= 1e-10.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp64|tf32|bf16]
    python bench.py --impl reference ...   # the CPU oracle, timed on the host

Multi-GPU (torchrun, one rank per GPU): independent replicas, one system per
rank, no data-path collective; value = solves of all ranks / max rank time.
"""
from __future__ import annotations

import argparse
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
WORKLOAD = "grid2383_n96"
WORKLOAD_DESC = ("grid2383_n96: synthetic 2,383-bus grid, 2,900 lines, 327 generators, "
                 "100 storage units, N=96 periods; blocks nA=10,486; S 9,600 x 9,600")
L2_FLUSH_BYTES = 256 << 20


def workload_desc(name):
    """The config.workload string: the named instance and its sizes."""
    if name == WORKLOAD:
        return WORKLOAD_DESC
    from gen import describe_workload

    return describe_workload(name)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
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


def cpu_reference_solve(prob, perm=None):
    """One oracle solve of the workload on the host cores (the CPU baseline).

    The ordering is analysis (once per pattern, like kkt_analyze on the GPU
    side) and is computed outside the timed region when `perm` is None.
    """
    import oracle

    if perm is None:
        perm = oracle.min_degree(prob.nA, prob.a_rowptr, prob.a_col, prob.nP)
    t0 = time.perf_counter()
    out = oracle.kkt_solve(prob, perm)
    dt = time.perf_counter() - t0
    return out, dt


# CPU work of one bounded oracle sample, in flops (the oracle runs the full
# 2,383-bus, 96-period solve, 3e11 flops, in about 14 s on 16 Grace cores)
CPU_SAMPLE_FLOPS = 6e11


def cpu_baseline_sample(workload, prob, block_flops):
    """The oracle timed on a bounded sample of the workload.

    Returns (line fields, oracle output of the full system or None).  A
    workload whose estimated oracle work, N * block_flops + nC^3 / 3, exceeds
    CPU_SAMPLE_FLOPS is sampled by its first N' periods (the largest N' within
    that work) and the rate scaled to the full system by the ratio of the two
    estimates."""
    import dataclasses

    import oracle
    from gen import CONFIGS, make_problem

    ns = prob.nC // prob.N if prob.N else 0
    est = lambda n: n * block_flops + (n * ns) ** 3 / 3.0  # noqa: E731
    full = est(prob.N)
    fields = {"unit": "solves/s", "cores": oracle.max_threads(), "host_cores": host_cores(), "kind": "oracle"}
    if full <= CPU_SAMPLE_FLOPS or workload not in CONFIGS:
        out, dt = cpu_reference_solve(prob)
        fields.update(value=1.0 / dt, sample=f"1 full solve of {workload} (FP64 oracle, OpenMP; "
                                             "ordering computed once, untimed)")
        return fields, out
    fit = [k for k in range(1, prob.N + 1) if est(k) <= CPU_SAMPLE_FLOPS]
    n = fit[-1] if fit else 1
    sub = make_problem(dataclasses.replace(CONFIGS[workload], n_per=n, name=f"{workload}_first{n}"))
    _, dt = cpu_reference_solve(sub)
    scale = full / est(n)
    fields.update(value=1.0 / (dt * scale),
                  sample=f"1 solve of {workload} over its first {n} of {prob.N} periods (FP64 oracle, "
                         f"OpenMP; {dt:.1f} s), scaled to the full system by its estimated work "
                         f"N*block_flops + nC^3/3 (x{scale:.1f})")
    return fields, None


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count()


def run_reference(args):
    """--impl reference: the CPU oracle, timed as it stands on the host cores."""
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from gen import CONFIGS, build_workload, make_problem

    prob = build_workload(args.workload)
    small = make_problem(CONFIGS["grid30_n24"])
    for _ in range(args.warmup):  # warm-up on the small instance (loads the library, threads)
        oracle.kkt_solve(small)
    perm = oracle.min_degree(prob.nA, prob.a_rowptr, prob.a_col, prob.nP)  # analysis, untimed
    times = []
    for _ in range(args.steps):
        _, dt = cpu_reference_solve(prob, perm)
        times.append(dt)
    total = sum(times)
    value = args.steps / total
    threads = oracle.max_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(args.workload), "precision": "fp64", "parallelism": "none (host)"},
        "latency_ms": {"p50": 1e3 * statistics.median(times),
                       "p99": 1e3 * max(times) if len(times) < 100 else
                       1e3 * sorted(times)[int(0.99 * len(times))]},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": threads, "kind": "oracle",
                         "sample": f"{args.steps} full solves of {args.workload}, ordering computed once "
                                   f"untimed (warm-up: {args.warmup} solves of grid30_n24)"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


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
    import numpy as np
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


def run_serve(args):
    """Poisson request stream over the size mix; p50/p99 latency and solves/s per rate."""
    import numpy as np
    import torch

    from paper_1907_05420_gb300 import binding as B

    out = {"metric": "KKT solves/s and p50/p99 latency under a Poisson request stream", "unit": "solves/s",
           "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
           "config": {"workload": f"serve: {args.serve_pool} resident patterns from the size mix; "
                                  "Poisson arrivals; every request carries fresh values",
                      "slots": args.serve_slots, "seconds_per_rate": args.serve_seconds,
                      "backlog": args.serve_backlog or 4 * args.serve_slots}}
    for prec in args.batch_precs.split(","):
        probs, hs, vals, xs = _mix_problems(args.serve_pool, prec)
        srv = B.KKTServer(slots=args.serve_slots,
                          device_budget_bytes=int(0.8 * torch.cuda.mem_get_info()[0]))
        rng = np.random.default_rng(4242)
        res = {}
        backlog = args.serve_backlog or 4 * args.serve_slots
        for rate in [float(r) for r in args.rates.split(",")]:
            # Poisson arrivals for 1 s of warm-up plus the measured window; a
            # request that finds `backlog` requests outstanding is shed (load
            # shedding keeps the queue, and so the drain after the window, bounded)
            lats, outstanding = [], {}
            shed = offered = 0
            t0 = time.perf_counter()
            t_measure, t_end = t0 + 1.0, t0 + 1.0 + args.serve_seconds
            t_next = t0

            def reap(block):
                for rid in list(outstanding):
                    got = srv.wait(rid) if block else srv.poll(rid)
                    if got is None:
                        continue
                    in_window = outstanding.pop(rid)
                    if in_window:
                        lats.append(got[1])

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
                k = int(rng.integers(0, len(probs)))
                a, b, c, r = vals[k]
                x = torch.empty_like(r)
                outstanding[srv.submit(hs[k], a, b, c, r, x)] = in_window
            reap(True)
            t_done = time.perf_counter()
            n = len(lats)
            res[str(int(rate))] = {"offered": offered, "served": n, "shed": shed,
                                   "solves_per_s": n / max(1e-9, t_done - t_measure),
                                   "p50_ms": float(np.percentile(lats, 50)) if n else None,
                                   "p99_ms": float(np.percentile(lats, 99)) if n else None}
        srv.close()
        for h in hs:
            B.kkt_destroy(h)
        out[prec] = res
    out["value"] = max(v["solves_per_s"] for v in out[args.batch_precs.split(",")[0]].values())
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="tf32", choices=["fp64", "tf32", "bf16", "f64emu"],
                    help="arithmetic of the dense factor of S on the timed path (default: the "
                         "mixed path, TF32 tensor cores with FP64 refinement)")
    ap.add_argument("--legs", default="fp64,f64emu,bf16,tf32+tcg,fp64+band,tf32+band",
                    help="other precision modes measured beside the timed path ('' for none)")
    ap.add_argument("--leg-steps", type=int, default=4)
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-precs", default="tf32,fp64")
    ap.add_argument("--batch-streams", type=int, default=8)
    ap.add_argument("--serve-pool", type=int, default=32)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--rates", default="50,100,200,500,1000,2000")
    ap.add_argument("--serve-backlog", type=int, default=0,
                    help="requests outstanding before new arrivals are shed (default 4 x slots)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the dense-tail autotuning at analysis (it times a few factorizations)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "mix64":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)

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

    prob = build_workload(args.workload)
    stream = torch.cuda.current_stream()
    a = torch.from_numpy(np.ascontiguousarray(prob.a_vals)).to(dev)
    b = torch.from_numpy(np.ascontiguousarray(prob.b_vals)).to(dev)
    c = torch.from_numpy(np.ascontiguousarray(prob.c_vals)).to(dev)
    r = torch.from_numpy(np.ascontiguousarray(prob.rhs)).to(dev)
    x = torch.empty_like(r)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def time_mode(mode, steps, warmup, sample_clocks=False):
        """Factor + refined solve of the workload, `steps` timed repetitions.

        mode: a precision name; a '+tcg' suffix also runs the Schur contraction on
        the tensor cores in that precision, '+band' limits the factor of S to its
        row envelope (the structured Schur factor)."""
        prec, _, extra = mode.partition("+")
        h = B.kkt_analyze(prob, B.kkt_default_options(prec, reduced_contraction=int(extra == "tcg"),
                                                     structured_s=int(extra == "band"),
                                                     autotune=0 if args.no_autotune else 1,
                                                     early_solve=1))
        info0 = B.kkt_get_info(h)

        def step_device():
            B.kkt_factor(h, a, b, c, stream)
            B.kkt_solve(h, r, x, 1, stream, allow_not_converged=True)

        for _ in range(warmup):
            step_device()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        launches0 = B.kkt_get_info(h)["n_launches"]
        clocks = ClockSampler(local) if sample_clocks else None
        if clocks:
            clocks.start()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        phases = {"a_block_factor": [], "b_schur_assembly": [], "c_dense_factor": [], "d_solve": []}
        etas, steps_ir, fallback = [], [], []
        t_wall0 = time.perf_counter()
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            step_device()
            ev[i][1].record(stream)
            inf = B.kkt_get_info(h)
            phases["a_block_factor"].append(inf["ms_block_factor"])
            phases["b_schur_assembly"].append(inf["ms_schur_assembly"])
            phases["c_dense_factor"].append(inf["ms_dense_factor"])
            phases["d_solve"].append(inf["ms_solve_device"])
            etas.append(inf["rel_residual"])
            steps_ir.append(inf["refine_steps"])
            fallback.append(inf["fell_back_fp64"])
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
        clk = clocks.stop() if clocks else None
        info = B.kkt_get_info(h)
        step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
        total_s = sum(step_ms) / 1e3
        if world > 1:
            import torch.distributed as dist

            t = torch.tensor([total_s], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            total_s = float(t.item())
        return {"h": h, "info0": info0, "info": info, "step_ms": step_ms, "total_s": total_s,
                "phases": phases, "etas": etas, "steps_ir": steps_ir, "fallback": fallback,
                "clocks": clk, "launches": info["n_launches"] - launches0, "wall_s": t_wall,
                "x": x.cpu().numpy()}

    main_run = time_mode(args.prec, args.steps, args.warmup, sample_clocks=True)
    h = main_run["h"]
    info0, info = main_run["info0"], main_run["info"]
    step_ms, phases = main_run["step_ms"], main_run["phases"]
    etas, steps_ir = main_run["etas"], main_run["steps_ir"]
    clk, launches, t_wall = main_run["clocks"], main_run["launches"], main_run["wall_s"]
    value = world * args.steps / main_run["total_s"]
    x_gpu = main_run["x"]

    # end to end through the public API with host buffers: H2D of the step's
    # inputs and D2H of the solution inside the timed region
    e2e = None
    if not args.no_e2e:
        pin = lambda arr: torch.from_numpy(np.ascontiguousarray(arr)).pin_memory()  # noqa: E731
        ha, hb, hc, hr = pin(prob.a_vals), pin(prob.b_vals), pin(prob.c_vals), pin(prob.rhs)
        hx = torch.empty_like(hr).pin_memory()
        for _ in range(max(1, args.warmup)):
            B.kkt_factor(h, ha, hb, hc, stream)
            B.kkt_solve(h, hr, hx, 1, stream, allow_not_converged=True)
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            flush.zero_()
            B.kkt_factor(h, ha, hb, hc, stream)
            B.kkt_solve(h, hr, hx, 1, stream, allow_not_converged=True)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        e2e_s = e0.elapsed_time(e1) / 1e3
        if world > 1:
            import torch.distributed as dist

            t = torch.tensor([e2e_s], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        h2d = sum(t.numel() * t.element_size() for t in (ha, hb, hc, hr))
        e2e = {"value": world * args.steps / e2e_s, "unit": "solves/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(hx.numel() * 8)}

    legs = {}
    for leg in [m for m in args.legs.split(",") if m and m != args.prec]:
        lr = time_mode(leg, args.leg_steps, 2)
        B.kkt_destroy(lr["h"])
        legs[leg] = {"value": world * args.leg_steps / lr["total_s"], "unit": "solves/s",
                     "ms_per_step": statistics.mean(lr["step_ms"]),
                     "latency_ms": {"p50": float(np.percentile(lr["step_ms"], 50)),
                                    "p99": float(np.percentile(lr["step_ms"], 99))},
                     "residual_eta_max": max(lr["etas"]), "refine_steps": lr["steps_ir"][-1],
                     "fell_back_fp64": lr["fallback"][-1],
                     "phases_ms": {kk: statistics.mean(v) for kk, v in lr["phases"].items()},
                     "_x": lr["x"]}

    # roofline of the dominant phase (algorithmic work / measured phase time)
    peaks, peak_kind = _peaks()
    fp64_gflops = B.kkt_measure_fp64_peak()
    N, nA, nC = prob.N, prob.nA, prob.nC
    k, nw = info["k_coupling_rows"], info["w_rows"]
    mean = {kk: statistics.mean(v) for kk, v in phases.items()}
    ir = statistics.mean(steps_ir)
    work = {
        "a_block_factor": {"flops": N * info["factor_flops"],
                           "bytes": 8.0 * N * (prob.nnzA + info["nnz_l"] + nA)},
        "b_schur_assembly": {"flops": N * nw * k * k, "bytes": 8.0 * N * 2 * nw * k},
        "c_dense_factor": {"flops": nC ** 3 / 3.0, "bytes": 8.0 * nC * nC},
        "d_solve": {"flops": 0.0,
                    "bytes": (1 + ir) * (8.0 * N * (2 * info["panel_doubles"] + 2 * nA) + 8.0 * nC * nC)},
    }
    dom = max(mean, key=mean.get)
    t_dom = mean[dom] / 1e3
    if dom == "d_solve":
        bound, peak, unit = "hbm", peaks["hbm_gbs"], "GB/s"
        achieved = work[dom]["bytes"] / t_dom / 1e9
        peak_src = f"hbm_gbs of {peak_kind} peaks"
    elif dom == "c_dense_factor" and args.prec != "fp64":
        # TF32 runs at half the BF16 rate (nominal 1.1 vs 2.25 PFLOP/s dense); the
        # emulated FP64 update issues 28 BF16 digit products per FP64 product
        ratio = {"tf32": 0.5, "bf16": 1.0, "f64emu": 1.0}[args.prec]
        mult = 28.0 if args.prec == "f64emu" else 1.0
        bound, peak, unit = "tensor", peaks["bf16_tflops"] * ratio, "TFLOP/s"
        achieved = mult * work[dom]["flops"] / t_dom / 1e12
        peak_src = (f"bf16_tflops of {peak_kind} peaks x {ratio} ({args.prec})" +
                    (", achieved counts the 28 digit products" if mult > 1 else ""))
    else:
        bound, peak, unit = "alu", fp64_gflops / 1e3, "TFLOP/s"
        achieved = work[dom]["flops"] / t_dom / 1e12
        peak_src = "FP64 FMA throughput measured by kkt_measure_fp64_peak in this run"
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": None, "phase": dom, "peak_source": peak_src}
    phase_report = {}
    for kk, ms in mean.items():
        s = ms / 1e3
        phase_report[kk] = {"ms": ms, "gflops": work[kk]["flops"] / s / 1e9 if s > 0 else None,
                            "gbs": work[kk]["bytes"] / s / 1e9 if s > 0 else None,
                            "hbm_frac": work[kk]["bytes"] / s / 1e9 / peaks["hbm_gbs"] if s > 0 else None}

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "tf32": "f64+tf32", "bf16": "f64+bf16", "f64emu": "f64+bf16x7"}[args.prec],
        "data": "synthetic",
        "config": {"workload": workload_desc(args.workload), "precision": args.prec,
                   "l2": "256 MB buffer written before every timed step",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "residual_eta_max": max(etas), "refine_steps_mean": ir,
        "roofline": roofline, "phases": phase_report, "fp64_peak_gflops_measured": fp64_gflops,
        "e2e": e2e, "clocks": clk, "gpu_launches": int(launches), "wall_s_timed": t_wall,
        "analyze_ms": info0["ms_analyze"], "refine_steps_last": steps_ir[-1],
        "dense_tail": {"cols": info0["dense_tail_cols"], "ratio": info0["tail_ratio"],
                       "augmented": bool(info0["tail_augmented"]),
                       "autotune_candidates": info0["autotune_candidates"]},
        "fell_back_fp64": main_run["fallback"][-1], "other_precisions": legs,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], out = cpu_baseline_sample(args.workload, prob, info0["factor_flops"])
        if out is not None:
            xo = out["x"]
            err = lambda xv: float(np.max(np.abs(xv - xo)) / np.max(np.abs(xo)))  # noqa: E731
            line["error_vs_oracle"] = err(x_gpu)
            for leg in legs.values():
                leg["error_vs_oracle"] = err(leg["_x"])
    for leg in legs.values():
        leg.pop("_x", None)
    B.kkt_destroy(h)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
