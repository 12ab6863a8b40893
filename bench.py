"""Benchmark of the CP-MDP GridWorld hot path on GB300.

Workload: 3-D GridWorld 64^3 (262,144 states), 6 actions, p = 0.8 (0.05 to
each perpendicular move), 5 % seeded obstacles, 8 goal cells with reward
U(0.5, 1), step reward -0.01, gamma = 0.99; FP32 value tensor.

One step = the whole hot path on that instance, inputs resident on the
device: fused value iteration from zeros to max|dV| < 1e-6 with the FP64
certifying sweep and policy extraction, then fused policy iteration from
zeros with its FP64 certifying sweep. The metric is state-action backups
per second over the step (|S| |A| per VI / improvement sweep, |S| per
evaluation sweep); time-to-1e-6 of the fused VI is reported next to the
plain unfused FP32 VI (one kernel per action, separate max and residual
kernels, residual checked on the host every sweep) on the same GPU.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU FP64 oracle (plain C, OpenMP) on the same
instance instead. Under torchrun each rank solves its own instance
(replicas: the path has no exchange step), value = all ranks' backups over
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "state-action backups/s and time to |dV|inf<1e-6 vs plain FP32 VI, same GB300"
UNIT = "state-action backups/s"
SIDE = 64
TOL = 1e-6
BYTES_VI = 13      # per state per VI sweep: V 4 + R 4 + code 1 + V' 4
BYTES_EVAL = 14    # + policy read
BYTES_IMPROVE = 14 # V 4 + R 4 + code 1 + policy 1 + V' 4 (the new policy's first evaluation step)
BYTES_GREEDY = 10  # V 4 + R 4 + code 1 + policy 1 (the initial greedy sweep writes no values)


def workload(seed):
    import cpmdp_inputs as ci
    return ci.config_3d(side=SIDE, seed=seed)


def config_dict(extra=None):
    d = {"workload": f"gridworld-3d-{SIDE}^3-A6-p0.8-obst5%-goals8-gamma0.99-fp32",
         "states": SIDE ** 3, "actions": 6, "tol": TOL,
         "step": "fused VI to 1e-6 + FP64 certify + fused PI + FP64 certify, zero init",
         "l2": "flushed between timed steps (256 MiB write)",
         "parallelism": "replicas (independent instance per rank)"}
    if extra:
        d.update(extra)
    return d


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        mhz, maxmhz, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                maxmhz.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not mhz:
            return None
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": max(maxmhz), "reasons": sorted(reasons),
                "samples": len(mhz)}


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = os.environ.get("CPMDP_BENCH_BACKEND", "nccl")
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return rank, world, local, pg


def aggregate(pg, units, ms, device=None):
    """Sum of units over ranks and max of the timed milliseconds."""
    if pg is None:
        return units, ms
    import torch
    dev = device if device is not None else "cpu"
    t = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    m = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    pg.all_reduce(m, op=pg.ReduceOp.MAX)
    return float(t.item()), float(m.item())


def sources_hash(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2103_00331_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def traffic_from_profile(kernel_file, scale=None):
    """DRAM bytes per launch of a kernel from its committed ncu summary, if
    that summary was taken on the current sources of that kernel (the
    summary's `sources:` line lists them, `sources_sha256_16:` their hash).
    With scale = a state count, the summary's bytes per state times that
    count (for captures taken on a smaller case of the same kernel)."""
    path = os.path.join(ROOT, "profiles", kernel_file)
    if not os.path.exists(path):
        return None
    vals = {}
    for ln in open(path):
        if ":" in ln and not ln.startswith("#"):
            k, v = ln.split(":", 1)
            vals[k.strip()] = v.strip()
    try:
        if vals.get("sources_sha256_16") != sources_hash(vals["sources"].split()):
            return None
        if scale is not None:
            return float(vals["dram_bytes_per_state"].split()[0]) * scale
        return float(vals["dram_bytes_per_launch"].split()[0])
    except (KeyError, ValueError, OSError):
        return None


def cpu_oracle_sample(gw, budget_s=12.0, max_reps=50):
    """The FP64 C oracle (as it stands) on the same instance: repeated full
    value-iteration solves to 1e-6 from zeros until ~budget_s of CPU time."""
    from oracle import cpfactor as oc
    oc.build()
    S, A = gw.nstates, 2 * len(gw.shape)
    t0 = time.perf_counter()
    backups, reps = 0, 0
    while True:
        _, _, k, _ = oc.value_iteration(gw, tol=TOL, max_iter=5000)
        backups += k * S * A
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= max_reps:
            break
    out = {"value": backups / el, "unit": UNIT, "cores": oc.threads(), "kind": "oracle",
           "sample": f"{reps} full FP64 VI solves to 1e-6 of the 64^3 instance ({k} sweeps each), "
                     f"{el:.1f} s on {oc.threads()} OpenMP threads"}
    # the same oracle on one core (a bounded sample: whole solves until ~budget_s / 3)
    nthreads = oc.threads()
    oc.set_threads(1)
    try:
        t0 = time.perf_counter()
        b1, r1 = 0, 0
        while True:
            _, _, k1, _ = oc.value_iteration(gw, tol=TOL, max_iter=5000)
            b1 += k1 * S * A
            r1 += 1
            el1 = time.perf_counter() - t0
            if el1 >= budget_s / 3 or r1 >= max_reps:
                break
    finally:
        oc.set_threads(nthreads)
    out["one_core"] = {"value": b1 / el1, "unit": UNIT, "cores": 1,
                       "sample": f"{r1} full FP64 VI solves of the same instance, {el1:.1f} s on 1 thread"}
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    gw = workload(0)
    from oracle import cpfactor as oc
    oc.build()
    S, A = gw.nstates, 2 * len(gw.shape)
    # each step: one full oracle VI solve to 1e-6 from zeros (a bounded sample of the step)
    for _ in range(args.warmup):
        oc.value_iteration(gw, tol=TOL, max_iter=5000)
    t0 = time.perf_counter()
    backups = 0
    for _ in range(args.steps):
        _, _, k, _ = oc.value_iteration(gw, tol=TOL, max_iter=5000)
        backups += k * S * A
    el = time.perf_counter() - t0
    value = backups / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict({"step": "CPU FP64 oracle VI solve to 1e-6 from zeros"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oc.threads(), "kind": "oracle",
                             "sample": f"{args.steps} FP64 VI solves of the 64^3 instance ({k} sweeps each)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, rank, world, local, pg):
    import torch
    import paper_2103_00331_gb300 as cp
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    gw = workload(rank)
    S, A = gw.nstates, 2 * len(gw.shape)
    f = cp.build_factors(gw, device=local)
    V = torch.zeros(S, dtype=torch.float32, device=dev)
    Vp = torch.zeros(S, dtype=torch.float32, device=dev)
    pi = torch.zeros(S, dtype=torch.uint8, device=dev)
    pip = torch.zeros(S, dtype=torch.uint8, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    vi_opts = cp.default_opts(tol=TOL, max_iter=5000)
    pi_opts = cp.default_opts(tol=TOL, max_iter=5000)

    # One step: value iteration from V = 0 and policy iteration from V = 0
    # (two zeroed buffers, prepared before the step), each with its FP64
    # certifying sweep. The device time of a step is the sum of the two
    # calls' elapsed_ms: CUDA events the library records on the stream
    # around its own launches, so a host-side stall between a Python event
    # and the library's first launch (GIL, other threads of the process)
    # cannot enter it. The Python-side event bracket is reported beside it.
    def step(ev=None):
        if ev:
            ev[0].record(stream)
        rv = cp.value_iteration(f, cp.F32, V, pi, opts=vi_opts, stream=stream)
        rp = cp.policy_iteration(f, cp.F32, Vp, pip, opts=pi_opts, stream=stream)
        if ev:
            ev[1].record(stream)
        return rv, rp

    for _ in range(max(args.warmup, 0)):
        V.zero_()
        Vp.zero_()
        step()
    torch.cuda.synchronize()
    if pg is not None:
        pg.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    total_ms, py_ms, vi_ms, pi_ms, backups, launches = 0.0, [], [], [], 0, 0
    vi_bytes, pi_bytes, vi_iters, pi_iters = 0, 0, [], []
    for _ in range(args.steps):
        V.zero_()
        Vp.zero_()
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        rv, rp = step(ev)
        torch.cuda.synchronize()
        vi_ms.append(rv["elapsed_ms"])
        pi_ms.append(rp["elapsed_ms"])
        py_ms.append(ev[0].elapsed_time(ev[1]))
        total_ms += rv["elapsed_ms"] + rp["elapsed_ms"]
        backups += rv["backups"] + rp["backups"]
        launches += 4   # persistent VI solve + certify sweep, persistent PI solve + certify sweep
        vi_iters.append(rv["iterations"])
        pi_iters.append(rp["iterations"])
        vi_bytes += rv["iterations"] * S * BYTES_VI
        pi_bytes += rp["eval_sweeps"] * S * BYTES_EVAL + rp["rounds"] * S * BYTES_IMPROVE + S * BYTES_GREEDY
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if pg is not None:
        pg.barrier()
    units, ms_max = aggregate(pg, backups, total_ms, device=dev)
    value = units / (ms_max / 1e3)
    per_step = {"timing": "device time of each step = elapsed_ms of its VI and PI calls (CUDA events the "
                          "library records on the stream around its launches)",
                "vi_ms": step_stats(vi_ms), "pi_ms": step_stats(pi_ms),
                "python_event_bracket_ms": step_stats(py_ms),
                "host_stall_ms_total": sum(py_ms) - total_ms,
                "pi_ms_each": [round(x, 4) for x in pi_ms], "vi_ms_each": [round(x, 4) for x in vi_ms],
                "python_bracket_ms_each": [round(x, 4) for x in py_ms],
                "pi_sweeps_each": pi_iters}

    # plain unfused FP32 VI on the same instance (the comparator of the metric)
    plain_opts = cp.default_opts(tol=TOL, max_iter=5000, fused=0, certify=0)
    plain_ms = []
    rpl = {"iterations": None}
    for i in range(0 if args.skip_plain else max(3, min(args.steps, 10)) + 1):
        V.zero_()
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rpl = cp.value_iteration(f, cp.F32, V, None, opts=plain_opts, stream=stream)
        torch.cuda.synchronize()
        if i > 0:
            plain_ms.append((time.perf_counter() - t0) * 1e3)
    fused_vi_ms = statistics.median(vi_ms)
    plain_vi_ms = statistics.median(plain_ms) if plain_ms else None
    # the same plain kernels with the stopping rule on the device (fused = 3:
    # a recorded 32-sweep graph replayed until the device flag is up), so the
    # gain from fusion is separated from the gain from not syncing every sweep
    plain3_opts = cp.default_opts(tol=TOL, max_iter=5000, fused=3, certify=0)
    plain3_ms = []
    rp3 = {"iterations": None}
    for i in range(0 if args.skip_plain else max(3, min(args.steps, 10)) + 1):
        V.zero_()
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rp3 = cp.value_iteration(f, cp.F32, V, None, opts=plain3_opts, stream=stream)
        torch.cuda.synchronize()
        if i > 0:
            plain3_ms.append((time.perf_counter() - t0) * 1e3)
    plain3_vi_ms = statistics.median(plain3_ms) if plain3_ms else None

    # the same step on the grid-barrier solver (one grid barrier per sweep),
    # for comparison with the barrier-free solver timed above
    gb_opts_vi = cp.default_opts(tol=TOL, max_iter=5000, fused=2)
    gb_opts_pi = cp.default_opts(tol=TOL, max_iter=5000, fused=2)
    gb_vi, gb_pi = [], []
    for i in range(max(3, min(args.steps, 10)) + 1):
        flush.zero_()
        V.zero_()
        Vp.zero_()
        torch.cuda.synchronize()
        gv = cp.value_iteration(f, cp.F32, V, pi, opts=gb_opts_vi, stream=stream)
        gp = cp.policy_iteration(f, cp.F32, Vp, pip, opts=gb_opts_pi, stream=stream)
        torch.cuda.synchronize()
        if i > 0:
            gb_vi.append(gv["elapsed_ms"])
            gb_pi.append(gp["elapsed_ms"])
    grid_barrier = {"kernels": "solve_vi_kernel<float,3,4> / solve_pi_kernel<float,3,4> (fused=2)",
                    "vi_ms": statistics.median(gb_vi), "pi_ms": statistics.median(gb_pi),
                    "vi_sweeps": gv["iterations"], "pi_sweeps": gp["iterations"],
                    "same_sweeps": gv["iterations"] == rv["iterations"] and gp["iterations"] == rp["iterations"]}

    # roofline of the dominant kernel (the persistent policy-iteration kernel,
    # one launch per step): algorithmic bytes of its launches over their
    # event-timed durations; the value-iteration kernel beside it
    hbm = measured_peaks().get("hbm_gbs")
    peak = hbm or 6800.0
    src = "measured (MEASURED_PEAKS.json hbm_gbs)" if hbm else "fallback 6.8 TB/s"
    ach_pi = (pi_bytes / len(pi_ms)) / (statistics.mean(pi_ms) / 1e3) / 1e9
    ach_vi = (vi_bytes / len(vi_ms)) / (statistics.mean(vi_ms) / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": ach_pi, "peak": peak, "unit": "GB/s", "frac": ach_pi / peak,
            "traffic": traffic_from_profile("flow_pi_kernel_gridworld64.txt"),
            "peak_source": src, "kernel": "flow_pi_kernel<3, 2> (barrier-free persistent PI, FP32, columns of two 4-state segments)",
            "algorithmic_bytes_per_launch": pi_bytes / len(pi_ms),
            "note": "64^3 working set (3.4 MB) stays in L2 across sweeps; per-sweep latency bound "
                    "(neighbour values through L2, no grid barrier)"}
    roof_vi = {"bound": "hbm", "achieved": ach_vi, "peak": peak, "unit": "GB/s", "frac": ach_vi / peak,
               "traffic": traffic_from_profile("flow_vi_kernel_gridworld64.txt"),
               "kernel": "flow_vi_kernel<3, 1> (barrier-free persistent VI, FP32)",
               "algorithmic_bytes_per_launch": vi_bytes / len(vi_ms)}

    # HBM-bound sweep: one fused backup of a 512^3 instance, event-timed
    large = None
    p0 = None
    if not args.skip_large:
        large = hbm_sweep(cp, dev, stream, hbm or 6800.0)
        p0 = paper_shaped_solve(cp, dev, stream)
    small = small_10x10(cp, dev, stream)

    dense = None
    if not args.skip_dense:
        dense = dense_measure(cp, dev, stream)

    batch = None
    if not args.skip_batch:
        batch = batch_measure(cp, dev, stream, seed=rank)
    warm = None
    if not args.skip_warmstart:
        warm = warmstart_measure(local)

    # end to end through the public API with host buffers: build_factors
    # (host -> device of the rewards and cell kinds), VI + PI, device -> host
    # of V and the policy after each. The host buffers are pinned and the
    # device value / policy buffers allocated once (as a serving caller keeps
    # them); the copies and the zeroing of V are inside the timed region
    # every step.
    import dataclasses
    rew_h = torch.from_numpy(np.ascontiguousarray(gw.reward, dtype=np.float64).reshape(-1)).pin_memory()
    gw_h = dataclasses.replace(gw, reward=rew_h.numpy().reshape(np.shape(gw.reward)))
    if getattr(gw, "cell", None) is not None:
        cell_h = torch.from_numpy(np.ascontiguousarray(gw.cell, dtype=np.uint8).reshape(-1)).pin_memory()
        gw_h = dataclasses.replace(gw_h, cell=cell_h.numpy().reshape(np.shape(gw.cell)))
    out_h = [(torch.empty(S, dtype=torch.float32).pin_memory(), torch.empty(S, dtype=torch.uint8).pin_memory())
             for _ in range(2)]
    # the caller's device buffers for values and policy, kept across requests
    Ve = torch.empty(S, dtype=torch.float32, device=dev)
    pe = torch.empty(S, dtype=torch.uint8, device=dev)
    e2e_ms = []
    e2e_units = 0
    for i in range(max(2, min(args.steps, 5)) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fe = cp.build_factors(gw_h, device=local)
        with torch.cuda.stream(stream):
            Ve.zero_()
        r1 = cp.value_iteration(fe, cp.F32, Ve, pe, opts=vi_opts, stream=stream)
        with torch.cuda.stream(stream):
            out_h[0][0].copy_(Ve, non_blocking=True)
            out_h[0][1].copy_(pe, non_blocking=True)
            Ve.zero_()
        r2 = cp.policy_iteration(fe, cp.F32, Ve, pe, opts=pi_opts, stream=stream)
        with torch.cuda.stream(stream):
            out_h[1][0].copy_(Ve, non_blocking=True)
            out_h[1][1].copy_(pe, non_blocking=True)
        stream.synchronize()
        fe.close()
        torch.cuda.synchronize()
        if i > 0:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
            e2e_units += r1["backups"] + r2["backups"]
    e2e_total, e2e_max = aggregate(pg, e2e_units, sum(e2e_ms), device=dev)
    e2e = {"value": e2e_total / (e2e_max / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": S * (8 + 1),           # R64 and the cell kinds uploaded by build_factors
           "d2h_bytes_per_step": 2 * S * (4 + 1),       # V and policy after VI and after PI
           "ms_per_step": statistics.median(e2e_ms)}

    cpu = None
    if rank == 0 and world >= 1 and not args.skip_cpu:
        cpu = cpu_oracle_sample(gw, budget_s=args.cpu_seconds)
        small["cpu_oracles"] = small_10x10_cpu()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_dict(), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks,
                "time_to_tol_ms": fused_vi_ms, "plain_fp32_vi_ms": plain_vi_ms,
                "speedup_vs_plain_fp32_vi": plain_vi_ms / fused_vi_ms if plain_vi_ms else None,
                "plain_fp32_vi_device_stop_ms": plain3_vi_ms,
                "speedup_vs_plain_fp32_vi_device_stop": plain3_vi_ms / fused_vi_ms if plain3_vi_ms else None,
                "plain_timing": "host wall clock around the call (host-checked: one residual read per sweep; "
                                "device stop: one flag read per 32 sweeps)",
                "vi_sweeps": statistics.median(vi_iters), "plain_vi_sweeps": rpl["iterations"],
                "plain_device_stop_sweeps": rp3["iterations"],
                "pi_sweeps": statistics.median(pi_iters), "pi_ms": statistics.median(pi_ms),
                "certified_residual": rv["certified_residual"], "error_bound": rv["error_bound"],
                "per_step": per_step, "grid_barrier_solver": grid_barrier, "paper_shaped_1000x1000": p0, "small_10x10": small,
                "hbm_sweep_512": large, "roofline_vi": roof_vi, "dense_64x4": dense, "batch_4096": batch,
                "warmstart_512x64": warm}
        print(json.dumps(line), flush=True)
    f.close()
    return 0


def batch_measure(cp, dev, stream, seed=0, count=4096, reps=3):
    """4096 independent 2-D / 3-D GridWorlds (sides U{8..128} / U{8..48},
    p ~ U(0.6, 0.95), gamma ~ U(0.9, 0.995)) solved to 1e-6 from zeros by one
    batched persistent launch, next to the same instances solved one at a
    time by the fused single-instance solver and by the plain FP32 VI (with
    its stop on the device and host-checked), every instance measured."""
    import torch
    import cpmdp_inputs as ci
    inst = ci.batch_gridworlds(count=count, seed=seed)
    B = cp.batch_build(inst, device=dev.index)
    V = torch.zeros(int(B.total_states), dtype=torch.float32, device=dev)
    opts = cp.default_opts(max_iter=5000)
    r, iters, _ = cp.batch_value_iteration(B, V, opts=opts, stream=stream)   # tunes and records the graph
    times, backups = [], 0
    for _ in range(reps):
        V.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r, iters, res = cp.batch_value_iteration(B, V, opts=opts, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        backups = r["backups"]
    batched_ms = statistics.median(times)
    solver = "shared-memory resident (resident_vi_kernel)" if r["solver"] == cp.SOLVER_BATCH_RESIDENT else \
        "batched kernel (batch_vi_kernel + barrier-free tail)"
    # the global-memory batched kernel with its barrier-free tail (fused = 4)
    # on the same batch, for comparison (same sweeps and values)
    gm_opts = cp.default_opts(max_iter=5000, fused=4)
    cp.batch_value_iteration(B, V, opts=gm_opts, stream=stream)      # tunes and records its graph
    gm_times = []
    for _ in range(reps):
        V.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rg, it_g, _ = cp.batch_value_iteration(B, V, opts=gm_opts, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        gm_times.append(e0.elapsed_time(e1))
    assert np.array_equal(it_g, iters)
    V.zero_()
    r, iters, res = cp.batch_value_iteration(B, V, opts=opts, stream=stream)
    # FP64 certifying sweep of every instance: certified residuals and the
    # FP64 argmax policy (packed like V)
    pol = torch.empty(int(B.total_states), dtype=torch.uint8, device=dev)
    cert_times = []
    cert = None
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        cert = cp.batch_certify(B, V, pol, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        cert_times.append(e0.elapsed_time(e1))
    certify_ms = statistics.median(cert_times)
    gam = np.array([g.gamma for g in inst])
    # one instance at a time, all instances: the fused single-instance solver,
    # the plain kernels with the device-side stop (fused = 3) and the plain
    # host-checked baseline (fused = 0)
    step = 1
    fused_ms, plain3_ms, plain_ms = 0.0, 0.0, 0.0
    popts = cp.default_opts(max_iter=5000, fused=0, certify=0)
    p3opts = cp.default_opts(max_iter=5000, fused=3, certify=0)
    fopts = cp.default_opts(max_iter=5000, certify=0)
    for i in range(count):
        f = cp.build_factors(inst[i], device=dev.index)
        Vi = torch.zeros(inst[i].nstates, dtype=torch.float32, device=dev)
        modes = (("fused", fopts), ("plain3", p3opts)) + ((("plain", popts),) if i % step == 0 else ())
        for mode, o in modes:
            Vi.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            cp.value_iteration(f, cp.F32, Vi, None, opts=o, stream=stream)
            torch.cuda.synchronize()
            dt = (time.perf_counter() - t0) * 1e3
            if mode == "fused":
                fused_ms += dt
            elif mode == "plain3":
                plain3_ms += dt
            else:
                plain_ms += dt
        f.close()
    B.close()
    # algorithmic bytes: every sweep of every instance reads V, R, code and
    # writes V' (13 B per state); the floor takes each global sweep at the
    # larger of its bytes at the measured HBM peak and the single-instance
    # solver's per-sweep latency (2.5 us at 64^3)
    sizes = np.array([g.nstates for g in inst], dtype=np.float64)
    sweeps = np.asarray(iters, dtype=np.int64)
    alg_bytes = float((sweeps * sizes).sum() * 13.0)
    peak = measured_peaks().get("hbm_gbs") or 6800.0
    order = np.argsort(sweeps)
    active = np.concatenate([[sizes.sum()], sizes.sum() - np.cumsum(sizes[order])])
    floor_ms = 0.0
    prev = 0
    for j, idx in enumerate(order):
        n = int(sweeps[idx]) - prev
        if n > 0:
            floor_ms += n * max(active[j] * 13.0 / (peak * 1e9) * 1e3, 2.5e-3)
            prev = int(sweeps[idx])
    return {"instances": count, "states": int(inst_states(inst)), "backups": int(backups), "solver": solver,
            "algorithmic_bytes": alg_bytes, "achieved_gbs": alg_bytes / (batched_ms * 1e6),
            "hbm_frac": alg_bytes / (batched_ms * 1e6) / peak, "model_floor_ms": floor_ms,
            "hbm_frac_note": "algorithmic bytes (13 B per state and sweep) / time; the resident solver keeps the "
                             "values in shared memory, so this is an effective rate (its bound is the ALU pipe)",
            "batched_ms": batched_ms, "batched_backups_per_s": backups / (batched_ms / 1e3),
            "global_memory_batched_kernel_ms": statistics.median(gm_times),
            "launch_sweeps": r["iterations"], "max_instance_sweeps": int(iters.max()),
            "graph_replay": bool(r["rounds"] == 1),
            "certify_ms": certify_ms, "batched_with_certify_ms": batched_ms + certify_ms,
            "max_certified_residual": float(cert.max()),
            "max_error_bound": float((cert / (1 - gam)).max()),
            "one_at_a_time_fused_ms": fused_ms, "plain_fp32_vi_device_stop_ms": plain3_ms,
            "plain_fp32_vi_ms": plain_ms,
            "speedup_vs_plain_fp32_vi_device_stop": plain3_ms / batched_ms,
            "speedup_vs_plain_fp32_vi": plain_ms / batched_ms,
            "note": f"one-at-a-time fused, device-stop plain and host-checked plain measured on all {count} "
                    f"instances (host wall clock per call)"}


def dense_measure(cp, dev, stream, reps=2):
    """Config 3: the 4-D dense CP model 64^4 (16.8M states, 8 actions, rank
    8, factor rows U(0,1) normalised, R ~ N(0,1), gamma = 0.95). Value
    iteration from V = 0 with BF16x3 tensor-core sweeps (defect correction
    against FP32 base expectations) until the FP64 residual max |T(V) - V| is
    below 1e-6, FP64 certifying sweeps and the FP64 argmax policy included;
    one BF16x3 sweep alone (tcgen05 passes) for the tensor roofline; one FP64
    sweep; the FP32 SIMT mode-product value iteration (residual read by the
    host each sweep) as the plain comparator; and the error against the FP64
    oracle's own value iteration at its 4096 stored sample states."""
    import torch
    import cpmdp_inputs as ci
    dc = ci.config_dense_4d(side=64, seed=0)
    f = cp.build_factors(dc, device=dev.index)
    S, A, Rk = dc.nstates, dc.nactions, dc.rank
    V = torch.zeros(S, dtype=torch.float32, device=dev)
    pi = torch.zeros(S, dtype=torch.uint8, device=dev)
    opts = cp.default_opts(tol=TOL, max_iter=1000)
    r = cp.value_iteration(f, cp.BF16X3, V, pi, opts=opts, stream=stream)   # warm-up: tiles, buffers
    times = []
    for _ in range(reps):
        V.zero_()
        torch.cuda.synchronize()
        r = cp.value_iteration(f, cp.BF16X3, V, pi, opts=opts, stream=stream)
        times.append(r["elapsed_ms"])
    solve_ms = statistics.median(times)

    def timed(fn, n=4):
        ts = []
        for i in range(n):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            if i:
                ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    Vb = torch.empty_like(V)
    sweep_ms = timed(lambda: cp.bellman_backup(f, cp.BF16X3, V, Vb, None, None, stream=stream))
    Vd = V.double()
    Wd = torch.empty_like(Vd)
    fp64_ms = timed(lambda: cp.bellman_backup(f, cp.F64, Vd, Wd, None, None, stream=stream), n=2)
    del Vd, Wd
    flops = 2.0 * 64 * 4 * S * A * Rk            # method flops per sweep (4 mode products per chain)
    pk = measured_peaks()
    bf16 = pk.get("bf16_tflops")
    peak = bf16 or 1900.0
    ach = flops / (sweep_ms * 1e9)
    roof = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "peak_source": "measured bf16 burst (MEASURED_PEAKS.json)" if bf16 else "fallback 1.9 PFLOP/s",
            "kernel": "dense_pass_a + dense_pass_b (BF16x3 tcgen05 sweep)",
            "flops_per_sweep": flops, "issued_bf16_tflops": 3 * ach, "issued_frac": 3 * ach / peak,
            "note": "achieved counts the method's FP32-equivalent flops (2 R D N per state-action); "
                    "BF16x3 issues three bf16 products for each"}
    # policy iteration on the tensor cores (BF16x3 evaluation sweeps, modified
    # policy iteration, FP64 certificate of the result)
    Vq = torch.zeros_like(V)
    piq = torch.zeros_like(pi)
    torch.cuda.synchronize()
    rq = cp.policy_iteration(f, cp.BF16X3, Vq, piq, opts=opts, stream=stream)
    pi_line = {"time_ms": rq["elapsed_ms"], "rounds": rq["rounds"], "eval_sweeps": rq["eval_sweeps"],
               "sweeps": rq["iterations"], "certified_residual": rq["certified_residual"],
               "error_bound": rq["error_bound"], "backups_per_s": rq["backups"] / (rq["elapsed_ms"] / 1e3)}
    del Vq, piq
    # plain comparator: FP32 SIMT mode products, residual read back each sweep
    Vp = torch.zeros_like(V)
    torch.cuda.synchronize()
    rp = cp.value_iteration(f, cp.F32, Vp, None, opts=cp.default_opts(tol=TOL, max_iter=1000, certify=0),
                            stream=stream)
    out = {"workload": "dense-cp-64^4-A8-R8-gamma0.95 (config 3)", "states": S, "actions": A, "rank": Rk,
           "time_to_tol_ms": solve_ms, "sweeps": r["iterations"], "rebases": r["rounds"],
           "fp64_certify_sweeps": r["eval_sweeps"], "residual": r["residual"],
           "certified_residual": r["certified_residual"], "error_bound": r["error_bound"],
           "backups_per_s": r["backups"] / (solve_ms / 1e3), "bf16x3_sweep_ms": sweep_ms,
           "fp64_sweep_ms": fp64_ms, "fp64_tflops": flops / (fp64_ms * 1e9),
           "fp64_frac_of_nominal_1.25": flops / (fp64_ms * 1e9) / 1.25, "roofline": roof,
           "policy_iteration_bf16x3": pi_line,
           "plain_fp32_simt_vi_ms": rp["elapsed_ms"], "plain_fp32_simt_vi_sweeps": rp["iterations"],
           "speedup_vs_plain_fp32_vi": rp["elapsed_ms"] / solve_ms}
    del Vp
    gold = os.path.join(ROOT, "tests", "golden", "dense64_vi_samples.npz")
    if os.path.exists(gold):
        g = np.load(gold)
        idx = torch.as_tensor(g["state"], device=dev)
        got = V[idx].double().cpu().numpy()
        gp = pi[idx].cpu().numpy()
        err = float(np.abs(got - g["value"]).max())
        bound = r["error_bound"] + float(g["certified_residual"]) / (1 - dc.gamma)
        sure = g["gap"] > 2 * dc.gamma * bound
        out["vs_fp64_oracle_vi"] = {"samples": int(len(idx)), "max_abs_diff": err,
                                    "max_rel_diff": err / float(g["max_abs_value"]),
                                    "oracle_sweeps": int(g["sweeps"]),
                                    "policy_equal_where_gap_exceeds_bound": int((gp[sure] == g["policy"][sure]).sum()),
                                    "policy_compared": int(sure.sum())}
    f.close()
    torch.cuda.empty_cache()
    return out


def warmstart_measure(device_index):
    """Config 5: the committed network (trained on 20,000 solved 32^3
    instances) warm-starts batched value iteration on 512 held-out 64^3
    instances; zero initialisation on the same instances beside it."""
    from paper_2103_00331_gb300 import warmstart as ws
    path = os.path.join(ROOT, "paper_2103_00331_gb300", "data", "warmstart_weights.npz")
    if not os.path.exists(path):
        return None
    net = ws.WarmStartNet.load(path, device=device_index)
    return ws.evaluate(net, count=512, side=64)


def step_stats(xs):
    """min / median / mean / max of per-step times (ms)."""
    return {"min": min(xs), "median": statistics.median(xs), "mean": statistics.mean(xs), "max": max(xs)}


def measured_peaks():
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(pk)) if os.path.exists(pk) else {}


def inst_states(inst):
    return sum(g.nstates for g in inst)


def paper_shaped_solve(cp, dev, stream):
    """Context only: the paper's largest 2-D GridWorld shape (1000 x 1000,
    4 actions, 22 absorbing cells of reward +100 / -100, about 800
    obstacles, step reward -3, gamma = 0.9, at most 1000 sweeps), solved by
    value iteration to 1e-6 in FP64 from zeros (grid-barrier solver: the
    grid is past the barrier-free solver's size). The paper's own time for
    this shape was taken on a CPU in Python; it is quoted as context, not
    as a baseline."""
    import torch
    import cpmdp_inputs as ci
    goals = [100.0 if i % 2 == 0 else -100.0 for i in range(22)]
    gw = ci.gridworld((1000, 1000), p=0.8, gamma=0.9, step_reward=-3.0, goal_rewards=goals,
                      obstacle_rate=800 / 1e6, seed=11)
    f = cp.build_factors(gw, device=dev.index)
    V = torch.zeros(gw.nstates, dtype=torch.float64, device=dev)
    pi = torch.zeros(gw.nstates, dtype=torch.uint8, device=dev)
    opts = cp.default_opts(tol=TOL, max_iter=1000)
    times = []
    r = None
    for i in range(4):
        V.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = cp.value_iteration(f, cp.F64, V, pi, opts=opts, stream=stream, raise_on_noconv=False)
        e1.record(stream)
        torch.cuda.synchronize()
        if i > 0:
            times.append(e0.elapsed_time(e1))
    f.close()
    return {"states": gw.nstates, "obstacles": int((gw.cell == ci.OBSTACLE).sum()), "terminals": 22,
            "precision": "f64", "sweeps": r["iterations"], "converged": r["status"] == cp.OK,
            "ms": statistics.median(times), "solver": r["solver"],
            "paper_context": "2,140.34 s for CP-MDP VI on this shape, CPU, Python (paper's runtime table)"}


def small_10x10(cp, dev, stream):
    """The 10 x 10 GridWorld (4 actions, p = 0.8 with 0.1 slips, step -0.04,
    +1 / -1 terminals, gamma = 0.9): FP64 value iteration to 1e-6 and FP64
    policy iteration from zeros on the GPU, one persistent launch each
    (100 states: latency bound), CUDA events, median of 10 after warm-up."""
    import torch
    import cpmdp_inputs as ci
    gw = ci.config_small_2d(0)
    f = cp.build_factors(gw, device=dev.index)
    V = torch.zeros(gw.nstates, dtype=torch.float64, device=dev)
    pi = torch.zeros(gw.nstates, dtype=torch.uint8, device=dev)
    opts = cp.default_opts(tol=TOL, max_iter=1000)
    out = {"states": gw.nstates, "actions": 4, "precision": "f64"}
    for mode in ("vi", "pi"):
        times, r = [], None
        for i in range(11):
            V.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if mode == "vi":
                r = cp.value_iteration(f, cp.F64, V, pi, opts=opts, stream=stream)
            else:
                r = cp.policy_iteration(f, cp.F64, V, pi, opts=opts, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            if i > 0:
                times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        out[mode] = {"ms": ms, "sweeps": r["iterations"], "backups_per_s": r["backups"] / (ms / 1e3)}
    f.close()
    return out


def small_10x10_cpu(reps=20):
    """The same 10 x 10 solves by the oracles as they stand: the tabular FP64
    oracle (numpy, P expanded from the GridWorld rules; VI and PI with exact
    evaluation) and the CP-factor C oracle (FP64 VI) on all host cores and on
    one core."""
    import cpmdp_inputs as ci
    from oracle import cpfactor as oc
    from oracle import tabular as tb
    gw = ci.config_small_2d(0)
    P = tb.transition_tabular(gw.shape, gw.cell, gw.p)
    R = gw.reward.reshape(-1)

    def timed(fn):
        fn()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        return (time.perf_counter() - t0) * 1e3 / reps

    oc.build()
    out = {"tabular_vi_ms": timed(lambda: tb.value_iteration(P, R, gw.gamma, gw.cell, tol=TOL)),
           "tabular_pi_ms": timed(lambda: tb.policy_iteration(P, R, gw.gamma, gw.cell)),
           "cp_factor_vi_ms": timed(lambda: oc.value_iteration(gw, tol=TOL, max_iter=1000)),
           "cp_factor_threads": oc.threads()}
    nthreads = oc.threads()
    oc.set_threads(1)
    try:
        out["cp_factor_vi_ms_one_core"] = timed(lambda: oc.value_iteration(gw, tol=TOL, max_iter=1000))
    finally:
        oc.set_threads(nthreads)
    return out


def hbm_sweep(cp, dev, stream, peak):
    """One fused FP32 backup sweep of a 512^3 GridWorld (134M states, out of
    L2): algorithmic bytes (13 per state) over the event-timed duration."""
    import torch
    import cpmdp_inputs as ci
    n = 512
    gw = ci.gridworld((n, n, n), p=0.8, gamma=0.99, step_reward=-0.01,
                      goal_rewards=list(ci.uniform(0, 12, 8, 0.5, 1.0)), obstacle_rate=0.05, seed=2)
    f = cp.build_factors(gw, device=dev.index)
    S = gw.nstates
    Va = torch.zeros(S, dtype=torch.float32, device=dev)
    Vb = torch.zeros(S, dtype=torch.float32, device=dev)
    res = torch.zeros(1, dtype=torch.float64, device=dev)
    times = []
    for i in range(13):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cp.bellman_backup(f, cp.F32, Va, Vb, None, res, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= 3:
            times.append(e0.elapsed_time(e1))
        Va, Vb = Vb, Va
    ms = statistics.median(times)
    ach = S * BYTES_VI / (ms / 1e3) / 1e9
    # value iteration of the same instance from zeros to max|dV| < 1e-6:
    # marching sweeps from a replayed CUDA graph with the stop decided on the
    # device (fused = 1), and the grid-barrier persistent solver (fused = 2);
    # library-recorded CUDA events, second of two runs (the first records the graph)
    solves = {}
    for fused in (1, 2):
        r = None
        for _ in range(2):
            Va.zero_()
            torch.cuda.synchronize()
            r = cp.value_iteration(f, cp.F32, Va, None, opts=cp.default_opts(tol=TOL, max_iter=5000, fused=fused,
                                                                               certify=0), stream=stream)
        gbs = r["iterations"] * S * BYTES_VI / (r["elapsed_ms"] / 1e3) / 1e9
        solves["march_graph" if fused == 1 else "grid_barrier"] = {
            "time_to_tol_ms": r["elapsed_ms"], "sweeps": r["iterations"], "achieved_gbs": gbs, "frac": gbs / peak,
            "solver": r["solver"], "backups_per_s": r["backups"] / (r["elapsed_ms"] / 1e3)}
    f.close()
    del Va, Vb
    torch.cuda.empty_cache()
    return {"kernel": "march_kernel<float,false> (plane-marching fused backup)", "states": S, "ms": ms,
            "bytes_per_state": BYTES_VI, "achieved_gbs": ach, "peak_gbs": peak, "frac": ach / peak,
            "traffic": traffic_from_profile("march_kernel_gridworld320.txt", scale=S),
            "solve_to_1e-6": solves,
            "note": "inputs 1.7 GB > L2; residual fused, policy not written; traffic scaled from a 320^3 capture; "
                    "solve frac = algorithmic bytes (13 per state and sweep) over the solve's time"}


def kernel_case(name, reps=3):
    """Run one kernel workload a few times and exit (for ncu captures):
    sweep512 / sweep320 = fused FP32 backup of a 512^3 / 320^3 GridWorld; dense64 / dense64f64 = one
    FP32 / FP64 SIMT sweep of the 64^4 dense CP model; dense64tc = one BF16x3 tensor-core sweep of it;
    solve64 / pi64 = fused
    FP32 value / policy iteration of the 64^3 instance (barrier-free solver);
    solve64b / pi64b = the same on the grid-barrier solver; ws512 = the warm-start network on
    512 x 16^3 coarse cells (six tensor-core convolutions); batch1024 = batched value iteration of
    1024 uneven GridWorlds (batched kernel, then the barrier-free tail); batch4096 = the 4096-instance
    batch, shared-memory-resident solver (fused=1) and batched kernel with tail (fused=4); batchres1024 = the
    resident solver on 1024 instances; batchcert = the FP64
    certifying sweep of that batch after its solve."""
    import torch
    import paper_2103_00331_gb300 as cp
    import cpmdp_inputs as ci
    dev = torch.device("cuda", 0)
    if name in ("sweep512", "sweep320"):
        n = int(name[5:])
        gw = ci.gridworld((n, n, n), p=0.8, gamma=0.99, step_reward=-0.01,
                          goal_rewards=list(ci.uniform(0, 12, 8, 0.5, 1.0)), obstacle_rate=0.05, seed=2)
        f = cp.build_factors(gw, device=0)
        Va = torch.zeros(gw.nstates, dtype=torch.float32, device=dev)
        Vb = torch.zeros_like(Va)
        res = torch.zeros(1, dtype=torch.float64, device=dev)
        for _ in range(reps):
            cp.bellman_backup(f, cp.F32, Va, Vb, None, res)
            Va, Vb = Vb, Va
    elif name == "dense64tc":
        dc = ci.config_dense_4d(side=64, seed=0)
        f = cp.build_factors(dc, device=0)
        Va = torch.as_tensor(ci.random_values(dc.shape, seed=2).reshape(-1).astype(np.float32)).to(dev)
        Vb = torch.empty_like(Va)
        res = torch.zeros(1, dtype=torch.float64, device=dev)
        for i in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            cp.bellman_backup(f, cp.BF16X3, Va, Vb, None, res)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            flops = 2.0 * 64 * 4 * dc.nstates * dc.nactions * dc.rank
            print(f"dense 64^4 BF16x3 tcgen05 sweep: {ms:.3f} ms, {flops / ms / 1e9:.1f} TFLOP/s (FP32-equivalent), "
                  f"{3 * flops / ms / 1e9:.1f} TFLOP/s bf16")
            Va, Vb = Vb, Va
    elif name == "dense64f64":
        dc = ci.config_dense_4d(side=64, seed=0)
        f = cp.build_factors(dc, device=0)
        Va = torch.as_tensor(ci.random_values(dc.shape, seed=2).reshape(-1)).to(dev)
        Vb = torch.empty_like(Va)
        res = torch.zeros(1, dtype=torch.float64, device=dev)
        for i in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            cp.bellman_backup(f, cp.F64, Va, Vb, None, res)
            e1.record()
            torch.cuda.synchronize()
            flops = 2.0 * 64 * 4 * dc.nstates * dc.nactions * dc.rank
            print(f"dense 64^4 FP64 SIMT sweep: {e0.elapsed_time(e1):.3f} ms, {flops / e0.elapsed_time(e1) / 1e9:.3f} TFLOP/s")
            Va, Vb = Vb, Va
    elif name == "dense64":
        dc = ci.config_dense_4d(side=64, seed=0)
        f = cp.build_factors(dc, device=0)
        Va = torch.as_tensor(ci.random_values(dc.shape, seed=2).reshape(-1).astype(np.float32)).to(dev)
        Vb = torch.empty_like(Va)
        res = torch.zeros(1, dtype=torch.float64, device=dev)
        for i in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            cp.bellman_backup(f, cp.F32, Va, Vb, None, res)
            e1.record()
            torch.cuda.synchronize()
            print(f"dense 64^4 FP32 SIMT sweep: {e0.elapsed_time(e1):.3f} ms")
            Va, Vb = Vb, Va
    elif name == "batch4096":
        inst = ci.batch_gridworlds(count=4096, seed=0)
        B = cp.batch_build(inst, device=0)
        V = torch.zeros(int(B.total_states), dtype=torch.float32, device=dev)
        for fused in (1, 4, 1):
            opts = cp.default_opts(tol=TOL, max_iter=5000, fused=fused)
            for _ in range(reps):
                V.zero_()
                r, iters, _ = cp.batch_value_iteration(B, V, opts=opts)
                print(f"batch of 4096, fused={fused}: {r['elapsed_ms']:.3f} ms, {r['iterations']} sweeps, "
                      f"solver {r['solver']}")
        B.close()
    elif name == "batchres1024":
        inst = ci.batch_gridworlds(count=1024, seed=0)
        B = cp.batch_build(inst, device=0)
        V = torch.zeros(int(B.total_states), dtype=torch.float32, device=dev)
        opts = cp.default_opts(tol=TOL, max_iter=5000)
        for _ in range(reps):
            V.zero_()
            r, iters, _ = cp.batch_value_iteration(B, V, opts=opts)
            print(f"batch of 1024, resident: {r['elapsed_ms']:.3f} ms, {r['iterations']} sweeps, solver {r['solver']}")
        B.close()
    elif name == "batch1024":
        inst = ci.batch_gridworlds(count=1024, seed=0)
        B = cp.batch_build(inst, device=0)
        V = torch.zeros(int(B.total_states), dtype=torch.float32, device=dev)
        opts = cp.default_opts(tol=TOL, max_iter=5000, fused=4)
        for _ in range(reps):
            V.zero_()
            r, iters, _ = cp.batch_value_iteration(B, V, opts=opts)
            print(f"batch of 1024: {r['elapsed_ms']:.3f} ms, {r['iterations']} sweeps, tail from sweep {r['tail_from']}")
        B.close()
    elif name == "batchcert":
        inst = ci.batch_gridworlds(count=1024, seed=0)
        B = cp.batch_build(inst, device=0)
        V = torch.zeros(int(B.total_states), dtype=torch.float32, device=dev)
        pol = torch.empty(int(B.total_states), dtype=torch.uint8, device=dev)
        cp.batch_value_iteration(B, V, opts=cp.default_opts(tol=TOL, max_iter=5000))
        for _ in range(reps):
            cert = cp.batch_certify(B, V, pol)
        print(f"batch certify of 1024 instances: max certified residual {cert.max():.3e}")
        B.close()
    elif name == "ws512":
        from paper_2103_00331_gb300 import warmstart as ws
        # six layers with dilations up to 4 (random weights: the time does not depend on them)
        net = ws.WarmStartNet(device=0, seed=0, dilations=(1, 2, 4, 2, 1, 1))
        dims = (512, 16, 16, 16)
        nv = int(np.prod(dims))
        feat = torch.zeros((nv, 64), dtype=torch.bfloat16, device=dev)
        feat[:, :net.n_feat] = torch.as_tensor(ci.random_values((nv, net.n_feat), seed=5).astype(np.float32)).to(dev)
        for i in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            net.predict(feat, dims)
            e1.record()
            ws.ws_sync()
            flops = 2.0 * nv * 27 * 64 * 64 * net.layers
            print(f"warm-start network, 512 x 16^3 coarse cells: {e0.elapsed_time(e1):.3f} ms, "
                  f"{flops / e0.elapsed_time(e1) / 1e9:.1f} TFLOP/s bf16 (tcgen05 convolutions)")
    elif name in ("solve64", "pi64", "solve64b", "pi64b"):
        gw = workload(0)
        fused = 2 if name.endswith("b") else 1
        f = cp.build_factors(gw, device=0)
        V = torch.zeros(gw.nstates, dtype=torch.float32, device=dev)
        pi = torch.zeros(gw.nstates, dtype=torch.uint8, device=dev)
        for _ in range(reps):
            V.zero_()
            if name.startswith("solve64"):
                cp.value_iteration(f, cp.F32, V, None, opts=cp.default_opts(max_iter=5000, certify=0, fused=fused))
            else:
                cp.policy_iteration(f, cp.F32, V, pi, opts=cp.default_opts(max_iter=5000, certify=0, fused=fused))
    else:
        raise SystemExit(f"unknown kernel case {name}")
    torch.cuda.synchronize()
    print(f"kernel case {name}: ok")
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--skip-large", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--skip-dense", action="store_true")
    ap.add_argument("--skip-warmstart", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--kernel-case", choices=["sweep512", "sweep320", "solve64", "pi64", "solve64b", "pi64b", "dense64", "dense64f64", "batch4096", "batchres1024",
                                              "dense64tc", "ws512", "batch1024", "batchcert"],
                    default=None,
                    help="run one kernel workload a few times (profiling) and exit")
    args = ap.parse_args()
    if args.kernel_case:
        return kernel_case(args.kernel_case)
    rank, world, local, pg = dist_setup(args.gpus)
    if args.impl == "reference":
        rc = run_reference(args, rank, world)
    else:
        rc = run_ours(args, rank, world, local, pg)
    if pg is not None:
        pg.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
