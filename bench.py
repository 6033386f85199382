"""Throughput of the forward-Euler step on GB300: lattice-site updates per second (GLUPS)
and the fraction of the measured HBM roofline.

Default workload: 3D Gray-Scott, periodic 256^3, two fields, h = 1, Du = 0.2, Dv = 0.1,
F = 0.04, k = 0.06, dt = 0.5, 7-point Laplacian, u = 1, v = 0 with 20 seeded 8^3 cubes
(u = 0.5, v = 0.25) and 1 % multiplicative noise.  One bench "step" = ``--substeps``
forward-Euler time steps of the whole grid (pf_step).  The state (2 fields x 2 copies x
64 MiB = 268 MB) is larger than the 129 MB L2, so no flush is needed between iterations.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pf|reference]
Under torchrun every rank runs its own replica (weak scaling, no data-path collective);
rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synthetic  # noqa: E402

METRIC = "lattice-site updates/s (GLUPS), % of measured HBM roofline"
UNIT = "GLUPS"
WORKLOAD = "gs3d_256"
BYTES_PER_LUP = {"gs": 16.0, "ac": 8.0, "ch": 8.0}  # k = 1: read + write every field once
TMA_TILES = {(64, 16), (128, 8), (128, 16)}
# Three coupled species (D, exponents E, rates K): a constant source, linear, quadratic,
# cubic and mixed monomials
RD3 = ((0.2, 0.05, 0.12),
       [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 2, 0], [2, 0, 1], [0, 0, 3]],
       [[0.03, -0.03, 0.0, 0.1, -1.0, 0.0, 0.0], [0.0, 0.0, -0.09, 0.0, 1.0, -0.4, 0.0],
        [0.0, 0.05, 0.0, -0.2, 0.0, 0.4, -0.3]])
# DRAM bytes (read + write) per launch from one ncu capture of each kernel as it is now
# (profiles/fe3d_tb2_gs3d_256.md, profiles/fe3d_tma_gs3d_256.md); reported only for that
# kernel and tile.
PROFILED_TRAFFIC = {("fe3d_tb2_kernel", 256, 8, 2): 224.83e6,
                    ("fe3d_tma_kernel", 64, 16, 1): 216.9e6}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ distributed plumbing

def _dist_init(use_cuda: bool):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if use_cuda else "gloo")
    return rank, world, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clock sampling

class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return self
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ oracle baseline

def _oracle_worker(conn, name):
    """One host process stepping its own copy of a workload with the oracle, on command:
    ("step", n) advances n steps and replies with the seconds taken; anything else ends it."""
    import oracle
    w = synthetic.WORKLOADS[name]
    x = tuple(a.astype(np.float64) for a in synthetic.workload_init(name))
    conn.send(("ready", x[0].size))
    while True:
        msg = conn.recv()
        if not (isinstance(msg, tuple) and msg[0] == "step"):
            break
        t0 = time.perf_counter()
        for _ in range(msg[1]):
            x = oracle.euler_step(w["model"], x, w["coeffs"], w["dt"], w["h"])
        conn.send(("done", time.perf_counter() - t0))
    conn.close()


class OracleWorkers:
    """``n`` spawned processes (this process may already hold a CUDA context, so no fork),
    each with its own copy of the workload: the oracle as it stands, run on ``n`` host cores
    at once. ``step(k)`` advances every copy k steps and returns the wall time of the round."""

    def __init__(self, n: int, name: str = WORKLOAD):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for _ in range(n):
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(b, name), daemon=True)
            p.start()
            self.conns.append(a)
            self.procs.append(p)
        self.sites = [c.recv()[1] for c in self.conns][0]

    def step(self, k: int) -> float:
        t0 = time.perf_counter()
        for c in self.conns:
            c.send(("step", k))
        for c in self.conns:
            c.recv()
        return time.perf_counter() - t0

    def close(self):
        for c in self.conns:
            try:
                c.send(("stop",))
            except (BrokenPipeError, OSError):
                pass
        for p in self.procs:
            p.join(timeout=30)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(budget_s: float = 12.0):
    """The FP64 oracle, as it stands, on the host: the full 256^3 grid, one step at a time,
    first in one process (``budget_s`` / 2 of time, at least one step), then in one process
    per host core, each stepping its own copy (rounds until ``budget_s`` / 2 has elapsed, at
    least one round). Both are reported; ``value`` and ``cores`` are the all-core figure."""
    import oracle
    w = synthetic.WORKLOADS[WORKLOAD]
    x = tuple(a.astype(np.float64) for a in synthetic.workload_init(WORKLOAD))
    sites = x[0].size
    n, t0 = 0, time.perf_counter()
    while True:
        x = oracle.euler_step(w["model"], x, w["coeffs"], w["dt"], w["h"])
        n += 1
        if time.perf_counter() - t0 >= budget_s / 2:
            break
    dt1 = time.perf_counter() - t0
    single = sites * n / dt1 / 1e9
    cores = host_cores()
    pool = OracleWorkers(cores)
    try:
        pool.step(1)  # warm-up round (first touches of every copy's arrays)
        rounds, total = 0, 0.0
        while total < budget_s / 2 or rounds == 0:
            total += pool.step(1)
            rounds += 1
    finally:
        pool.close()
    multi = sites * cores * rounds / total / 1e9
    return {"value": multi, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_core": {"value": single, "cores": 1,
                            "sample": f"{n} FP64 numpy step(s) of the full 256^3 Gray-Scott "
                                      f"grid in one process ({dt1:.1f} s)"},
            "sample": f"{cores} processes (one per host core), each stepping its own copy of "
                      f"the full 256^3 Gray-Scott grid with the FP64 numpy oracle: {rounds} "
                      f"timed round(s) of one step each ({total:.1f} s) after one untimed "
                      f"round; single-process figure under single_core"}


def run_reference(args, rank, world):
    """The reference arm: the oracle as it stands on every host core (one process per core,
    each stepping its own copy of the full 256^3 grid); one bench step = one oracle step of
    every copy."""
    if rank != 0:
        return
    cores = host_cores()
    pool = OracleWorkers(cores)
    try:
        for _ in range(args.warmup):
            pool.step(1)
        dt = sum(pool.step(1) for _ in range(args.steps))
    finally:
        pool.close()
    sites = pool.sites
    value = sites * cores * args.steps / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "gs3d_256: 3D Gray-Scott 256^3 periodic, 2 fields, dt=0.5, "
                               f"one bench step = 1 forward-Euler step of each of {cores} "
                               "copies (oracle, one process per host core)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} timed rounds; each round one FP64 numpy "
                                   f"step of the full 256^3 grid in each of {cores} processes"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm

def run_gpu(args, rank, world, local):
    import torch
    import paper_2109_02598_gb300 as pf

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    w = synthetic.WORKLOADS[WORKLOAD]
    x0 = synthetic.workload_init(WORKLOAD)
    sites = x0[0].size
    S = args.substeps
    with torch.cuda.stream(stream):
        g = pf.Grid(x0[0].shape, 2, w["h"], stream=stream).set_model(w["model"], w["coeffs"], w["dt"])
        g.write_fields(x0)
        tuning = g.autotune(5)  # the fastest tile on this GPU (state unchanged)
        launches_per_step = sum(1 for _ in _launch_schedule(S, tuning[2]))

        # ---- device-resident timing
        for _ in range(args.warmup):
            g.step(S)
        g.synchronize()
        _barrier(world)
        sampler = ClockSampler(local).start() if rank == 0 else None
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            g.step(S)
        ev1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        ms = ev0.elapsed_time(ev1)
        ms = _max_over_ranks(ms, world, dev)
        _barrier(world)

        # ---- end to end through the public API: every job uploads its fields from pinned
        # host memory, runs its steps and downloads its result. Jobs alternate between two
        # grids on two streams with the non-waiting host copies, so one job's copies overlap
        # the other's steps, as a caller that pipelines jobs runs them. A job's steps wait
        # for the previous job's steps (an event across the streams): each launch spans
        # every SM, and two grids' launches sharing the SMs would break the lock-step over z
        # that keeps neighbouring tiles' halo rows in L2. The timed region holds every copy
        # and every step of args.steps jobs.
        stream2 = torch.cuda.Stream(device=dev)
        g2 = pf.Grid(x0[0].shape, 2, w["h"], stream=stream2).set_model(
            w["model"], w["coeffs"], w["dt"])
        g2.set_tuning(*tuning)
        grids = [g, g2]
        streams = [stream, stream2]
        host_in = [torch.from_numpy(a).pin_memory() for a in x0]
        host_out = [[torch.empty_like(h).pin_memory() for h in host_in] for _ in range(2)]
        last_steps = [None]

        def job(j):
            gg, st = grids[j % 2], streams[j % 2]
            for i, h in enumerate(host_in):
                gg.write_field_async(i, h)
            if last_steps[0] is not None:
                st.wait_event(last_steps[0])
            gg.step(S)
            last_steps[0] = torch.cuda.Event()
            last_steps[0].record(st)
            for i, h in enumerate(host_out[j % 2]):
                gg.read_field_async(i, h)

        for j in range(max(2, args.warmup)):  # records both grids' step graphs
            job(j)
        for gg in grids:
            gg.synchronize()
        torch.cuda.synchronize()
        _barrier(world)
        t0 = time.perf_counter()
        for j in range(args.steps):
            job(j)
        for gg in grids:
            gg.synchronize()
        torch.cuda.synchronize()
        e2e_s = _max_over_ranks(time.perf_counter() - t0, world, dev)
        g2.close()
        g.close()

    multi = None
    if world > 1 and not args.no_companions:
        try:
            multi = multi_rank_companions(stream, rank, world, dev)
        except Exception as exc:  # reported in the line, never fatal for the headline
            multi = {"error": f"{type(exc).__name__}: {exc}"}
    if rank != 0:
        return
    hbm, peak_kind = _peaks()
    if tuning[2] == 2:
        kernel_name = "fe3d_tb2_kernel (TMA-staged z-streaming, 2 time steps per pass, 7-point GS)"
    elif tuple(tuning[:2]) in TMA_TILES:
        kernel_name = "fe3d_tma_kernel (TMA-staged z-streaming, 7-point GS)"
    else:
        kernel_name = "fe3d_r1_kernel (general z-streaming, 7-point GS)"
    n_launch = args.steps * launches_per_step
    lups = sites * S * args.steps * world
    value = lups / (ms * 1e-3) / 1e9
    launch_ms = ms / n_launch  # every launch of the plan does k steps (S is a multiple of k)
    k = tuning[2]
    # per launch: k steps of every site at the k = 1 algorithmic 16 B/LUP (the figure can
    # exceed the HBM peak when k > 1, since a depth-k launch moves each field once for k steps)
    alg_bytes = BYTES_PER_LUP[w["model"]] * sites * k
    achieved = alg_bytes / (launch_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "gs3d_256: 3D Gray-Scott 256^3 periodic, 2 fields, Du=0.2 Dv=0.1 "
                               "F=0.04 k=0.06 dt=0.5 h=1, 7-point Laplacian, 20 seeded 8^3 cubes "
                               "+ 1% noise",
                   "substeps_per_step": S, "tile": list(tuning[:2]), "k": k,
                   "l2": "inputs larger than L2 (268 MB ping-pong state vs 129 MB L2)",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm,
                     "peak_kind": f"{peak_kind} (copy, MEASURED_PEAKS.json hbm_gbs)"
                     if peak_kind == "measured" else "fallback",
                     "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": PROFILED_TRAFFIC.get((kernel_name.split()[0],) + tuple(tuning)),
                     "traffic_note": "ncu dram__bytes_read+write per launch, 1 capture; writes "
                                     "still dirty in L2 at kernel end are not counted",
                     "kernel": kernel_name,
                     "bytes_convention": "k=1 algorithmic 16 B per lattice-site update x sites "
                                         "x k steps per launch",
                     "alg_bytes_per_launch": alg_bytes, "launch_ms": launch_ms},
        "e2e": {"value": sites * S * args.steps * world / e2e_s / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": int(sum(a.nbytes for a in x0)),
                "d2h_bytes_per_step": int(sum(a.nbytes for a in x0)),
                "pipeline": "jobs alternate between two grids on two streams; pinned host "
                            "buffers; each job's copies overlap the other grid's steps, and "
                            "each job's steps follow the previous job's steps"},
        "gpu_launches": n_launch,
        "clocks": clocks,
    }
    if not args.no_companions:
        line["companions"] = companions(stream, hbm)
        if multi is not None:
            line["companions"]["multi_rank"] = multi
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_budget)
    print(json.dumps(line), flush=True)
    summary = summary_line(line)
    if summary:
        print(summary, file=sys.stderr, flush=True)


def summary_line(line) -> str:
    """One short stderr line after the JSON line with the figures a log tail should keep:
    the headline, the batched and adjoint ratios to the plain step, the Model B grids and the
    oracle on one and on all host cores."""
    parts = [f"summary: gs3d_256 {line['value']:.1f} GLUPS ({line['roofline']['frac']:.3f} of "
             f"measured HBM, k=1 bytes), e2e {line['e2e']['value']:.1f}"]
    c = line.get("companions")
    if c:
        b = c["batched_gs2d_512x"]
        a = c["adjoint_gs2d_512"]
        parts.append(f"batched 512x {b['glups']:.1f} GLUPS = {b['vs_plain_gs2d_4096']:.3f} x plain "
                     f"4096^2 ({c['plain_gs2d_4096']['glups']:.1f})")
        if "vs_plain_gs2d_512" in b:
            parts.append(f"= {b['vs_plain_gs2d_512']:.3f} x plain 512^2 "
                         f"({c['plain_gs2d_512']['glups']:.1f})")
        parts.append(f"adjoint 512^2x2000 = {a['ratio_vs_plain']:.2f} x plain forward "
                     f"(default tuning; autotuned {a['autotuned']['ratio_vs_plain']:.2f} x)")
        for k in ("ch2d_2048", "ch2d_8192", "ac2d_128"):
            if k in c:
                parts.append(f"{k} {c[k]['glups']:.1f} GLUPS")
        wr = c.get("widened_rows", {})
        if "error" in wr:
            parts.append(f"widened rows: {wr['error']}")
        for r in wr.get("stencils_gs", []):
            parts.append(f"gs {r['shape']} {r['stencil']} {r['glups']:.1f}")
        for r in wr.get("species3", []):
            parts.append(f"3 species {r['shape']} {r['glups']:.1f}")
    cb = line.get("cpu_baseline")
    if cb:
        parts.append(f"oracle 1 core {cb['single_core']['value']:.4f}, {cb['cores']} cores "
                     f"{cb['value']:.4f} GLUPS")
    return "; ".join(parts)


def multi_rank_companions(stream, rank, world, dev):
    """Under torchrun (every rank): the 512-instance batch split over the ranks by
    shard_instances (no data exchange; weak in instances, strong in the batch), and the
    256^3 Gray-Scott grid split into z-slabs over the ranks (strong scaling: boundary planes
    exchanged over NCCL every k steps). Times are the slowest rank's, with a barrier on
    both sides."""
    import torch
    import torch.distributed as dist
    import paper_2109_02598_gb300 as pf
    out = {}
    with torch.cuda.stream(stream):
        specs = synthetic.batch_instances(512, seed=4)
        mine = pf.shard_instances([q["n"] ** 2 for q in specs], rank, world)
        b = pf.Batch([dict(n=specs[i]["n"], Du=0.2, Dv=0.1, F=specs[i]["F"], k=specs[i]["k"])
                      for i in mine], 0.5, stream=stream)
        for j, i in enumerate(mine):
            u, v = synthetic.batch_instance_init(specs[i]["n"], i)
            b.write(j, 0, u).write(j, 1, v)
        b.autotune(3)
        b.run(2000)
        torch.cuda.synchronize()
        dist.barrier()
        ms = _time(stream, lambda: b.run(2000))
        ms = _max_over_ranks(ms, world, dev)
        sites = _sum_over_ranks(float(b.sites), world, dev)
        b.close()
        out["batched_gs2d_512x_sharded"] = {"ranks": world, "instances_here": len(mine),
                                            "glups": sites * 2000 / (ms * 1e-3) / 1e9,
                                            "ms": ms}
        w = synthetic.WORKLOADS[WORKLOAD]
        x0 = synthetic.workload_init(WORKLOAD)
        k = 4
        sg = pf.SlabGrid(x0[0].shape, 2, w["model"], w["coeffs"], w["dt"], w["h"], k=k,
                         stream=stream)
        sg.write_global(x0)
        sg.step(2 * k)
        torch.cuda.synchronize()
        dist.barrier()
        steps = 200
        t0 = time.perf_counter()
        sg.step(steps)
        torch.cuda.synchronize()
        dt = _max_over_ranks(time.perf_counter() - t0, world, dev)
        sg.close()
        out["slab_gs3d_256"] = {"ranks": world, "k_steps_per_exchange": k, "steps": steps,
                                "glups": x0[0].size * steps / dt / 1e9,
                                "scaling": "strong (one 256^3 grid split into z-slabs)"}
    return out


def _sum_over_ranks(x: float, world: int, device=None) -> float:
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t)
    return float(t.item())


def _time(stream, fn, reps=1):
    """Device time (ms) of ``reps`` calls of ``fn`` on ``stream`` with CUDA events."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def companions(stream, hbm):
    """The other workloads, each timed on the device: the 512-instance batched Gray-Scott
    run against plain 2D grids of 4096^2 and 512^2, the adjoint against the plain forward run
    at the same size, and the Cahn-Hilliard 2048^2 and 8192^2 and Allen-Cahn 128^2 steps."""
    import torch
    import paper_2109_02598_gb300 as pf
    out = {}
    with torch.cuda.stream(stream):
        # ---- batched: 512 x 2D Gray-Scott, sides log-uniform in [64, 512], 2000 steps
        out["batched_gs2d_512x"] = batch_timing(stream, 2000, hbm)
        bglups = out["batched_gs2d_512x"]["glups"]
        # ---- plain 2D Gray-Scott of comparable state size (4096^2, 268 MB ping-pong)
        u, v = synthetic.gray_scott_init((4096, 4096), seed=9, n_seeds=1024, side=8)
        g = pf.Grid((4096, 4096), 2, stream=stream).set_model("gs", (0.2, 0.1, 0.04, 0.06), 0.5)
        g.write_fields((u, v))
        t2 = g.autotune(3)
        g.step(200)  # records the graph of this run length
        ms = _time(stream, lambda: g.step(200))
        pglups = 4096 * 4096 * 200 / (ms * 1e-3) / 1e9
        out["plain_gs2d_4096"] = {"glups": pglups, "tuning": list(t2)}
        out["batched_gs2d_512x"]["vs_plain_gs2d_4096"] = bglups / pglups
        g.close()
        # ---- and a plain 512^2 grid, the size of the batch's largest instances
        u, v = synthetic.gray_scott_init((512, 512), seed=10, n_seeds=16, side=8)
        g = pf.Grid((512, 512), 2, stream=stream).set_model("gs", (0.2, 0.1, 0.04, 0.06), 0.5)
        g.write_fields((u, v))
        t5 = g.autotune(5)
        g.step(2000)  # records the graph of this run length
        ms = _time(stream, lambda: g.step(2000))
        p5 = 512 * 512 * 2000 / (ms * 1e-3) / 1e9
        out["plain_gs2d_512"] = {"glups": p5, "tuning": list(t5)}
        out["batched_gs2d_512x"]["vs_plain_gs2d_512"] = bglups / p5
        g.close()
        # ---- adjoint 512^2, 2000 steps, sqrt(N) checkpoints vs the plain forward run
        out["adjoint_gs2d_512"] = adjoint_timing(stream, 512, 2000)
        # ---- Cahn-Hilliard 2048^2 (L2-resident), the same recipe on 8192^2 (268 MB per
        # field, out of L2) and Allen-Cahn 128^2
        for name, wname, shape, steps in (("ch2d_2048", "ch2d_2048", None, 2000),
                                          ("ch2d_8192", "ch2d_2048", (8192, 8192), 500),
                                          ("ac2d_128", "ac2d_128", None, 1000)):
            w = synthetic.WORKLOADS[wname]
            shape = shape or w["shape"]
            x0 = synthetic.workload_init(wname, shape)
            g = pf.Grid(shape, 1, stream=stream).set_model(w["model"], w["coeffs"], w["dt"])
            g.write_fields(x0)
            t = g.autotune(5)
            g.step(steps)  # records the graph of this run length
            ms = _time(stream, lambda: g.step(steps))
            sites = int(np.prod(shape))
            glups = sites * steps / (ms * 1e-3) / 1e9
            out[name] = {"steps": steps, "glups": glups, "tuning": list(t)}
            if w["model"] == "ch":
                out[name]["hbm_frac_k1_bytes"] = glups * 8.0 / hbm
            g.close()
        # ---- the paper's performance table (Sec. 3.1) with the forward-Euler solver:
        # 10^4 steps of Models A and C; device time and end to end (host in/out)
        rows = []
        for case in synthetic.PAPER_TABLE:
            nsteps = synthetic.PAPER_TABLE_STEPS
            x0 = synthetic.paper_timing_init(case["model"], case["shape"])
            g = pf.Grid(case["shape"], len(x0), stream=stream).set_model(
                case["model"], case["coeffs"], case["dt"])
            g.write_fields(x0)
            t = g.autotune(3)
            g.step(nsteps)  # records the graph
            dev_ms = _time(stream, lambda: g.step(nsteps))
            t0 = time.perf_counter()
            g.write_fields(x0)
            g.step(nsteps)
            g.read_fields()
            e2e_s = time.perf_counter() - t0
            sites = int(np.prod(case["shape"]))
            rows.append({"model": "A" if case["model"] == "ac" else "C",
                         "shape": "x".join(str(v) for v in case["shape"][::-1]),
                         "steps": nsteps, "device_s": dev_ms / 1e3, "e2e_s": e2e_s,
                         "glups": sites * nsteps / (dev_ms * 1e-3) / 1e9, "tuning": list(t),
                         "paper_best_cpu_s": case["paper_best_s"]})
            g.close()
        out["paper_table_forward_euler"] = {
            "rows": rows,
            "note": "paper times are whole-program runs of its semi-implicit spectral solver "
                    "on 2016-2017 desktop CPUs (context only)"}
        out["paper_table_spectral"] = paper_table_spectral(stream)
    try:  # reported in the line, never fatal for the headline
        out["widened_rows"] = widened_rows(stream, hbm)
    except Exception as exc:
        out["widened_rows"] = {"error": f"{type(exc).__name__}: {exc}"}
    return out


def _grid_rate(pf, stream, shape, model, coeffs, dt, x0, steps, stencil="std"):
    """GLUPS and tuning of ``steps`` forward-Euler steps of one grid, autotuned, timed on the
    device after one untimed call of the same length (which records its graph)."""
    g = pf.Grid(shape, len(x0), stream=stream).set_model(model, coeffs, dt)
    if stencil != "std":
        g.set_stencil(stencil)
    g.write_fields(x0)
    t = g.autotune(3)
    g.step(steps)
    ms = _time(stream, lambda: g.step(steps))
    g.close()
    return int(np.prod(shape)) * steps / (ms * 1e-3) / 1e9, list(t)


def _host_us(fn, reps):
    """Host wall time (us) per call of a call that ends with a host synchronisation."""
    fn()
    t0 = time.perf_counter()
    for _ in range(reps):
        fn()
    return (time.perf_counter() - t0) * 1e6 / reps


def widened_rows(stream, hbm):
    """The rows beyond the headline step, each measured on the device: the isotropic and
    fourth-order Laplacians (Sec. 2.2.2) beside the 5-/7-point one on the same grids, three
    coupled reaction-diffusion species (Sec. 2.3's coupled equations of motion), and the
    analysis calls (mass and free-energy reductions, the structure factor of Sec. 3 and the
    Porod fit), the last timed per call with its host synchronisation. ``hbm_frac_k1`` is the
    k = 1 byte count (every field read and written once per update) over the measured copy
    bandwidth."""
    import torch
    import paper_2109_02598_gb300 as pf
    out = {}
    gs = (0.2, 0.1, 0.04, 0.06)
    with torch.cuda.stream(stream):
        # ---- Laplacian stencils on Gray-Scott 4096^2 (200 steps) and 256^3 (20 steps)
        rows = []
        for shape, steps, stencils in (((4096, 4096), 200, ("std", "iso", "4th")),
                                       ((256, 256, 256), 20, ("std", "iso", "iso27"))):
            x0 = synthetic.gray_scott_init(shape, seed=11, n_seeds=1024 if len(shape) == 2 else 20,
                                           side=8)
            for st in stencils:
                glups, t = _grid_rate(pf, stream, shape, "gs", gs, 0.5, x0, steps, st)
                rows.append({"shape": "x".join(str(v) for v in shape[::-1]), "stencil": st,
                             "points": {"std": 5 if len(shape) == 2 else 7, "iso": 9 if len(shape) == 2
                                        else 19, "4th": 9, "iso27": 27}[st],
                             "steps": steps, "glups": glups, "tuning": t,
                             "hbm_frac_k1": glups * BYTES_PER_LUP["gs"] / hbm})
        out["stencils_gs"] = rows
        # ---- three coupled species: a constant source, linear, quadratic, cubic and mixed
        # monomials; 24 B per update at k = 1
        D, E, K = RD3
        rows = []
        for shape, steps in (((4096, 4096), 100), ((256, 256, 256), 20)):
            n = int(np.prod(shape))
            x0 = tuple(synthetic.uniform(12, 60 + i, n, 0.05, 0.9).reshape(shape).astype(np.float32)
                       for i in range(3))
            glups, t = _grid_rate(pf, stream, shape, "rd", pf.rd_coeffs(D, E, K), 0.2, x0, steps)
            rows.append({"shape": "x".join(str(v) for v in shape[::-1]), "species": 3,
                         "monomials": len(E), "steps": steps, "glups": glups, "tuning": t,
                         "hbm_frac_k1": glups * 24.0 / hbm})
        out["species3"] = rows
        # ---- analysis calls on resident grids: mass (one field, 4 B per site) and energy
        rows = []
        for shape, model, coeffs, dt, nf in (((256, 256, 256), "ac", (1.0, 1.0), 0.05, 1),
                                             ((2048, 2048), "ac", (1.0, 1.0), 0.05, 1),
                                             ((128, 128, 128), "c", (1.0,) * 5, 0.005, 2)):
            x0 = synthetic.paper_timing_init(model, shape)[:nf]
            g = pf.Grid(shape, nf, stream=stream).set_model(model, coeffs, dt)
            g.write_fields(x0)
            sites = int(np.prod(shape))
            m_us = _host_us(lambda: g.mass(0), 20)
            e_us = _host_us(g.energy, 10)
            rows.append({"shape": "x".join(str(v) for v in shape[::-1]), "model": model,
                         "mass_us": m_us, "mass_gbs": sites * 4 / (m_us * 1e-6) / 1e9,
                         "energy_us": e_us, "energy_fields": nf})
            if len(shape) == 2 or model == "c":
                s_us = _host_us(lambda: g.structure_factor(0, 32), 5)
                c, mean, cnt = g.structure_factor(0, 32)
                f_us = _host_us(lambda: pf.porod_fit(c, mean, cnt, float(c[len(c) // 2]),
                                                     float(c[-2])), 50)
                rows[-1].update({"structure_factor_us": s_us, "porod_fit_us": f_us})
            g.close()
        out["analysis"] = rows
        out["note"] = ("stencils and species on the forward-Euler step, timed with CUDA events; "
                       "analysis calls by host wall time per call including the synchronisation")
    return out


def paper_table_spectral(stream):
    """The paper's performance table (Sec. 3.1) with the solver it was measured with: 10^4
    semi-implicit spectral steps of Models A and C on 128^2, 512^2 and 64^3.  ``e2e_s`` covers
    what the paper's whole-program time covers on the GPU side: building the solver (plans and
    the A, B N tables), copying the initial fields in, the steps, and reading the result."""
    import torch
    import paper_2109_02598_gb300 as pf
    rows = []
    with torch.cuda.stream(stream):
        for case in synthetic.PAPER_TABLE:
            nsteps = synthetic.PAPER_TABLE_STEPS
            x0 = synthetic.paper_timing_init(case["model"], case["shape"])
            sp = pf.Spectral(case["shape"], case["model"], case["coeffs"], case["dt"],
                             stream=stream)
            sp.write_fields(x0)
            sp.step(64)  # records the step graph
            dev_ms = _time(stream, lambda: sp.step(nsteps))
            sp.close()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sp = pf.Spectral(case["shape"], case["model"], case["coeffs"], case["dt"],
                             stream=stream)
            sp.write_fields(x0)
            sp.step(nsteps)
            final = sp.read_fields()
            e2e_s = time.perf_counter() - t0
            sp.close()
            sites = int(np.prod(case["shape"]))
            rows.append({"model": "A" if case["model"] == "ac" else "C",
                         "shape": "x".join(str(v) for v in case["shape"][::-1]),
                         "steps": nsteps, "device_s": dev_ms / 1e3, "e2e_s": e2e_s,
                         "us_per_step": dev_ms * 1e3 / nsteps,
                         "mlups": sites * nsteps / (dev_ms * 1e-3) / 1e6,
                         "paper_best_cpu_s": case["paper_best_s"],
                         "paper_best_over_e2e": case["paper_best_s"] / e2e_s,
                         "final_finite": bool(all(np.isfinite(x).all() for x in final)),
                         "final_max_abs": float(max(np.abs(x).max() for x in final))})
    return {"rows": rows,
            "note": "same solver, sizes, step count and initial conditions as the paper's "
                    "table; its times are whole-program runs on 2016-2017 desktop CPUs"}


def run_spectral_case(spec: str):
    """One spectral case: paper initial conditions, Delta t of the paper-table runs, STEPS
    steps timed with CUDA events after one untimed call of the same length."""
    import torch
    import paper_2109_02598_gb300 as pf
    parts = spec.split(":")
    model, shape, steps = parts[0], tuple(int(v) for v in parts[1].split("x")), int(parts[2])
    engine = parts[3] if len(parts) > 3 else "auto"
    shape = shape[::-1]  # given as NX x NY [x NZ]; arrays are (NZ,) NY, NX
    coeffs = {"ac": (1.0, 1.0), "ch": (1.0, 1.0, 1.0), "c": (1.0,) * 5}[model]
    dt = {"ac": 0.05, "ch": 0.05, "c": 0.005}[model]
    x0 = synthetic.paper_timing_init("ac" if model == "ch" else model, shape)[:1 if model != "c" else 2]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sp = pf.Spectral(shape, model, coeffs, dt, stream=stream).set_engine(engine)
        sp.write_fields(x0)
        sp.step(steps)
        ms = _time(stream, lambda: sp.step(steps))
        final = sp.read_fields()
        used = sp.engine
        sp.close()
    print(json.dumps({"spectral": spec, "engine": used, "steps": steps,
                      "us_per_step": ms * 1e3 / steps,
                      "final_finite": bool(all(np.isfinite(x).all() for x in final))}))


def batch_timing(stream, steps: int, hbm: float) -> dict:
    """The batched workload: 512 independent 2D Gray-Scott grids, sides log-uniform in
    [64, 512], seeded F and k; autotuned, then `steps` steps timed as one CUDA-graph run after
    one untimed run of the same length."""
    import paper_2109_02598_gb300 as pf
    specs = synthetic.batch_instances(512, seed=4)
    b = pf.Batch([dict(n=q["n"], Du=0.2, Dv=0.1, F=q["F"], k=q["k"]) for q in specs], 0.5,
                 stream=stream)
    for i, q in enumerate(specs):
        u, v = synthetic.batch_instance_init(q["n"], i)
        b.write(i, 0, u).write(i, 1, v)
    tuning = b.autotune(3)
    b.run(steps)
    ms = _time(stream, lambda: b.run(steps))
    glups = b.sites * steps / (ms * 1e-3) / 1e9
    res = {"steps": steps, "sites": b.sites, "ms": ms, "glups": glups, "tuning": list(tuning),
           "hbm_frac_k1_bytes": glups * 16 / hbm,
           "launch": f"one CUDA graph per {steps} steps"}
    b.close()
    return res


def run_batch_case(steps: int):
    """The batched workload alone, printing its JSON line."""
    import torch
    hbm, _ = _peaks()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        res = batch_timing(stream, steps, hbm)
    print(json.dumps({"batch": steps, **res}))


def adjoint_timing(stream, n: int, steps: int) -> dict:
    """The Gray-Scott adjoint workload's recipe on an n x n grid for `steps` steps: the plain
    forward run, the checkpointed forward and the reverse pass, each timed with CUDA events
    after one untimed call of the same kind (which records its CUDA graph and allocates its
    checkpoints), so the timed calls are the steady state an optimisation loop sees."""
    import paper_2109_02598_gb300 as pf
    w = synthetic.WORKLOADS["gs2d_adjoint_512"]
    u0, v0 = synthetic.workload_init("gs2d_adjoint_512", shape=(n, n))
    g = pf.Grid((n, n), 2, stream=stream).set_model("gs", w["coeffs"], w["dt"])
    g.write_fields((u0, v0))
    g.step(steps)
    plain = _time(stream, lambda: g.step(steps))
    g.write_fields((u0, v0))
    pf.adjoint_forward(g, steps)
    fwd = _time(stream, lambda: pf.adjoint_forward(g, steps))
    gu = g.read_field(0, device=True) * 0.01  # any dL/dx_N: the cost does not depend on it
    gv = g.read_field(1, device=True) * 0.01
    pf.adjoint_backward(g, gu, gv)
    bwd = _time(stream, lambda: pf.adjoint_backward(g, gu, gv))
    # the same with the grid autotuned (the plain run and the checkpointed forward take the
    # tuned tile and depth; the reverse pass's recomputation and adjoint steps are k = 1)
    g.write_fields((u0, v0))
    tuning = g.autotune(3)
    g.write_fields((u0, v0))
    g.step(steps)
    plain_t = _time(stream, lambda: g.step(steps))
    g.write_fields((u0, v0))
    pf.adjoint_forward(g, steps)
    fwd_t = _time(stream, lambda: pf.adjoint_forward(g, steps))
    pf.adjoint_backward(g, gu, gv)
    bwd_t = _time(stream, lambda: pf.adjoint_backward(g, gu, gv))
    g.close()
    res = {"steps": steps, "plain_forward_ms": plain, "adjoint_forward_ms": fwd,
           "adjoint_backward_ms": bwd, "ratio_vs_plain": (fwd + bwd) / plain,
           "reverse_us_per_step": bwd * 1e3 / steps,
           "checkpoint_interval": int(np.ceil(np.sqrt(steps))),  # the library's default
           "tuning": "the grid's default (64x16, k = 1)",
           "autotuned": {"tuning": list(tuning), "plain_forward_ms": plain_t,
                         "adjoint_forward_ms": fwd_t, "adjoint_backward_ms": bwd_t,
                         "ratio_vs_plain": (fwd_t + bwd_t) / plain_t}}
    return res


def run_adjoint_case(spec: str):
    """One adjoint case alone (N:STEPS), timed as adjoint_timing does."""
    import torch
    n, steps = (int(v) for v in spec.split(":"))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        res = adjoint_timing(stream, n, steps)
    print(json.dumps({"adjoint": spec, **res}))


def run_euler_case(spec: str):
    """One forward-Euler case: the paper's U(-1, 1) initial fields (Gray-Scott: seeded
    squares), the coefficients and Delta t of the parity tests, STEPS steps timed with CUDA
    events after one untimed call of the same length."""
    import torch
    import paper_2109_02598_gb300 as pf
    parts = spec.split(":")
    model, shape, steps = parts[0], tuple(int(v) for v in parts[1].split("x"))[::-1], int(parts[2])
    stencil = parts[6] if len(parts) >= 7 else "std"
    if model == "rd3":  # the three coupled species of the widened-rows companion
        model, dt = "rd", 0.2
        coeffs = pf.rd_coeffs(*RD3)
        n = int(np.prod(shape))
        x0 = tuple(synthetic.uniform(12, 60 + i, n, 0.05, 0.9).reshape(shape).astype(np.float32)
                   for i in range(3))
    else:
        coeffs = {"ac": (1.0, 1.0), "ch": (1.0, 1.0, 1.0), "gs": (0.2, 0.1, 0.04, 0.06),
                  "c": (1.0,) * 5}[model]
        dt = {"ac": 0.05, "ch": 0.01, "gs": 0.5, "c": 0.005}[model]
        if model == "gs":
            x0 = synthetic.gray_scott_init(shape, seed=3, n_seeds=8, side=8)
        else:
            x0 = tuple(0.5 * x for x in
                       synthetic.paper_timing_init("c" if model == "c" else "ac", shape))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = pf.Grid(shape, len(x0), stream=stream)
        if stencil != "std":
            g.set_stencil(stencil)
        g.set_model(model, coeffs, dt).write_fields(x0)
        if len(parts) >= 6:
            g.set_tuning(int(parts[3]), int(parts[4]), int(parts[5]))
        else:
            g.autotune(3)
        g.step(steps)
        ms = _time(stream, lambda: g.step(steps))
        tuning = g.tuning
        g.close()
    sites = int(np.prod(shape))
    print(json.dumps({"euler": spec, "tuning": list(tuning), "steps": steps,
                      "us_per_step": ms * 1e3 / steps,
                      "glups": sites * steps / (ms * 1e-3) / 1e9}))


def _launch_schedule(n, k):
    left = n
    while left > 0:
        kk = k
        while kk > left:
            kk >>= 1
        yield kk
        left -= kk


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pf", choices=["pf", "reference"])
    ap.add_argument("--substeps", type=int, default=250)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-companions", action="store_true",
                    help="skip the batched / adjoint / CH / AC measurements")
    ap.add_argument("--spectral", metavar="MODEL:NXxNY[xNZ]:STEPS[:ENGINE]",
                    help="time one spectral-solver case alone (e.g. c:512x512:200:cufft) "
                         "and print its JSON line instead of the bench line")
    ap.add_argument("--euler", metavar="MODEL:NXxNY[xNZ]:STEPS[:TX:TY:K[:STENCIL]]",
                    help="time one forward-Euler case alone (autotuned unless a tuning is "
                         "given; e.g. ac:128x128:1000) and print its JSON line")
    ap.add_argument("--adjoint", metavar="N:STEPS",
                    help="time the Gray-Scott adjoint alone on an N x N grid (forward with "
                         "checkpoints, reverse pass, and the plain forward run) and print its "
                         "JSON line")
    ap.add_argument("--batch", metavar="STEPS", type=int,
                    help="time the 512-instance batched Gray-Scott workload alone")
    args = ap.parse_args()
    if args.batch:
        run_batch_case(args.batch)
        return
    if args.adjoint:
        run_adjoint_case(args.adjoint)
        return
    if args.spectral:
        run_spectral_case(args.spectral)
        return
    if args.euler:
        run_euler_case(args.euler)
        return
    if args.impl == "reference":
        rank, world, _ = _dist_init(False)
        run_reference(args, rank, world)
        return
    rank, world, local = _dist_init(True)
    run_gpu(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
