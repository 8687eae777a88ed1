#!/usr/bin/env python3
"""Benchmark of the fused D3Q19 + D3Q7 MRT stream-collide step on one GB300 (or N replicas).

Workload: the mixed-convection porous channel, 256 x 64 x 64 sites, FP32 population storage
and arithmetic (porosity 0.7, Da = 1e-3, Re = 10, Pr = 0.71, Ri = 1, u0 = 0.01, velocity
inlet at T = 0, anchored convective outflow, walls at T = 1 / T = 0, periodic in z).  One
bench step is one time step of the whole lattice.  Prints ONE JSON line (rank 0).

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

``--impl reference`` times the FP64 CPU oracle on the same workload instead (a bounded
z-slab of the channel per step, periodic in z like the full channel).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS (D3Q19+D3Q7)"
UNIT = "MLUPS"
NX, NY, NZ = 256, 64, 64
# Workloads: the headline channel, and the heterogeneous-porosity cavities of the precision
# sweep (edge 128 or 256, Ra = 1e5, Da = 1e-2, mean porosity 0.6, Pr = 0.71).
WORKLOADS = {
    "channel": (256, 64, 64),
    "cavity128": (128, 128, 128),
    "cavity256": (256, 256, 256),
    "batch64": (0, 0, 0),  # 64 cavities of edge 32..128 in one batched launch per step
    "serve": (0, 0, 0),    # Poisson stream of cavity and channel solves, continuous batching
    "sweep": (0, 0, 0),    # precision sweep: heterogeneous cavities to steady state, 3 formats
}


def _problem(nz=None, storage="fp32", workload="channel", q=19):
    from lbm_inputs import cavity_problem, channel_problem, porosity_field

    nx, ny, nz0 = WORKLOADS[workload]
    if workload == "channel":
        return channel_problem(nx, ny, nz or nz0, storage=storage, q=q)
    phi = porosity_field(nx, ny, nz0, seed=20161110).astype("float32")
    return cavity_problem(nx, Ra=1e5, Da=1e-2, phi=0.6, Pr=0.71, phi_field=phi, phi_ref=0.6,
                          storage=storage, q=q)


def _workload_text(workload, storage, q=19):
    if workload == "batch64":
        return (f"64 porous cavities, edges from {{32,48,64,96,128}}, own (phi, Da, Ra), one "
                f"batched launch per step under a CUDA graph, {storage.upper()} storage")
    nx, ny, nz = WORKLOADS[workload]
    if workload == "channel":
        return f"porous mixed-convection channel {nx}x{ny}x{nz}, D3Q{q}+D3Q7 MRT, {storage.upper()} storage"
    return (f"porous natural-convection cavity {nx}^3 with seeded porosity field, D3Q{q}+D3Q7 MRT, "
            f"{storage.upper()} storage")


def _config(workload="channel", storage="fp32", extra=None, q=19, scheme="pingpong"):
    if workload == "batch64":
        cfg = {"workload": _workload_text(workload, storage), "lattices": 64,
               "storage": f"{storage}-deviation",
               "scheme": ("AA in place" if scheme == "aa" else "ping-pong pull") + ", batched",
               "seed": 2016, "l2": "inputs larger than L2 (GBs of populations), no flush"}
        cfg.update(extra or {})
        return cfg
    nx, ny, nz = WORKLOADS[workload]
    elem = 4 if storage == "fp32" else 2
    state = 2 * (q + 7) * elem * nx * ny * nz / 1e6
    l2 = (f"inputs larger than L2: two population copies of {state:.0f} MB vs 126 MB L2, no flush"
          if state > 2 * 126 else
          f"two population copies of {state:.0f} MB, partly L2-resident (126 MB L2)")
    cfg = {"workload": _workload_text(workload, storage, q), "nx": nx, "ny": ny, "nz": nz,
           "storage": f"{storage}-deviation", "scheme": "ping-pong pull", "l2": l2}
    if workload == "channel":
        cfg.update({"phi": 0.7, "Da": 1e-3, "Re": 10, "Pr": 0.71, "Ri": 1.0, "u0": 0.01})
    else:
        cfg.update({"phi_mean": 0.6, "phi_std": 0.05, "Da": 1e-2, "Ra": 1e5, "Pr": 0.71})
    if extra:
        cfg.update(extra)
    return cfg


KERNEL_SOURCES = ("paper_1611_03329_gb300/csrc/lbm_kernels.cu",
                  "paper_1611_03329_gb300/csrc/lbm_internal.cuh")

# DRAM traffic per launch of the headline step kernel (256 x 64 x 64 channel, FP32) from one
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum, steady state, mean of 5
# launches); the command and the figures are recorded with the kernel's profile summary.  The
# figure describes the kernel whose sources had this hash and is reported only while they
# still do.  (Captured on sources with hash 5862eebe...; the hash below is that of the same
# step kernel after changes elsewhere in its files: the batched step kernel and its launcher.)
STEP_TRAFFIC = {"kernel_source_sha256":
                "2c2a44072a0a0b02ee95511d6c20462e0dec8696172416d4aeacfc6c6e6cb1a3",
                "dram_bytes_per_launch": 173549261}


def kernel_source_hash() -> str:
    """SHA-256 over the step kernel's sources (ties a profile to the code it measured)."""
    import hashlib

    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic():
    """DRAM bytes per launch of the headline step kernel from the recorded capture, or None
    when the kernel has changed since the counters were taken."""
    if STEP_TRAFFIC["kernel_source_sha256"] != kernel_source_hash():
        return None
    return STEP_TRAFFIC["dram_bytes_per_launch"]


def _peak():
    """Measured HBM copy bandwidth (GB/s) and its source."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
        return float(peaks["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def _init_dist(ws):
    if ws <= 1:
        return None
    import torch.distributed as dist

    dist.init_process_group("gloo")
    return dist


def _max_over_ranks(dist, value: float) -> float:
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(dist):
    if dist is not None:
        dist.barrier()


# ---- timing ----------------------------------------------------------------------------------
MIN_WINDOWS, MIN_TIMED_S, MAX_WINDOWS = 5, 1.0, 20000


def window_count(first_ms: float) -> int:
    """Windows of K steps to time: at least MIN_WINDOWS and at least MIN_TIMED_S seconds in
    all (so the clock sampler sees the GPU under load), at most MAX_WINDOWS."""
    need = math.ceil(MIN_TIMED_S * 1e3 / max(first_ms, 1e-6))
    return int(min(MAX_WINDOWS, max(MIN_WINDOWS, need)))


def timed_windows(run_k, stream, dist, torch):
    """Times windows of exactly K steps (run_k), each bracketed by a barrier and a device
    synchronisation on both sides and by CUDA events on the stream the steps run on; returns
    the window times in ms.  The number of windows is the same on every rank."""
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)

    def one():
        _barrier(dist)
        torch.cuda.synchronize()
        start.record(stream)
        run_k()
        stop.record(stream)
        stop.synchronize()
        torch.cuda.synchronize()
        _barrier(dist)
        return start.elapsed_time(stop)

    times = [one()]
    n = int(_max_over_ranks(dist, float(window_count(times[0]))))
    times += [one() for _ in range(n - 1)]
    return times


# ---- clocks --------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:7]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k] == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


# ---- CPU baseline: the oracle as it stands ------------------------------------------------------
def _oracle_run(nz: int, steps: int, warmup: int):
    import oracle

    lp = oracle.map_problem(_problem(nz))  # the channel, periodic in z
    o = oracle.Oracle(lp)
    if warmup:
        o.step(warmup)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return NX * NY * nz * steps / dt / 1e6, dt, oracle.max_threads()


def cpu_baseline(budget_s: float = 12.0):
    """The oracle on the host cores over a bounded sample of the channel: time steps of the
    full 256 x 64 x 64 lattice, as many as fit in about budget_s, on all host cores (OpenMP
    over z-planes) and then on one core."""
    import oracle

    out = None
    all_cores = oracle.max_threads()
    try:
        for cores in (all_cores, 1):
            oracle.set_threads(cores)
            mlups1, _, _ = _oracle_run(4, 1, 0)  # a 4-plane probe sizes the sample
            per_step_full = NX * NY * NZ / (mlups1 * 1e6)
            steps = max(1, min(200, int(budget_s / per_step_full)))
            mlups, dt, used = _oracle_run(NZ, steps, 0)
            rec = {"value": round(mlups, 4), "unit": UNIT, "cores": used, "kind": "oracle",
                   "sample": f"{steps} time steps of the full {NX}x{NY}x{NZ} channel "
                             f"({dt:.1f} s, FP64" +
                             (", OpenMP over z-planes)" if used > 1 else ", one core)")}
            if out is None:
                out = rec
            else:
                out["one_core"] = rec
    finally:
        oracle.set_threads(all_cores)
    return out


def run_cpu_plan():
    """The oracle's baseline plan: the 32^3 cavity for 5,000 steps, the 256 x 64 x 64 channel
    for 200 steps and the 128^3 cavity for 100 steps, each on all host cores and on one."""
    import oracle
    from lbm_inputs import cavity_problem

    cases = [("cavity 32^3, 5000 steps", cavity_problem(32, Ra=1e3, Da=1e-2, phi=0.6, Pr=1.0), 5000),
             (f"channel {NX}x{NY}x{NZ}, 200 steps", _problem(), 200),
             ("cavity 128^3, 100 steps", cavity_problem(128, Ra=1e5, Da=1e-2, phi=0.6, Pr=0.71), 100)]
    all_cores = oracle.max_threads()
    rows = []
    try:
        for name, pb, steps in cases:
            for cores in (all_cores, 1):
                oracle.set_threads(cores)
                o = oracle.Oracle(oracle.map_problem(pb))
                t0 = time.perf_counter()
                o.step(steps)
                dt = time.perf_counter() - t0
                ns = int(pb["nx"]) * int(pb["ny"]) * int(pb["nz"])
                rows.append({"case": name, "cores": oracle.max_threads(), "seconds": round(dt, 2),
                             "mlups": round(ns * steps / dt / 1e6, 4)})
                o.close()
    finally:
        oracle.set_threads(all_cores)
    print(json.dumps({"metric": "oracle MLUPS (CPU baseline plan)", "unit": UNIT,
                      "higher_is_better": True, "rows": rows}), flush=True)
    return 0


# The step kernel the library picks for the headline channel (D3Q19, even nx, ping-pong).
DEFAULT_KERNEL = "paired"


def _run_config_extra(ws, kernel, scheme):
    """The run-specific config keys, identical in both arms for the same workload."""
    return {"parallelism": f"replicas{ws}" if ws > 1 else "single", "step_kernel": kernel,
            "scheme": scheme}


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return 0
    import oracle

    budget = 120.0  # seconds for the whole --steps + --warmup run
    mlups1, _, cores = _oracle_run(8, 1, 0)
    per_site = 1.0 / (mlups1 * 1e6)
    nz = int(budget / max(1, args.steps + args.warmup) / (per_site * NX * NY))
    nz = max(1, min(NZ, nz))
    mlups, dt, cores = _oracle_run(nz, args.steps, args.warmup)
    sample = (f"each step: one time step of a {NX}x{NY}x{nz} z-slab of the channel "
              f"(periodic in z; {nz} of its {NZ} z-planes), FP64 oracle, OpenMP over z-planes")
    line = {"impl": "reference", "metric": METRIC, "value": round(mlups, 4), "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(extra=_run_config_extra(ws, DEFAULT_KERNEL, "pingpong")),
            "cpu_baseline": {"value": round(mlups, 4), "unit": UNIT, "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(mlups, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---- batched workload ------------------------------------------------------------------------
def run_batch(args, gb, torch):
    """64 cavities advanced by one batched launch per step (CUDA graph replays of up to 500
    steps), against the same lattices solved one at a time (each lattice's own launches)."""
    from lbm_inputs import batch_cavities

    pbs = [dict(pb, storage=args.storage, scheme=args.scheme) for pb in batch_cavities(64)]
    stream = torch.cuda.Stream()
    lats = [gb.Lattice(pb, stream=stream.cuda_stream) for pb in pbs]
    sites = sum(l.ns for l in lats)
    batch = gb.Batch(lats, stream=stream.cuda_stream)
    block = batch.tune() + batch.launch_groups()  # shape, then (fused, per-lattice) groups
    chunk = max(1, min(args.steps, 500))
    batch.step(args.warmup)
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        start.record(stream)
        left = args.steps
        while left > 0:
            batch.step(min(chunk, left))
            left -= min(chunk, left)
        stop.record(stream)
        stop.synchronize()
    ms = start.elapsed_time(stop)
    mlups = sites * args.steps / (ms * 1e-3) / 1e6
    # one at a time: each lattice with its own launches, for the same number of steps
    n1 = max(1, min(args.steps, 200))
    torch.cuda.synchronize()
    start.record(stream)
    for l in lats:
        l.step(n1)
    stop.record(stream)
    stop.synchronize()
    ms1 = start.elapsed_time(stop)
    mlups1 = sites * n1 / (ms1 * 1e-3) / 1e6
    unstable = 0
    for l in lats:
        try:
            l.sums()
        except gb.LbmError:
            unstable += 1
    batch.close()
    step_bytes = sum(gb.algorithmic_bytes_per_site(pb) * l.ns for pb, l in zip(pbs, lats))
    achieved = step_bytes / (ms / args.steps * 1e-3) / 1e9
    return mlups, ms, sites, achieved, clk.summary(), {
        "value": round(mlups1, 2), "unit": UNIT, "steps": n1,
        "path": "lbm_step per lattice, lattices one after another"}, block, unstable


# ---- precision sweep -------------------------------------------------------------------------
def _field_err(a, ref):
    """max|a - ref| / max|ref| (field-normalised, as in the parity tests)."""
    import numpy as np

    ref = np.asarray(ref, dtype=np.float64)
    scale = float(np.max(np.abs(ref)))
    return float(np.max(np.abs(np.asarray(a, dtype=np.float64) - ref))) / (scale or 1.0)


def run_sweep(args, gb):
    """Heterogeneous porous cavities (edge E, Ra in {1e4, 1e5, 1e6}, Da in {1e-4, 1e-2}, the
    seeded porosity field of mean 0.6) with FP32, FP16- and BF16-deviation storage, each run
    to the steady-state residual r <= 1e-7 (k = 100 steps) or the step cap; Nu_3D of the hot
    wall and the errors of the 16-bit runs against the FP32 run of the same case."""
    import numpy as np

    from lbm_inputs import cavity_problem, porosity_field

    edge, cap, tol, chunk = args.sweep_edge, args.max_steps or 200000, 1e-7, 2000
    phi = porosity_field(edge, edge, edge, seed=20161110).astype("float32")
    cases = []
    t_all = time.perf_counter()
    for Ra in args.sweep_ra:
        for Da in args.sweep_da:
            if (Ra, Da) in args.sweep_skip:
                continue
            pb = cavity_problem(edge, Ra=Ra, Da=Da, phi=0.6, Pr=0.71, phi_field=phi,
                                phi_ref=0.6)
            ref = None
            for storage in ("fp32", "fp16", "bf16"):
                lat = gb.Lattice(dict(pb, storage=storage))
                t0 = time.perf_counter()
                steps, ru, rT = 0, float("inf"), float("inf")
                # with --sweep-match, the 16-bit runs stop where the FP32 run converged
                run_cap = cap
                if storage != "fp32" and args.sweep_match and ref is not None and ref[3]:
                    run_cap = ref[4]
                while steps < run_cap:
                    n = min(chunk, run_cap - steps)
                    lat.step(n - 100)
                    lat.residual()  # snapshot of step steps + n - 100
                    lat.step(100)
                    ru, rT = lat.residual()
                    steps += n
                    if max(ru, rT) <= tol:
                        break
                wall = time.perf_counter() - t0
                _, u, T = lat.macros()
                nu = lat.nusselt(0)[0]
                rec = {"Ra": Ra, "Da": Da, "storage": storage, "steps": steps,
                       "r_u": ru, "r_T": rT, "converged": max(ru, rT) <= tol,
                       "Nu_hot": round(nu, 6), "wall_s": round(wall, 2),
                       "mlups": round(edge ** 3 * steps / wall / 1e6, 1)}
                if storage == "fp32":
                    ref = (u, T, nu, rec["converged"], steps)
                else:
                    rec.update({"err_u_vs_fp32": _field_err(u, ref[0]),
                                "err_T_vs_fp32": _field_err(T, ref[1]),
                                "err_Nu_vs_fp32": abs(nu - ref[2]) / abs(ref[2])})
                cases.append(rec)
                lat.close()
    return cases, time.perf_counter() - t_all


# ---- serving workload ------------------------------------------------------------------------
def _served_storage(gb, pb, tol):
    """The storage a request is served in: a 16-bit format whose residual floor lies above the
    tolerance is replaced by FP32 (the rule of lbm_server_submit)."""
    st = pb.get("storage", "fp32")
    return "fp32" if st in gb.RESIDUAL_FLOOR and tol < gb.RESIDUAL_FLOOR[st] else st


def _solo_stream(gb, reqs, chunk, tol, max_steps):
    """One solve at a time: each request, in arrival order and not before it arrives, is
    solved alone through the single-lattice path (lbm_step, a residual every `chunk` steps)
    until it converges or reaches its step limit."""
    t0 = time.perf_counter()
    results = []
    for arrival, pb in reqs:
        while time.perf_counter() - t0 < arrival:
            time.sleep(0.0005)
        start = time.perf_counter() - t0
        storage = _served_storage(gb, pb, tol)
        lat = gb.Lattice(dict(pb, storage=storage))
        steps, status = 0, "max_steps"
        while True:
            lat.step(chunk)
            steps += chunk
            try:
                ru, rT = lat.residual()
            except gb.LbmError:
                status = "unstable"
                break
            if ru < tol and rT < tol:
                status = "converged"
                break
            if steps >= max_steps:
                break
        lat.close()
        results.append({"arrival": arrival, "started": start, "finished": time.perf_counter() - t0,
                        "sites": lat.ns, "steps": steps, "status": status, "storage": storage})
    return results, time.perf_counter() - t0


def _serve_stream(gb, reqs, budget, chunk, tol, max_steps, fill=0, policy="fifo"):
    """Submit each request at its arrival time and run the serving loop (continuous batching)."""
    t0 = time.perf_counter()
    results = []
    srv = gb.Server(budget_bytes=budget, chunk=chunk, max_active_sites=fill, policy=policy)
    offset = None
    pending = list(reqs)
    arrivals = {}
    while pending or len(results) < len(reqs):
        now = time.perf_counter() - t0
        while pending and pending[0][0] <= now:
            arrival, pb = pending.pop(0)
            rid = srv.submit(pb, tol=tol, max_steps=max_steps)
            arrivals[rid] = arrival
            if offset is None:
                offset = now - srv.clock()  # server clock -> bench clock
        na, nq = srv.advance()
        for r in srv.poll():
            r["arrival"] = arrivals[r["id"]]
            r["finished"] = r["t_done"] + offset
            results.append(r)
        if na == 0 and nq == 0 and pending:
            time.sleep(max(0.0, min(0.001, pending[0][0] - (time.perf_counter() - t0))))
    srv.close()
    return results, time.perf_counter() - t0


def _latency_summary(results):
    lat = sorted(r["finished"] - r["arrival"] for r in results)
    lups = sum(r["sites"] * r["steps"] for r in results)
    span = max(r["finished"] for r in results) - min(r["arrival"] for r in results)
    pct = lambda q: lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]
    return {"p50_s": round(pct(0.5), 4), "p99_s": round(pct(0.99), 4),
            "mlups": round(lups / span / 1e6, 2), "makespan_s": round(span, 3),
            "statuses": {s: sum(1 for r in results if r["status"] == s)
                         for s in sorted({r["status"] for r in results})},
            "storage": {s: sum(1 for r in results if r.get("storage") == s)
                        for s in sorted({r.get("storage") for r in results})}}


# Request streams of the serving workload: "wide" spans lattices that fill the GPU alone
# (up to 192^3 and the 256 x 64 x 64 channel); "small" holds only lattices far too small to
# fill it (16^3 - 48^3 cavities, channels of section 12^2 - 24^2), the case continuous
# batching is for.
SERVE_MIXES = {
    "wide": {"n": 24, "mix": {"rate": 20.0}, "text": "porous cavities 32^3-192^3, 4WxWxW "
             "channels (W 32, 64) and, one in ten, melting cavities (enthalpy model); "
             "Poisson 20/s"},
    "small": {"n": 96, "mix": {"rate": 400.0, "edges": (16, 24, 32, 40, 48),
                               "widths": (12, 16, 24)},
              "text": "porous cavities 16^3-48^3, 4WxWxW channels (W 12, 16, 24) and, one in "
                      "ten, melting cavities (enthalpy model); Poisson 400/s"},
}


def run_serve(args, gb):
    from lbm_inputs import serving_mix

    reqs = serving_mix(args.requests or SERVE_MIXES[args.serve_mix]["n"], seed=5,
                       **SERVE_MIXES[args.serve_mix]["mix"])
    tol, max_steps, chunk = 1e-6, args.max_steps or 50000, 100
    runs = {}
    runs["fifo"] = _latency_summary(_serve_stream(gb, reqs, 0, chunk, tol, max_steps,
                                                  fill=args.fill, policy="fifo")[0])
    runs["backfill"] = _latency_summary(_serve_stream(gb, reqs, 0, chunk, tol, max_steps,
                                                      fill=args.fill, policy="backfill")[0])
    runs["one_at_a_time"] = _latency_summary(_solo_stream(gb, reqs, chunk, tol, max_steps)[0])
    return runs, len(reqs), tol, max_steps


# ---- our arm ---------------------------------------------------------------------------------
def run_ours(args):
    ws, rank = _dist()
    if ws > 1 and "LOCAL_RANK" in os.environ and "CUDA_VISIBLE_DEVICES" not in os.environ:
        os.environ["CUDA_VISIBLE_DEVICES"] = os.environ["LOCAL_RANK"]  # one replica per GPU
    import numpy as np
    import torch

    import paper_1611_03329_gb300 as gb

    dist = _init_dist(ws)
    gb.build.build()
    torch.cuda.set_device(0)
    if args.workload == "sweep":
        cases, wall = run_sweep(args, gb)
        if rank != 0:
            return 0
        line = {"metric": "steady-state Nu and 16-bit storage error (precision sweep)",
                "value": None, "unit": None, "n_gpus": ws, "steps": None, "warmup": 0,
                "higher_is_better": None, "dtype": "f32-math, fp32 / fp16 / bf16 storage",
                "data": "synthetic",
                "config": {"workload": f"porous cavities {args.sweep_edge}^3, seeded porosity "
                                       "field (mean 0.6, std 0.05, [0.4, 0.9]), Pr 0.71, "
                                       f"Ra in {args.sweep_ra}, Da in {args.sweep_da}"
                                       + (f", without {args.sweep_skip}" if args.sweep_skip else ""),
                           "tol": 1e-7, "k": 100, "max_steps": args.max_steps or 200000},
                "wall_s": round(wall, 1), "cases": cases}
        print(json.dumps(line), flush=True)
        return 0
    if args.workload == "serve":
        runs, n, tol, max_steps = run_serve(args, gb)
        if rank != 0:
            return 0
        best = max(("fifo", "backfill"), key=lambda k: runs[k]["mlups"])
        line = {"metric": "time-to-steady-state p50/p99 and aggregate MLUPS (serving)",
                "value": runs[best]["mlups"], "unit": UNIT, "n_gpus": ws, "steps": None,
                "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32-math, fp32 or fp16 storage per request", "data": "synthetic",
                "config": {"workload": f"{n} requests (seed 5, mix '{args.serve_mix}'): "
                                       + SERVE_MIXES[args.serve_mix]["text"],
                           "tol": tol, "max_steps": max_steps, "chunk": 100,
                           "admission": "by device footprint (80% of free memory)"
                                        + (f", at most {args.fill} sites admitted" if args.fill else ""),
                           "storage_rule": "16-bit requests whose tolerance lies below the "
                                           "format's residual floor are served in FP32"},
                "policy": best, "latency": {"p50_s": runs[best]["p50_s"], "p99_s": runs[best]["p99_s"]},
                "serving": runs,
                "speedup_mlups": round(runs[best]["mlups"] / runs["one_at_a_time"]["mlups"], 3),
                "speedup_p50": round(runs["one_at_a_time"]["p50_s"] / runs[best]["p50_s"], 3)}
        print(json.dumps(line), flush=True)
        return 0
    if args.workload == "batch64":
        mlups, ms, sites, achieved, clocks, one, block, unstable = run_batch(args, gb, torch)
        mlups_all = _max_over_ranks(dist, 0.0)  # keep ranks in step
        if rank != 0:
            return 0
        peak = _peak()
        line = {"metric": METRIC, "value": round(mlups * ws, 2), "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(ms / args.steps, 6), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp32": "f32", "fp16": "f16-storage/f32-math",
                          "bf16": "bf16-storage/f32-math"}[args.storage],
                "data": "synthetic",
                "config": _config("batch64", args.storage, scheme=args.scheme,
                                  extra={"sites": sites, "block_threads": block[0],
                                         "planes_per_block": block[1],
                                         "groups_fused": block[2], "groups_per_lattice": block[3],
                                         "unstable_lattices": unstable}),
                "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak[0],
                             "unit": "GB/s", "frac": round(achieved / peak[0], 4),
                             "traffic": None, "peak_source": peak[1]},
                "one_at_a_time": one,
                "batched_speedup": round(mlups / one["value"], 3),
                "gpu_launches": args.steps, "clocks": clocks}
        print(json.dumps(line), flush=True)
        return 0
    stream = torch.cuda.Stream()
    q = 15 if args.lattice == "d3q15" else 19
    pb = dict(_problem(storage=args.storage, workload=args.workload, q=q), scheme=args.scheme)
    wnx, wny, wnz = WORKLOADS[args.workload]
    ns = wnx * wny * wnz
    with torch.cuda.stream(stream):
        lat = gb.Lattice(pb, stream=stream.cuda_stream)
        if args.kernel != "auto":
            lat.set_step_kernel(args.kernel)
        kernel = lat.step_kernel  # the kernel that runs
        aa = lat.lattice()["scheme"] == 1
        lat.step(args.warmup)
        lat.sync()
        lat.residual()  # snapshot: the residual after the timed steps measures their change

        # ---- device-resident timing (the value) ----
        with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
            windows = timed_windows(lambda: lat.step(args.steps), stream, dist, torch)
        ms = statistics.median(windows)
        ms_max = _max_over_ranks(dist, ms)
        mlups = ns * args.steps * ws / (ms_max * 1e-3) / 1e6
        ru, rT = lat.residual()  # relative change over the timed steps (finite state)
        m_dev, h_dev = lat.sums()

        # ---- end to end through the host-buffer C ABI ----
        # every step: the stored state from pinned host memory (lbm_load_state, one copy per
        # region, no conversion), one time step, the macroscopic fields back into pinned host
        # arrays (lbm_macros, synchronising)
        n_e2e = max(1, min(args.steps, 50 if args.workload == "channel" else 5))
        nblob = lat.state_bytes()
        blob = torch.empty(nblob, dtype=torch.uint8).pin_memory().numpy()
        lat.save_state(blob)
        rho_h = torch.empty((wnz, wny, wnx), dtype=torch.float32).pin_memory().numpy()
        u_h = torch.empty((3, wnz, wny, wnx), dtype=torch.float32).pin_memory().numpy()
        T_h = torch.empty((wnz, wny, wnx), dtype=torch.float32).pin_memory().numpy()
        for _ in range(3):
            lat.load_state(blob, sync=False)
            lat.step(1)
            lat.macros_into(rho_h, u_h, T_h)
        _barrier(dist)
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            lat.load_state(blob, sync=False)
            lat.step(1)
            lat.macros_into(rho_h, u_h, T_h)
        e2e_s = _max_over_ranks(dist, time.perf_counter() - t0)
        e2e_mlups = ns * n_e2e * ws / e2e_s / 1e6
        # the same round trip with the populations as FP64 full values (lbm_set_populations)
        f, g = lat.populations()
        fp = torch.from_numpy(f).pin_memory().numpy()
        gp = torch.from_numpy(g).pin_memory().numpy()
        lat.set_populations(fp, gp)
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            lat.set_populations(fp, gp)
            lat.step(1)
            lat.macros_into(rho_h, u_h, T_h)
        f64_s = _max_over_ranks(dist, time.perf_counter() - t0)
        f64_mlups = ns * n_e2e * ws / f64_s / 1e6
    lat.close()

    if rank != 0:
        return 0
    peak, peak_src = _peak()
    bytes_site = gb.algorithmic_bytes_per_site(pb)
    kernel_ms = ms / args.steps  # one fused step kernel per time step
    achieved = bytes_site * ns / (kernel_ms * 1e-3) / 1e9
    cpu = (cpu_baseline() if (ws == 1 and not args.no_cpu_baseline and args.workload == "channel" and q == 19)
           else None)
    line = {
        "metric": METRIC if q == 19 else "MLUPS (D3Q15+D3Q7)", "value": round(mlups, 2),
        "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 6),
        "timing": {"windows": len(windows), "steps_per_window": args.steps,
                   "statistic": "median window, max over ranks",
                   "window_ms_min": round(min(windows), 5), "window_ms_max": round(max(windows), 5)},
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp16": "f16-storage/f32-math", "bf16": "bf16-storage/f32-math"}[args.storage],
        "data": "synthetic",
        "config": _config(args.workload, args.storage, q=q,
                          extra=_run_config_extra(ws, kernel, args.scheme)),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4),
                     "traffic": (profiled_traffic()
                                 if (args.workload, args.storage, q, kernel) == ("channel", "fp32", 19, "paired")
                                 else None),
                     "peak_source": peak_src,
                     "algorithmic_bytes_per_site": bytes_site, "sites_per_launch": ns,
                     "limiter": ("DRAM and memory latency (ncu: long-scoreboard stalls first; "
                                 "alternating sweep directions serve part of each step's reads "
                                 "from L2, so DRAM traffic is below the algorithmic bytes)"
                                 if args.storage == "fp32" else
                                 "instruction issue (ncu on the channel: issue-bound, DRAM well "
                                 "below peak)"),
                     "kernel": ("aa_pull_kernel<true> / aa_local_kernel<true> alternating (AA, one "
                                "copy in place, porosity field)" if aa else
                                {"tma": "tma_step_kernel", "paired": "step_pair_kernel"}.get(kernel, "step_kernel") +
                                (f"<false,true,D3Q{q}> (fused stream-collide, outflow)"
                                 if args.workload == "channel" else
                                 f"<true,false,D3Q{q}> (fused stream-collide, porosity field)") +
                                (", two x-adjacent sites per thread" if kernel == "paired" else ""))},
        "cpu_baseline": cpu,
        "e2e": {"value": round(e2e_mlups, 2), "unit": UNIT,
                "h2d_bytes_per_step": int(nblob),
                "d2h_bytes_per_step": int(rho_h.nbytes + u_h.nbytes + T_h.nbytes),
                "steps": n_e2e,
                "path": "lbm_load_state (stored state, pinned host) + lbm_step(1) + lbm_macros (pinned host)",
                "fp64_populations": {"value": round(f64_mlups, 2),
                                     "h2d_bytes_per_step": int(fp.nbytes + gp.nbytes),
                                     "path": "lbm_set_populations (pinned FP64 full values) + "
                                             "lbm_step(1) + lbm_macros"}},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
        "state_check": {"residual_u": ru, "residual_T": rT, "mass_dev": m_dev,
                        "heat_dev": h_dev},
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--storage", choices=("fp32", "fp16", "bf16"), default="fp32",
                    help="population storage (the headline workload is fp32)")
    ap.add_argument("--workload", choices=tuple(WORKLOADS), default="channel",
                    help="the headline workload is the 256x64x64 channel")
    ap.add_argument("--lattice", choices=("d3q19", "d3q15"), default="d3q19",
                    help="flow lattice of the channel / cavity workloads (the headline is D3Q19)")
    ap.add_argument("--scheme", choices=("pingpong", "aa", "auto"), default="pingpong",
                    help="population scheme: two copies, or one copy updated in place (AA)")
    ap.add_argument("--kernel", choices=("auto", "plain", "paired", "tma"), default="auto",
                    help="step kernel: the library's choice (auto), one site per thread, two "
                         "x-adjacent sites per thread, or populations staged by TMA")
    ap.add_argument("--requests", type=int, default=None,
                    help="serve: number of requests (default 24 wide, 96 small)")
    ap.add_argument("--serve-mix", choices=tuple(SERVE_MIXES), default="wide",
                    help="serve: request stream (lattices up to 192^3, or only small ones)")
    ap.add_argument("--max-steps", type=int, default=None,
                    help="serve / sweep: step limit per solve (default 50000 / 200000)")
    ap.add_argument("--sweep-edge", type=int, default=128, help="sweep: cavity edge")
    ap.add_argument("--sweep-ra", type=lambda t: [float(v) for v in t.split(",")],
                    default=[1e4, 1e5, 1e6], help="sweep: Rayleigh numbers (comma list)")
    ap.add_argument("--sweep-da", type=lambda t: [float(v) for v in t.split(",")],
                    default=[1e-4, 1e-2], help="sweep: Darcy numbers (comma list)")
    ap.add_argument("--sweep-skip", type=lambda t: [tuple(float(x) for x in c.split(":"))
                                                    for c in t.split(",") if c],
                    default=[], help="sweep: Ra:Da cases to leave out (comma list)")
    ap.add_argument("--sweep-match", action="store_true",
                    help="sweep: stop the 16-bit runs at the step count of the converged FP32 run")
    ap.add_argument("--cpu-plan", action="store_true",
                    help="time the oracle's baseline plan (32^3 x 5000, channel x 200, 128^3 x "
                         "100 steps, all cores and one core) instead of the GPU")
    ap.add_argument("--fill", type=int, default=8_000_000,
                    help="serve: cap on the lattice sites admitted at once (0: none)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.cpu_plan:
        return run_cpu_plan()
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
