#!/usr/bin/env python3
"""Throughput of the 1D2V flashover step on GB300: phase-space cell-updates/s
and the step kernel's fraction of the HBM roofline.

Workload (default): 1024 x 256 x 256 cells (67.1 M), velocity spans
v1 in +-6e7 m/s and v2 in +-3e7 m/s, h_max = 20 um, dt at CFL 0.4,
delta_max 3, A_max 400 eV, T_se 2 eV, J = 1 A/m^2 on [10, 15] um at
T_fe = 4 eV, f0 = 1e-6 relative seeded noise; the applied field is swept
over E_y in {-5e5, -1e6, -3e6} V/m, so one benchmark step advances the
three field instances by one solver step each (201 M cell-updates).
The headline precision (f stored and advected in FP32, moments, fluxes,
surface charge and ledger in FP64) is timed first; the FP64 path on the
same workload is reported side by side.

Launch: ``python bench.py [--gpus N] [--steps K] [--warmup W]``; for N > 1
one process per GPU under torchrun, each rank running its own independent
instances (replicas: the workload has no data exchange between instances).
``--impl reference`` times the CPU oracle instead (see DESIGN).
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

import numpy as np  # noqa: E402

from paper_2303_14119_gb300 import synth  # noqa: E402

WORKLOAD = "full_1024x256x256"
METRIC = "phase-space cell-updates/s"
UNIT = "cell-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(synth.WORKLOADS))
    ap.add_argument("--no-side", action="store_true", help="skip the side-by-side precision")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end measurement")
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="steps of the end-to-end run (0: the workload's own step count, "
                         "at most 20000)")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the batched parameter sweep (sweep_256) in the default line")
    ap.add_argument("--sweep-steps", type=int, default=200,
                    help="timed batch steps of the sweep_256 measurement")
    ap.add_argument("--no-batch", action="store_true",
                    help="step each instance alone instead of as one batch")
    ap.add_argument("--chunk-len", type=int, default=0,
                    help="planes per x-chunk of every instance instead of the autotuner's choice "
                         "(for profiling runs, where the tuner's timing trials are distorted)")
    ap.add_argument("--collisions", action="store_true",
                    help="switch on the BGK collision term (Eqs. 3-5; T_e 2 eV, ln Lambda 10)")
    ap.add_argument("--reflection", type=float, default=0.0,
                    help="electron reflection coefficient R_f at the wall")
    ap.add_argument("--scheme", default="unsplit", choices=["unsplit", "lie", "strang"],
                    help="time scheme (the split schemes step each instance alone)")
    ap.add_argument("--tile-rows", type=int, default=-1,
                    help="v1-row cap of every instance's whole-CTA tiles (0: the default "
                         "tiles) instead of the autotuner's tile search (-1)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_over_ranks(value, dist, op="max"):
    """Max (time) or sum (throughput) of a per-rank float over the process
    group; the value itself when there is no group."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t[0])


def job_throughput(world, n_inst, cells, steps, ms_max):
    """Whole-job cell-updates/s: every rank advanced its own n_inst instances
    by `steps` steps; the job took the slowest rank's time."""
    return world * n_inst * cells * steps / (ms_max / 1e3)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def kernel_traffic(workload, precision):
    """Per-launch DRAM bytes of the dominant step kernel of `workload` at
    `precision` from the committed ncu summaries, if there is a record for
    that pair and its source hash matches the current kernel source."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.txt")
    if not os.path.exists(path):
        return None
    from paper_2303_14119_gb300 import _build
    vals = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_hash") != _build.source_hash():
        return None
    key = "%s_%s" % (workload, precision)
    return float(vals[key]) if key in vals else None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        smax = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if r[4 + q] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------- our arm
SCHEMES = {"unsplit": 0, "lie": 1, "strang": 2}
PASSES = {"unsplit": 1, "lie": 2, "strang": 3}  # passes over f per step


def make_grids(fk, w, precision, stream, phys=None):
    """The workload's instances; phys: optional terms of Eq. 2 and the wall
    (collisions, reflection) and the time scheme."""
    grids = []
    for Ey in w.get("Ey_sweep", (w["Ey"],)):
        g = fk.Grid(w["nx"], w["nv1"], w["nv2"], w["h_max"], -w["v1_span"], w["v1_span"],
                    -w["v2_span"], w["v2_span"], cfl=w["cfl"], precision=precision,
                    stream=stream)
        g.set_fields(Ey)
        g.set_see(w["delta_max"], w["A_max"], w["k_s"], w["T_se"])
        g.set_source(w["J"], w["x_lo"], w["x_hi"], w["T_fe"])
        if phys:
            if phys["collisions"]:
                g.set_collisions(2.0, 10.0, True)
            if phys["reflection"] > 0.0:
                g.set_reflection(phys["reflection"])
            if phys["scheme"] != "unsplit":
                g.set_scheme(SCHEMES[phys["scheme"]])
        grids.append(g)
    return grids


def time_arm(fk, torch, w, precision, f0, steps, warmup, dist, device, batch=True,
             kernel_steps=50, chunk_len=0, tile_rows=-1, phys=None):
    """Time `steps` steps of the workload's instances after `warmup` steps,
    as users run them: each step a CUDA-graph replay (batch: one step-kernel
    launch per unit layout and one finalize launch for all instances, x-chunks
    and v1 tiles autotuned before the warm-up; else each instance's own
    graph).  chunk_len > 0 pins the x-chunks, tile_rows >= 0 the tile-row cap
    (0: the default tiles), each instead of the autotuner's choice.  The
    step kernel's own launch durations (CUDA events around each launch,
    direct launches) are taken in a separate pass of `kernel_steps` steps
    after the timed region, for the roofline."""
    # every grid runs on torch's current stream (a created stream, not the
    # legacy default), so the events below bracket exactly the grids' work
    stream = torch.cuda.current_stream().cuda_stream
    assert stream, "time_arm needs a non-default current stream"
    grids = make_grids(fk, w, precision, stream, phys)
    for g in grids:
        if tile_rows >= 0:
            g.set_tile_rows(tile_rows)
        g.set_f(f0)
    b = fk.Batch(grids, stream) if batch else None
    tuned = 0
    if b is not None:
        if chunk_len > 0:
            b.set_chunks([chunk_len] * len(grids))
        else:
            # four steps per trial: the tile plans differ by about 1 %
            tuned = b.autotune(4, tiles=tile_rows < 0)

    def advance(n):
        if b is not None:
            b.step(n)
        else:
            for g in grids:
                g.step(n)

    advance(warmup)
    if b is not None:
        assert b.sync() == [fk.FK_OK] * len(grids)
    else:
        for g in grids:
            g.sync()
    clocks = ClockSampler(device)
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    if b is not None:
        b.step(steps)
    else:
        for _ in range(steps):
            for g in grids:
                g.step(1)
    e1.record()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    ck = clocks.stop()
    # the step kernel's launch durations, in a pass of their own
    if b is not None:
        b.set_kernel_timing(True)
    else:
        for g in grids:
            g.set_kernel_timing(True)
    advance(kernel_steps)
    cells = w["nx"] * w["nv1"] * w["nv2"]
    if b is not None:
        launches, kms = b.kernel_timing()
        b.set_kernel_timing(False)
        assert b.sync() == [fk.FK_OK] * len(grids)
        info = b.info()
        ginfo = grids[0].info()
        plan = dict(mode="batch", units=info["units"], smem_bytes=info["smem_bytes"],
                    ctas_per_sm=info["ctas_per_sm"], chunk_len=b.chunks(),
                    n_tiles=ginfo["n_tiles"], tile_rows=ginfo["tile_rows"],
                    tile_cap=[g.info()["tile_cap"] for g in grids], autotune_steps=tuned,
                    timed="CUDA-graph replay (32 steps per graph)",
                    kernel_times="CUDA events around each step-kernel launch, separate "
                                 "pass of %d direct-launched steps" % kernel_steps)
        cells_per_launch = cells * len(grids)
        gpu_launches = (info["step_launches"] + 1) * steps  # step kernel(s) + finalize
        b.close()
    else:
        launches, kms = 0, 0.0
        for g in grids:
            n, t = g.kernel_timing()
            launches += n
            kms += t
            g.set_kernel_timing(False)
            g.sync()
        info = grids[0].info()
        plan = dict(mode="per-instance", timed="CUDA-graph replay per instance",
                    **{k: info[k] for k in ("kernel", "n_tiles", "n_chunks", "chunk_len")})
        cells_per_launch = cells
        # per step: the pass(es), the Strang mid-step fold, the finalize
        scheme = phys["scheme"] if phys else "unsplit"
        per_step = {"unsplit": 2, "lie": 3, "strang": 5}[scheme]
        gpu_launches = per_step * steps * len(grids)
    return dict(ms=ms, launches=launches, kernel_ms=kms, cells=cells, n_inst=len(grids),
                cells_per_launch=cells_per_launch, gpu_launches=gpu_launches, clocks=ck,
                grids=grids, kernel=plan)


def e2e_arm(fk, torch, w, precision, f0_pinned, steps, batch=True, plan=None, phys=None):
    """The user's loop through the C ABI with host buffers: upload f0 from
    pinned host memory, then per step advance (the instances as one batch,
    or each alone) and read n_e, E_x, sigma and the wall fluxes back (the
    batch: queued into pinned slots, step n's read while step n + 1 runs),
    finally read f back; all inside the timed region.  plan: the batch's
    x-chunks and tile caps (as time_arm's autotuner left them), set up
    before the timed region."""
    stream = torch.cuda.current_stream().cuda_stream
    assert stream, "e2e_arm needs a non-default current stream"
    grids = make_grids(fk, w, precision, stream, phys)
    if batch and plan is not None:
        for g, cap in zip(grids, plan["tile_cap"]):
            g.set_tile_rows(cap)
    nx = w["nx"]
    # an FP32 grid exchanges f with the host in its own storage type
    f32 = precision == fk.FK_F32
    if f32:
        f_host = torch.empty(f0_pinned.shape, dtype=torch.float32, pin_memory=True).numpy()
        f_host[...] = f0_pinned
    else:
        f_host = f0_pinned
    out_f = torch.empty(f0_pinned.shape, dtype=torch.float32 if f32 else torch.float64,
                        pin_memory=True).numpy()
    ne = np.empty(nx)
    ex = np.empty(nx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g in grids:
        if f32:
            g.set_f32(f_host)
        else:
            g.set_f(f_host)
    b = fk.Batch(grids, stream) if batch else None
    if b is not None and plan is not None:
        b.set_chunks(plan["chunk_len"])
    ne_all = np.empty(nx * len(grids))
    ex_all = np.empty(nx * len(grids))
    slot = 0
    for q in range(steps):
        if b is not None:
            # one step of every instance, then every instance's n_e, E_x,
            # sigma and wall fluxes queued for read-back into a pinned slot;
            # the previous step's are collected while this step runs
            b.step(1)
            b.moments_enqueue(slot)
            if q > 0:
                b.moments_collect(slot ^ 1, ne_all, ex_all)
            slot ^= 1
        else:
            for g in grids:
                g.step(1)
                fk.fk_moments(g.h, nx, ne, ex)
                g.surface_charge()
    if b is not None and steps > 0:
        b.moments_collect(slot ^ 1, ne_all, ex_all)  # the last step's
    for g in grids:
        if f32:
            g.get_f32(out_f)
        else:
            g.get_f(out_f)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    if b is not None:
        b.close()
    for g in grids:
        g.close()
    cells = w["nx"] * w["nv1"] * w["nv2"]
    n = len(grids)
    h2d = n * f_host.nbytes / steps
    d2h = n * (2 * nx * 8 + 3 * 8) + n * out_f.nbytes / steps
    return dict(value=n * cells * steps / dt, unit=UNIT, h2d_bytes_per_step=int(h2d),
                d2h_bytes_per_step=int(d2h), steps=steps)


def oracle_rate(w, threads, seconds):
    """Cell-updates/s of the FP64 oracle on `threads` host threads (None: the
    serial checker build), over as many whole steps of one field instance
    of the workload as fit in about `seconds` (at least one)."""
    import oracle
    shape = (w["nx"], w["nv1"], w["nv2"])
    o = oracle.Oracle(*shape, w["h_max"], -w["v1_span"], w["v1_span"], -w["v2_span"],
                      w["v2_span"], cfl=w["cfl"], threads=threads)
    o.set_fields(w["Ey"])
    o.set_see(w["delta_max"], w["A_max"], w["k_s"], w["T_se"])
    o.set_source(w["J"], w["x_lo"], w["x_hi"], w["T_fe"])
    o.set_state(synth.initial_f(shape, w["seed"], w["noise_rel"], w["J"], w["T_fe"]), 0.0)
    cells = int(np.prod(shape))
    n, t = 0, 0.0
    while t < seconds or n == 0:
        t0 = time.perf_counter()
        o.step(1)
        t += time.perf_counter() - t0
        n += 1
        if n * cells > 4e9:
            break
    used = o.threads
    o.close()
    return n * cells / t, n, used


def cpu_baseline(w, seconds=10.0):
    """The FP64 oracle as it stands on the host: its OpenMP build on every
    host core (loops over x-planes threaded, sums in plane order) and its
    serial build on one core, each on a bounded sample of the workload."""
    shape = (w["nx"], w["nv1"], w["nv2"])
    cores = os.cpu_count() or 1
    v_all, n_all, used = oracle_rate(w, cores, seconds)
    v_one, n_one, _ = oracle_rate(w, None, seconds)
    return {"value": v_all, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": "%d step(s) of one %dx%dx%d field instance (E_y=%g V/m), FP64, %d threads "
                      "(OpenMP over x-planes) of %d host cores"
                      % (n_all, *shape, w["Ey"], used, cores),
            "one_core": {"value": v_one, "unit": UNIT, "cores": 1,
                         "sample": "%d step(s), serial build" % n_one}}


# GB300 FP64 FMA peak derived from unit counts and clock: 152 SMs x 2 FP64
# FMA per cycle x 2.07 GHz = 0.629 T FMA/s = 1.26 TFLOP/s (NVIDIA's figure is
# 1.25 TFLOP/s; a register-resident FMA loop measured 0.596 T FMA/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2.07e9 * 2 / 1e12
DFMA_PER_CELL = 4  # the FP64 update is four fused multiply-adds per cell


def roofline(res, precision, peak, peak_kind, workload, passes=1, plain=True):
    """passes: passes over f per timed launch (one read of f and one write
    each; the split schemes' passes are timed together); plain: the
    workload's default physics, the only case the traffic record covers."""
    bpc = 4 if precision == "f32" else 8
    if res["launches"] == 0:
        return None
    avg_s = res["kernel_ms"] / res["launches"] / 1e3
    alg_bytes = passes * 2 * bpc * res["cells_per_launch"]  # one read of f^n, one write of f^{n+1}
    achieved = alg_bytes / avg_s / 1e9
    hbm = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
           "frac": round(achieved / peak, 4),
           "traffic": kernel_traffic(workload, precision) if plain else None,
           "peak_kind": "%s (copy bandwidth)" % peak_kind,
           "kernel": "fused upwind step", "avg_launch_us": round(avg_s * 1e6, 2),
           "alg_bytes_per_launch": alg_bytes}
    if precision == "f32":
        return hbm
    # FP64 on GB300 is bound by the FP64 pipe, not by HBM (every pass of a
    # split step runs the fused update, four DFMA per cell)
    flops = passes * 2 * DFMA_PER_CELL * res["cells_per_launch"]
    tflops = flops / avg_s / 1e12
    return {"bound": "alu", "achieved": round(tflops, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
            "unit": "TFLOP/s", "frac": round(tflops / FP64_PEAK_TFLOPS, 4),
            "traffic": hbm["traffic"], "peak_kind": "derived (FP64 FMA units x clock)",
            "kernel": "fused upwind step", "avg_launch_us": hbm["avg_launch_us"],
            "alg_flops_per_launch": flops,
            "hbm": {k: hbm[k] for k in ("achieved", "peak", "unit", "frac")}}


def run_ours(args):
    rank, world, local = dist_env()
    import torch
    from paper_2303_14119_gb300 import fk
    fk.load()
    torch.cuda.set_device(local)
    torch.cuda.set_stream(torch.cuda.Stream())
    dist = None
    if world > 1:
        import torch.distributed as td
        td.init_process_group("gloo")
        dist = td
    w = synth.WORKLOADS[args.workload]
    shape = (w["nx"], w["nv1"], w["nv2"])
    f0 = torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
    f0[...] = synth.initial_f(shape, w["seed"], w["noise_rel"], w["J"], w["T_fe"])
    peak, peak_kind = measured_peaks()
    prec = fk.FK_F32 if args.precision == "f32" else fk.FK_F64
    phys = dict(collisions=args.collisions, reflection=args.reflection, scheme=args.scheme)
    plain = not args.collisions and args.reflection == 0.0 and args.scheme == "unsplit"
    # batches step the unsplit scheme only: a split scheme steps each instance alone
    batch = not args.no_batch and args.scheme == "unsplit"
    passes = PASSES[args.scheme]
    res = time_arm(fk, torch, w, prec, f0, args.steps, args.warmup, dist, local,
                   batch=batch, chunk_len=args.chunk_len, tile_rows=args.tile_rows, phys=phys)
    for g in res.pop("grids"):
        g.close()
    ms = reduce_over_ranks(res["ms"], dist, "max")
    value = job_throughput(world, res["n_inst"], res["cells"], args.steps, ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": "%s, E_y sweep %s V/m (%d instances per step)"
                               % (args.workload, list(w.get("Ey_sweep", (w["Ey"],))), res["n_inst"]),
                   "cells_per_instance": res["cells"], "precision_storage": args.precision,
                   "accumulators": "f64", "l2": "inputs larger than L2 (no flush)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline(res, args.precision, peak, peak_kind, args.workload, passes, plain),
        "kernel_plan": res["kernel"],
        "gpu_launches": res["gpu_launches"],
        "clocks": res["clocks"],
    }
    if not plain:
        line["config"]["physics"] = dict(
            collisions="BGK, T_e 2 eV, ln Lambda 10" if args.collisions else "off",
            reflection=args.reflection, scheme=args.scheme,
            passes_per_step=passes, timed_launches=("the step kernel" if passes == 1 else
                                                    "the %d passes of a step together" % passes))
    if not args.no_side:
        other = "f64" if args.precision == "f32" else "f32"
        oprec = fk.FK_F64 if other == "f64" else fk.FK_F32
        osteps = max(1, args.steps // (2 if other == "f64" else 1))
        r2 = time_arm(fk, torch, w, oprec, f0, osteps, args.warmup, dist, local,
                      batch=batch, phys=phys)
        for g in r2.pop("grids"):
            g.close()
        line["side_by_side"] = {other: {
            "value": world * r2["n_inst"] * r2["cells"] * osteps / (r2["ms"] / 1e3),
            "ms_per_step": r2["ms"] / osteps, "steps": osteps,
            "roofline": roofline(r2, other, peak, peak_kind, args.workload, passes, plain),
            "clocks": r2["clocks"]}}
    if not args.no_e2e:
        e2e_steps = args.e2e_steps or min(int(w.get("steps", 100)), 20000)
        e2e = e2e_arm(fk, torch, w, prec, f0, e2e_steps, batch=batch,
                      plan=res["kernel"] if batch else None, phys=phys)
        e2e["value"] = reduce_over_ranks(e2e["value"], dist, "sum")
        line["e2e"] = e2e
    if not args.no_sweep:
        # the second half of the metric: batched instances/hr of the sweep
        # against the same instances stepped one after another
        sw = measure_sweep(fk, torch, "sweep_256", args.precision, args.sweep_steps,
                           max(3, min(args.warmup, 10)), dist, local, world)
        line["batched_sweep"] = {k: sw[k] for k in (
            "metric", "value", "unit", "ms_per_step", "steps", "config", "cell_updates_per_s",
            "sequential", "speedup_vs_sequential", "equal_accuracy", "autotune", "roofline",
            "clocks")}
        line["gpu_launches_batched_sweep"] = sw["gpu_launches"]
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(w)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def make_sweep_grids(fk, instances, precision, stream):
    """One grid per sweep instance, f0 = 0 and sigma = 0 (the run starts
    from an uncharged, empty gap)."""
    grids = []
    for p in instances:
        g = fk.Grid(p["nx"], p["nv1"], p["nv2"], p["h_max"], -p["v1_span"], p["v1_span"],
                    -p["v2_span"], p["v2_span"], cfl=p["cfl"], precision=precision,
                    stream=stream)
        g.set_fields(p["Ey"])
        g.set_see(p["delta_max"], p["A_max"], p["k_s"], p["T_se"])
        g.set_source(p["J"], p["x_lo"], p["x_hi"], p["T_fe"])
        grids.append(g)
    return grids


def measure_sweep(fk, torch, workload, precision, steps, warmup, dist, local, world=1):
    """Batched workload: every instance of the parameter sweep
    (synth.sweep_instances) or of the surrogate's training runs
    (synth.surrogate_runs) stepped as one batch (x-chunks autotuned per size
    bucket), against the same instances stepped one after another with
    fk_step (each instance's steps as CUDA-graph replays).  Both arms give
    bitwise identical states; the metric is instances per hour at the
    workload's steps per instance, from the timed per-step rate.  Returns
    the JSON object of the measurement."""
    stream = torch.cuda.current_stream().cuda_stream
    w = synth.WORKLOADS[workload]
    ins = synth.batch_instances(w)
    prec = fk.FK_F32 if precision == "f32" else fk.FK_F64
    grids = make_sweep_grids(fk, ins, prec, stream)
    twins = make_sweep_grids(fk, ins, prec, stream)
    cells = float(sum(p["nx"] * p["nv1"] * p["nv2"] for p in ins))
    b = fk.Batch(grids, stream)
    t0 = time.perf_counter()
    tuned = b.autotune(2)
    tune_s = time.perf_counter() - t0
    b.step(warmup)
    # kernel durations for the roofline (direct launches with event pairs)
    kt_steps = 8
    b.set_kernel_timing(True)
    b.step(kt_steps)
    launches, kms = b.kernel_timing()
    b.set_kernel_timing(False)
    pre = tuned + warmup + kt_steps
    assert b.sync() == [fk.FK_OK] * len(ins)
    # batched arm: graph replay
    clocks = ClockSampler(local)
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    b.step(steps)
    e1.record()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms_b = reduce_over_ranks(e0.elapsed_time(e1), dist, "max")
    ck = clocks.stop()
    st_b = b.sync()
    # sequential arm: the twins reach the same step untimed, then each
    # instance runs its timed steps alone, one instance after another
    for g in twins:
        g.step(pre)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    e0.record()
    for g in twins:
        g.step(steps)
    e1.record()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms_s = reduce_over_ranks(e0.elapsed_time(e1), dist, "max")
    # equal accuracy: identical states (sigma of every instance, f of a few)
    same_sigma = sum(int(ga.surface_charge() == gb.surface_charge())
                     for ga, gb in zip(grids, twins))
    checks = list(range(0, len(ins), max(1, len(ins) // 8)))
    same_f = sum(int(np.array_equal(grids[q].get_f(), twins[q].get_f())) for q in checks)
    info = b.info()
    chunks = b.chunks()
    b.close()
    for g in grids + twins:
        g.close()
    per_inst = w["steps"]
    if "sweep" in w:
        workload_text = ("%s: %d instances, nx 128-512, nv1 = nv2 64-192, E_y log-uniform "
                         "3e5-5e6 V/m, delta_max 2-4, A_max 250-600 eV, T_se 1-5 eV, one seed "
                         "(%d); f0 = 0" % (workload, len(ins), w["seed"]))
    else:
        workload_text = ("%s: %d surrogate training runs of 64 x 48 x 48, E_y log-uniform "
                         "3e5-5e6 V/m, delta_max 2-4, A_max 250-600 eV, T_se 1-5 eV, J "
                         "log-uniform 1e5-1e7 A/m^2, h_max 16-24 um, one seed (%d); f0 = 0; "
                         "%d steps reach the 1.25 ns horizon at the smallest gap"
                         % (workload, len(ins), w["seed"], per_inst))
    ms_step_b = ms_b / steps
    ms_step_s = ms_s / steps
    value = world * len(ins) * 3600.0 / (ms_step_b * per_inst / 1e3)
    seq = world * len(ins) * 3600.0 / (ms_step_s * per_inst / 1e3)
    peak, peak_kind = measured_peaks()
    res = dict(launches=launches, kernel_ms=kms, cells_per_launch=cells)
    roof = roofline(res, precision, peak, peak_kind, workload)
    if roof is not None:
        if info["step_launches"] == 1:
            roof["kernel"] = "batched fused upwind step (all %d instances per launch)" % len(ins)
        else:  # whole-CTA and half-CTA units: two launches, timed together per step
            roof["kernel"] = ("batched fused upwind step (all %d instances per step: one launch "
                              "of whole-CTA units, one of half-CTA units, timed together)"
                              % len(ins))
            roof["traffic"] = None  # a record covers one launch
    return {
        "metric": "batched instances/hr (%d steps per instance)" % per_inst, "value": value,
        "unit": "instances/hr", "n_gpus": world, "steps": steps, "warmup": warmup,
        "ms_per_step": ms_step_b, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": precision, "data": "synthetic",
        "config": {"workload": workload_text,
                   "cells_all_instances": cells, "steps_per_instance": per_inst,
                   "rate": "instances/hr from the timed per-step time x %d steps" % per_inst,
                   "l2": "inputs larger than L2 (no flush)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "cell_updates_per_s": world * cells * steps / (ms_b / 1e3),
        "sequential": {"value": seq, "unit": "instances/hr", "ms_per_step": ms_step_s,
                       "cell_updates_per_s": world * cells * steps / (ms_s / 1e3),
                       "how": "fk_step(n) per instance, one instance after another"},
        "speedup_vs_sequential": ms_s / ms_b,
        "equal_accuracy": {"sigma_bitwise_identical": "%d/%d" % (same_sigma, len(ins)),
                           "f_bitwise_identical": "%d/%d checked" % (same_f, len(checks)),
                           "status_ok": "%d/%d" % (st_b.count(fk.FK_OK), len(ins))},
        "autotune": {"steps": tuned, "seconds": round(tune_s, 3), "buckets": info["buckets"],
                     "units_per_launch": info["units"],
                     "chunk_len_range": [min(chunks), max(chunks)]},
        "roofline": roof,
        "gpu_launches": (info["step_launches"] + 1) * steps,  # step kernel(s) + finalize
        "clocks": ck,
    }


def run_sweep(args):
    """A batched workload as the benchmark's own line (--workload)."""
    rank, world, local = dist_env()
    import torch
    from paper_2303_14119_gb300 import fk
    fk.load()
    torch.cuda.set_device(local)
    torch.cuda.set_stream(torch.cuda.Stream())
    dist = None
    if world > 1:
        import torch.distributed as td
        td.init_process_group("gloo")
        dist = td
    line = measure_sweep(fk, torch, args.workload, args.precision, args.steps, args.warmup,
                         dist, local, world)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_reference(args):
    """The oracle arm: each step is one FP64 oracle step of one field
    instance of the workload (a bounded sample), on every host core (the
    oracle's OpenMP build: loops over x-planes threaded, sums in plane
    order, bitwise equal to its serial build)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    w = synth.WORKLOADS[args.workload]
    if "sweep" in w or "runs" in w:  # the sampled instance: the batch's first
        w = synth.batch_instances(w)[0]
    shape = (w["nx"], w["nv1"], w["nv2"])
    cores = os.cpu_count() or 1
    o = oracle.Oracle(*shape, w["h_max"], -w["v1_span"], w["v1_span"], -w["v2_span"],
                      w["v2_span"], cfl=w["cfl"], threads=cores)
    o.set_fields(w["Ey"])
    o.set_see(w["delta_max"], w["A_max"], w["k_s"], w["T_se"])
    o.set_source(w["J"], w["x_lo"], w["x_hi"], w["T_fe"])
    o.set_state(synth.initial_f(shape, w["seed"], w["noise_rel"], w["J"], w["T_fe"]), 0.0)
    steps = max(1, min(args.steps, 20))
    warm = max(0, min(args.warmup, 1))
    o.step(warm)
    t0 = time.perf_counter()
    o.step(steps)
    t = time.perf_counter() - t0
    cells = int(np.prod(shape))
    value = cells * steps / t
    used = o.threads
    o.close()
    sample = ("%d FP64 oracle step(s) of one %dx%dx%d field instance, %d threads (OpenMP over "
              "x-planes) of %d host cores" % (steps, *shape, used, cores))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": warm, "ms_per_step": t / steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "cells_per_instance": cells},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif any(k in synth.WORKLOADS[args.workload] for k in ("sweep", "runs")):
        run_sweep(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
