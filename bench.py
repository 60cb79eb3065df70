"""Benchmark of the GB300 CoRdE stepper; prints ONE JSON line on rank 0.

Headline (``value``): device time per simulated time step of one 512-element
inextensible guidewire rod (10 constraint iterations, dt = 1e-4 s) stepped 10 time steps
per persistent launch with a seeded 1 kHz insertion/twist drive (the paper's Section 3.3
instrument; metric "us/step 512-elem rod (10 steps/launch)").  One bench step is 100
launches = 1000 time steps = 0.1 s of simulated time.  L2 is flushed (a 256 MiB write)
between bench steps, outside the timed intervals.

Also reported: ``e2e`` (the haptic loop through the C ABI with host buffers, host wall
clock: one persistent launch in lock-step; per tick the host writes the drive into
mapped pinned memory, the kernel runs 10 steps and publishes all node positions to
pinned host memory, the host copies them; beside it a launch per tick through
rod_step_io, with explicit copies, and the asynchronous mailbox loop), ``latency``
(against the measured empty-barrier floors, with and without launch overlap),
``roofline`` of the step kernel, ``cpu_baseline`` (the FP64 oracle on the host cores,
one core, as the paper's serial CPU version), ``batched`` (4096 rods of log-uniform
length in [16, 2048], element-steps/s and its rooflines), ``adjoint`` (adjoint/forward
time), ``pair``, ``long_rods``, ``vessel_contact`` and ``self_collision``.

``--impl reference`` times the FP64 CPU oracle on the same workload and metric.
For N > 1 (torchrun) every rank runs its own replica of the single-rod workload and the
batched workload sharded by rods (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "µs/step 512-elem rod (10 steps/launch); batched element-steps/s; adjoint/fwd"
UNIT = "us/step"
STEPS_PER_LAUNCH = 10
LAUNCHES_PER_BENCH_STEP = 100

# Algorithmic FP32 operations per element per time step (adds, multiplies, divides,
# square roots of the method as stated, counted by the oracle's op-counting scalar):
# inextensible rod 293 + 41 per constraint iteration; extensible rod 306.
FLOPS_PER_EL_STEP_BASE = 293.0
FLOPS_PER_EL_ITER = 41.0
# Algorithmic HBM bytes per element per launch: state read + written (r, w, v, q, omega:
# 4 float4 = 64 B each way) plus the per-joint parameters read (u-hat, K: 32 B).
BYTES_PER_EL_LAUNCH = 64 + 64 + 32


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", "-i", str(self.gpu),
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
               "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
               "clocks_event_reasons.sw_power_cap",
               "--format=csv,noheader,nounits", "-lms", "100"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[3 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _kernel_source_hash():
    h = hashlib.sha256()
    for f in ("corde_step.cuh", "corde_common.cuh"):
        with open(os.path.join(ROOT, "paper_2509_04277_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(kernel_key):
    """DRAM bytes per launch from the committed ncu summary, if taken on this kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None, None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel_key)
    if not e or e.get("source_hash") != _kernel_source_hash():
        return None, None
    return e.get("dram_bytes_per_launch"), e.get("units_per_launch")


def measure_fp32_peak(corde):
    """The device's FP32 FMA throughput, measured by the library's micro-benchmark
    (rod_fp32_peak): every SM full of independent FMA chains, plain and through the
    paired-lane FMA.  Burst: best of three short launches (~10 ms), the peak for a kernel
    timed alone; sustained: one launch of about two seconds, the peak for a kernel timed
    inside a long step."""
    info = corde.rod_device_info()
    burst = {}
    for packed in (False, True):
        burst["packed" if packed else "scalar"] = max(corde.rod_fp32_peak(packed, 4, 512, 20000) for _ in range(3))
    best = max(burst, key=burst.get)
    t0 = time.perf_counter()
    sustained = corde.rod_fp32_peak(best == "packed", 4, 512, 8_000_000)
    return {"burst_tflops": round(burst[best], 3), "sustained_tflops": round(sustained, 3),
            "by_form_tflops": {k: round(v, 3) for k, v in burst.items()}, "n_sms": info["n_sms"],
            "sustained_seconds": round(time.perf_counter() - t0, 2),
            "how": "rod_fp32_peak: 4 blocks of 512 threads per SM, 8 independent FMA chains per thread "
                   "(scalar FMA, and float2 through the paired-lane FMA); CUDA events; best form"}


def flops_per_el_step(n_iters: int, inextensible: bool = True) -> float:
    if not inextensible:
        return 306.0
    return FLOPS_PER_EL_STEP_BASE + FLOPS_PER_EL_ITER * n_iters


# --------------------------------------------------------------------------- our arm


def run_single_rod(args, torch, corde, W, rank):
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    rod = W.guidewire(512, seed=2 + rank)
    n_launch_total = LAUNCHES_PER_BENCH_STEP * (args.warmup + args.steps)
    drive_np = W.sinusoid_drive(2 + rank, n_launch_total, STEPS_PER_LAUNCH * rod.dt).astype(np.float32)
    drive = torch.as_tensor(drive_np, device=dev).contiguous()
    b = corde.RodBatch([rod])
    if args.no_autotune:
        b.set_plan(2, 256)
    else:
        b.autotune(STEPS_PER_LAUNCH)
    plan = [int(x) for x in b.plan()[0][:2]]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def bench_step(k, events=None):
        for j in range(LAUNCHES_PER_BENCH_STEP):
            row = drive[k * LAUNCHES_PER_BENCH_STEP + j]
            if events is not None:
                events[j][0].record(stream)
            b.step(STEPS_PER_LAUNCH, drive=row)
            if events is not None:
                events[j][1].record(stream)

    for k in range(args.warmup):
        bench_step(k)
    torch.cuda.synchronize()
    brackets = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
    clocks = ClockSampler(torch.cuda.current_device())
    if rank == 0:
        clocks.start()
    _barrier(torch)
    torch.cuda.synchronize()
    launches = 0
    for k in range(args.steps):
        flush.fill_(float(k))
        brackets[k][0].record(stream)
        bench_step(args.warmup + k)
        brackets[k][1].record(stream)
        launches += LAUNCHES_PER_BENCH_STEP * b.last_launch_count()
    torch.cuda.synchronize()
    _barrier(torch)
    clk = clocks.stop() if rank == 0 else None
    total_ms = sum(s.elapsed_time(e) for s, e in brackets)
    # per-launch durations, bracketed one by one in an extra untimed bench step (the
    # events between launches add gaps, so they stay out of the timed region)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(LAUNCHES_PER_BENCH_STEP)]
    bench_step(args.warmup + args.steps - 1, ev)
    torch.cuda.synchronize()
    kern_ms = [s.elapsed_time(e) for s, e in ev]
    us_per_step = total_ms * 1e3 / (args.steps * LAUNCHES_PER_BENCH_STEP * STEPS_PER_LAUNCH)
    # context, untimed: the same launches without launch overlap (each kernel is scheduled
    # only after the previous one has ended)
    b.set_launch_overlap(False)
    e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_a.record(stream)
    bench_step(args.warmup + args.steps - 1)
    e_b.record(stream)
    torch.cuda.synchronize()
    no_overlap_us = e_a.elapsed_time(e_b) * 1e3 / (LAUNCHES_PER_BENCH_STEP * STEPS_PER_LAUNCH)
    b.set_launch_overlap(True)
    rc, diag = b.diagnostics()

    # e2e: the haptic loop through the C ABI with host buffers.  One call per tick
    # (rod_step_io): the kernel reads the drive from pinned host memory and writes the
    # positions after its last step to pinned host memory; then the host waits.
    pin_drive = torch.empty((1, 8), dtype=torch.float32, pin_memory=True)
    pin_pos = torch.empty((512, 4), dtype=torch.float32, pin_memory=True)
    n_e2e = LAUNCHES_PER_BENCH_STEP * max(1, args.steps)
    host_drive = drive_np
    pd = pin_drive.numpy()

    def tick_io(j):
        pd[0] = host_drive[j % host_drive.shape[0]]
        corde.rod_step_io(b.handle, STEPS_PER_LAUNCH, pin_drive, pin_pos, stream)
        stream.synchronize()

    def tick_copies(j):
        pd[0] = host_drive[j % host_drive.shape[0]]
        corde.rod_set_input(b.handle, pin_drive, stream)
        b.step(STEPS_PER_LAUNCH)
        corde.rod_get_state(b.handle, pin_pos, None, None, None, stream)
        stream.synchronize()

    e2e = {}
    for name, tick in (("io", tick_io), ("copies", tick_copies)):
        for j in range(20):
            tick(j)
        t0 = time.perf_counter()
        for j in range(n_e2e):
            tick(j)
        e2e[name] = (time.perf_counter() - t0) * 1e6 / n_e2e
    e2e_us = e2e["io"] / STEPS_PER_LAUNCH

    # The paper's asynchronous haptic loop: one persistent launch; every tick the host
    # writes the drive into the mailbox and pulls the newest snapshot of all positions,
    # which the kernel publishes every 10 steps without waiting for the host.
    n_ticks = n_e2e
    corde.rod_mailbox_enable(b.handle, STEPS_PER_LAUNCH, 64)
    corde.rod_mailbox_positions_enable(b.handle)
    snap = np.zeros((512, 4), np.float32)
    # snapshot steps count from the handle's first step: the launch ends at base + its steps
    total_steps = corde.rod_steps_done(b.handle) + (n_ticks + 40) * STEPS_PER_LAUNCH
    b.step((n_ticks + 40) * STEPS_PER_LAUNCH)
    first = last = -1
    t_first = t_last = 0.0
    ticks = 0
    t_limit = time.perf_counter() + 60.0
    while ticks < n_ticks + 20 and last < total_steps and time.perf_counter() < t_limit:
        corde.rod_mailbox_write(b.handle, host_drive[ticks % host_drive.shape[0]].reshape(1, 8))
        s = corde.rod_mailbox_positions(b.handle, 0, snap)
        while s <= last and s < total_steps and time.perf_counter() < t_limit:
            s = corde.rod_mailbox_positions(b.handle, 0, snap)
        last = s
        ticks += 1
        if ticks == 20:
            first, t_first = s, time.perf_counter()
    t_last = time.perf_counter()
    stream.synchronize()
    corde.rod_mailbox_disable(b.handle)
    persistent = {"ticks": ticks, "first": first, "last": last}
    if first > 0 and last > first:
        persistent = {"us_per_step": (t_last - t_first) * 1e6 / (last - first), "ticks": ticks - 20,
                      "steps": last - first}

    # Lock-step persistent loop: the kernel waits (bounded) at every 10th step for the
    # host's next drive; the host writes drive 0, then per tick k one native call waits
    # for the snapshot after tick k's 10 steps, writes drive k + 1 and reads all positions.
    corde.rod_mailbox_enable(b.handle, STEPS_PER_LAUNCH, 64)
    corde.rod_mailbox_positions_enable(b.handle)
    corde.rod_mailbox_lockstep(b.handle, True, 2_000_000)
    base = corde.rod_steps_done(b.handle)
    b.step((n_ticks + 20) * STEPS_PER_LAUNCH)
    t_start, done = None, 0
    corde.rod_mailbox_write(b.handle, host_drive[0].reshape(1, 8))
    for k in range(n_ticks + 20):
        target = base + (k + 1) * STEPS_PER_LAUNCH
        # the next tick's drive goes out as soon as this tick's snapshot is seen, so the
        # kernel steps while the host copies
        nxt = host_drive[(k + 1) % host_drive.shape[0]].reshape(1, 8) if k + 1 < n_ticks + 20 else None
        try:
            s = corde.rod_mailbox_tick(b.handle, 0, target, nxt, snap, 10_000_000)
        except corde.CordeError:
            break
        if s != target:
            break
        done += 1
        if k == 19:
            t_start = time.perf_counter()
    t_end = time.perf_counter()
    stream.synchronize()
    lock_status = corde.rod_mailbox_status(b.handle)
    corde.rod_mailbox_disable(b.handle)
    lockstep = {"ticks": done, "status": lock_status}
    if t_start is not None and done == n_ticks + 20:
        lockstep = {"us_per_step": (t_end - t_start) * 1e6 / (n_ticks * STEPS_PER_LAUNCH),
                    "per_tick_us": (t_end - t_start) * 1e6 / n_ticks, "ticks": n_ticks, "status": lock_status}
    b.close()
    # empty-barrier floors of each scope (the step kernel uses block barriers)
    floors = {
        "block_ns": corde.rod_barrier_floor(0, threads=plan[1], n_iters=200000),
        "warp_ns": corde.rod_barrier_floor(1, n_iters=200000),
        "cluster2_ns": corde.rod_barrier_floor(2, threads=128, cluster=2, n_iters=100000),
        "cluster8_ns": corde.rod_barrier_floor(2, threads=128, cluster=8, n_iters=100000),
        "grid_sync_ns": corde.rod_barrier_floor(3, threads=128, cluster=1, n_iters=20000),
    }
    return {
        "floors": floors,
        "us_per_step": us_per_step,
        "us_per_step_without_launch_overlap": no_overlap_us,
        "total_ms": total_ms,
        "kernel_ms_avg": total_ms / (args.steps * LAUNCHES_PER_BENCH_STEP),
        "kernel_ms_isolated": float(np.mean(kern_ms)),
        "kernel_ms_median": float(np.median(kern_ms)),
        "launches": launches,
        "clocks": clk,
        "diag": diag[0].tolist(),
        "diag_rc": rc,
        "e2e_us": e2e_us,
        "e2e_launch_us": e2e["io"],
        "e2e_copies_launch_us": e2e["copies"],
        "e2e_persistent": persistent,
        "e2e_lockstep": lockstep,
        "n_nodes": 512,
        "n_iters": rod.n_iters,
        "plan": plan,
    }


BATCH_ITERS = os.path.join(ROOT, "tests", "golden", "batch_iters_seed4.json")


def batch_iteration_table():
    """Per-rod constraint iterations of the 4096-rod batch for which the FP64 oracle holds
    every segment within 1e-3 of its rest length over 1000 steps (written by
    tests/golden/make_batch_iters.py from the oracle alone)."""
    with open(BATCH_ITERS) as f:
        return json.load(f)["n_iters"]


def run_batched(args, torch, corde, W, rank, world, n_iters=None):
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    from paper_2509_04277_gb300 import sharding

    rods = W.batched_rods(4096, seed=4, n_iters=n_iters)
    mine = [rods[i] for i in sharding.shard([r.n_nodes for r in rods], rank, world)] if world > 1 else rods
    b = corde.RodBatch(mine)
    n_elem = b.n_elem
    S = args.batched_steps_per_launch or 100
    if not args.no_autotune:
        b.autotune(S)
    steps_autotuned = False
    if args.batched_steps_per_launch is None and not args.no_autotune:
        S = b.autotune_steps((10, 25, 50, 100, 200), 400)
        steps_autotuned = True
    n_launch = max(1, args.batched_steps // S)
    plan = b.plan()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    st0 = b.state_numpy()
    b.step(S)  # warm-up launch, then back to the initial state: the timed launches run steps 0 .. 999
    corde.rod_set_state(b.handle, st0["pos4"], st0["quat4"], st0["vel4"], st0["omega4"])
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(n_launch)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(n_launch)]
    _barrier(torch)
    torch.cuda.synchronize()
    launches = 0
    for k in range(n_launch):
        flush.fill_(float(k))
        starts[k].record(stream)
        b.step(S)
        ends[k].record(stream)
        launches += b.last_launch_count()
    torch.cuda.synchronize()
    _barrier(torch)
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    rc, diag = b.diagnostics()
    b.close()
    total_s = sum(ms) / 1e3
    el_steps = n_elem * S * n_launch
    return {
        "n_rods": len(mine),
        "n_elements": n_elem,
        "steps_per_launch": S,
        "steps_per_launch_autotuned": steps_autotuned,
        "launches": n_launch,
        "gpu_launches": launches,
        "seconds": total_s,
        "element_steps_per_s": el_steps / total_s,
        "ms_per_launch": float(np.mean(ms)),
        "plan": sorted({(int(a), int(c), int(k)) for a, c, k in plan}),
        "max_len_err": float(diag[:, 0].max()),
        "diag_rc": rc,
        "n_iters_histogram": {int(k): int(v) for k, v in zip(*np.unique([r.n_iters for r in mine],
                                                                         return_counts=True))},
        "flops_per_launch": sum(flops_per_el_step(r.n_iters) * r.n_nodes for r in mine) * S,
        "bytes_per_launch": BYTES_PER_EL_LAUNCH * n_elem,
    }


def run_adjoint(args, torch, corde, W, n_rods=1):
    """Adjoint workload: 256-element rod(s), 200 steps at dt = 1e-4 s, checkpoints every
    20 steps.  Times the plain forward (one persistent launch), the recorded rollout and
    the reverse pass."""
    stream = torch.cuda.current_stream()
    rods = [W.adjoint_rod(256, seed=5 + k) for k in range(n_rods)]
    b = corde.RodBatch(rods)
    n_steps, ckpt = 200, 20
    st = b.state_numpy()
    targets = [W.tip_target(5 + k, n_steps, r.dt, r.pos[-1]) for k, r in enumerate(rods)]
    g = torch.zeros((n_steps, b.n_elem, 4), dtype=torch.float32, device="cuda")

    def timed(fn, reps=5):
        ts = []
        for _ in range(reps):
            b.set_rod_states([b.rod_state(st, r) for r in range(n_rods)])
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts)), out

    fwd_ms, _ = timed(lambda: b.step(n_steps))
    fwd_launches = b.last_launch_count()
    roll_ms, traj = timed(lambda: b.rollout(n_steps, ckpt))
    for k, rod in enumerate(rods):
        tip = int(b.offsets[k + 1]) - 1
        g[:, tip, :3] = 2.0 * (traj[:, tip, :3] - torch.as_tensor(targets[k], dtype=torch.float32, device="cuda"))
    adj_ms, grads = timed(lambda: b.adjoint(g))
    finite = bool(all(torch.isfinite(v).all().item() for v in grads.values()))
    launch_info = corde.rod_adjoint_info(b.handle)
    b.close()
    el_steps = sum(r.n_nodes for r in rods) * n_steps
    # algorithmic DRAM bytes of the reverse pass: the loss gradient dL/dpos it reads
    # (16 B per element-step) and the checkpoints it restarts from (64 B per element per
    # checkpoint); the per-segment recomputed states stay L2-resident
    adj_bytes = el_steps * 16.0 + sum(r.n_nodes for r in rods) * 64.0 * (n_steps // ckpt)
    hbm = _peaks()[0].get("hbm_gbs", 6800.0)
    # the library's choice (rod_set_adjoint_record_budget, default 1 GiB): record each
    # segment's sweeps when they fit (compact layout for more rods than SMs), else
    # recompute every step before its reverse
    nt = launch_info["threads_per_block"]
    slots = rods[0].n_iters + 1 if launch_info["compact_records"] else 2 * rods[0].n_iters
    rec_bytes = ckpt * n_rods * slots * 2 * nt * 12
    mode = launch_info["mode"]
    layout = ", compact" if launch_info["compact_records"] else ""
    desc = (f"record mode ({rec_bytes / 2**20:.1f} MiB of sweep records per segment{layout})" if mode == "record"
            else "recompute mode")
    return {"n_rods": n_rods, "n_nodes": 256, "n_steps": n_steps, "ckpt_every": ckpt,
            "reverse_pass": desc,
            "launch": launch_info,
            "roofline_hbm": {"bytes": adj_bytes, "achieved_gbs": round(adj_bytes / (adj_ms * 1e-3) / 1e9, 2),
                             "peak_gbs": hbm, "frac": round(adj_bytes / (adj_ms * 1e-3) / 1e9 / hbm, 5),
                             "note": "latency-bound like the forward: one block per rod"},
            "fwd_ms": round(fwd_ms, 4), "fwd_launches": fwd_launches, "rollout_recorded_ms": round(roll_ms, 4),
            "adjoint_ms": round(adj_ms, 4), "adjoint_over_fwd": round(adj_ms / fwd_ms, 3),
            "adjoint_over_recorded_rollout": round(adj_ms / roll_ms, 3),
            "fwd_element_steps_per_s": el_steps / (fwd_ms * 1e-3),
            "adjoint_element_steps_per_s": el_steps / (adj_ms * 1e-3), "gradients_finite": finite}


def run_pair(args, torch, corde, W, fp32):
    """Catheter/guidewire pair, 2 x 512 elements, binding modes v0/v1/v2, 1, 10 and 50 time
    steps per launch (about 1000 steps each), drives updated every launch."""
    stream = torch.cuda.current_stream()
    out = {}
    for mode in (0, 1, 2):
        for S in (1, 10, 50):
            cat, gw = W.catheter_guidewire(512, seed=3, beta0=-100.25)
            l0 = gw.length / 511
            n_launch = max(20, 1000 // S)
            dcs, dgs = W.pair_drives(3, n_launch + 5, S * gw.dt, l0, -100.25)
            drv = torch.as_tensor(np.stack([dcs, dgs], axis=1).astype(np.float32), device="cuda").contiguous()
            b = corde.RodBatch([cat, gw])
            b.bind(0, 1, mode)
            for k in range(5):
                b.step(S, drive=drv[k])
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(n_launch):
                b.step(S, drive=drv[5 + k])
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            out[f"v{mode}_{S}ts"] = round(ms * 1e3 / (n_launch * S), 4)
            b.close()
    # the oracle's pair step on one host core, a bounded sample per mode
    import oracle

    cpu = {}
    for mode in (0, 1, 2):
        cat, gw = W.catheter_guidewire(512, seed=3, beta0=-100.25)
        so, si = oracle.state_of(cat), oracle.state_of(gw)
        n, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < 1.0 or n == 0:
            so, si = oracle.step_pair(cat, so, gw, si, mode, -100.25, 10)
            n += 10
        cpu[f"v{mode}"] = round((time.perf_counter() - t0) * 1e6 / n, 2)
    flops_step = 2 * 512 * flops_per_el_step(10)  # the two rods' steps (binding not counted)
    peak = fp32["burst_tflops"]
    frac = {k: round(flops_step / (v * 1e-6) / 1e12 / peak, 7) for k, v in out.items()}
    sms = fp32["n_sms"]
    return {"unit": "us/step", "workload": "2 x 512 inextensible rods (catheter r=1 mm E=2 GPa, guidewire "
                                           "r=0.45 mm E=60 GPa), one thread block per pair", "us_per_step": out,
            "roofline_alu": {"flops_per_step": flops_step, "peak_tflops": round(peak, 2),
                             "peak_source": "measured (rod_fp32_peak, burst)",
                             "frac_of_gpu": frac, "note": f"one pair = one thread block on one SM: at most 1/{sms} "
                                                          f"of the GPU; x{sms} gives the fraction of that SM"},
            "cpu_oracle_us_per_step": cpu,
            "speedup_vs_oracle_1core_10ts": {f"v{m}": round(cpu[f"v{m}"] / out[f"v{m}_10ts"], 1) for m in (0, 1, 2)}}


def run_extensible(args, torch, corde, W):
    """The plain extensible rod (no constraint iterations): the 64-element clamped
    pendulum as configured (L = 1 m, r = 1 mm, E = 50 GPa, G = 20 GPa, gravity, Rayleigh
    damping 0.1, dt = 1e-5 s) and the same rod with 1000 elements, the length of the
    paper's extensible comparison (Table 1); 1000 steps at 10 steps per launch, timed
    after 100 steps, beside the oracle on one host core."""
    import oracle

    stream = torch.cuda.current_stream()
    out = {}
    for n in (64, 1000):
        rod = W.extensible_pendulum(n, seed=1)
        b = corde.RodBatch([rod])
        b.autotune(STEPS_PER_LAUNCH)
        for _ in range(10):
            b.step(STEPS_PER_LAUNCH)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(100):
            b.step(STEPS_PER_LAUNCH)
        e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / (100 * STEPS_PER_LAUNCH)
        plan = [int(x) for x in b.plan()[0]]
        b.close()
        # the oracle on one host core, a bounded sample (about one second)
        s = oracle.state_of(rod)
        k, t0 = 0, time.perf_counter()
        while k == 0 or time.perf_counter() - t0 < 1.0:
            s = oracle.step(rod, s, STEPS_PER_LAUNCH)
            k += STEPS_PER_LAUNCH
        cpu_us = (time.perf_counter() - t0) * 1e6 / k
        out[str(n)] = {"us_per_step": round(us, 4), "plan": plan, "cpu_oracle_1core_us_per_step": round(cpu_us, 2),
                       "speedup_vs_oracle_1core": round(cpu_us / us, 1)}
    return {"unit": "us/step", "steps_per_launch": STEPS_PER_LAUNCH, "by_elements": out,
            "workload": "extensible clamped pendulum (L=1 m, r=1 mm, E=50 GPa, G=20 GPa, rho=6500, gravity, "
                        "Rayleigh damping 0.1, dt=1e-5 s), 1000 steps at 10 per launch",
            "paper_context": {"extensible_gpu_us_per_step_10tskl": {"100": 26.0, "1000": 31.0},
                              "extensible_speedup_vs_original_corde": 40.0,
                              "hardware": "GeForce GTX 560 (Fermi), host-visible times (Table 1)"}}


def run_long_rods(args, torch, corde, W):
    """Latency per step against rod length (the paper's near-constant-time claim for rods
    spread over several SMs, Fig. 7): guidewire rods (L = 1.5 m) of 512 ... 131072 nodes,
    10 steps per launch; rods above 2048 nodes run on a thread-block cluster, above 32768
    on a cooperative grid (2048 nodes per block)."""
    stream = torch.cuda.current_stream()
    out = {}
    for n in (512, 1024, 2048, 3072, 4096, 8192, 16384, 32768, 65536, 131072):
        rod = W.guidewire(n, seed=7)
        b = corde.RodBatch([rod])
        if n <= 2048:
            b.autotune(STEPS_PER_LAUNCH)
        plan = [int(x) for x in b.plan()[0]]
        for _ in range(20):
            b.step(STEPS_PER_LAUNCH)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(100):
            b.step(STEPS_PER_LAUNCH)
        e1.record(stream)
        torch.cuda.synchronize()
        out[str(n)] = {"us_per_step": round(e0.elapsed_time(e1) * 1e3 / (100 * STEPS_PER_LAUNCH), 4),
                       "plan": plan}
        b.close()
    return out


def run_tube(args, torch, corde, W):
    """Guidewire insertion into a curved vessel (contact constraints with Coulomb friction
    against an analytic tube): 512 nodes, vessel centreline radius 0.5 m, inner radius
    2 mm, mu = 0.1, base pushed at 5 cm/s; 10 steps per launch, 100 launches timed after
    300 steps of settling (the wire then presses on the outer wall), beside the same
    rod without the vessel."""
    stream = torch.cuda.current_stream()
    drive = torch.as_tensor(np.array([[0.05, 0, 0, 0, 0, 0, 2.0, 0]], np.float32), device="cuda")
    out = {}
    for with_tube in (True, False):
        rod, tube = W.vessel_guidewire(512, seed=11)
        b = corde.RodBatch([rod])
        if with_tube:
            b.set_tube(0, tube)
        b.autotune(STEPS_PER_LAUNCH)
        for _ in range(30):
            b.step(STEPS_PER_LAUNCH, drive=drive)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(100):
            b.step(STEPS_PER_LAUNCH, drive=drive)
        e1.record(stream)
        torch.cuda.synchronize()
        key = "vessel" if with_tube else "free"
        out[key] = {"us_per_step": round(e0.elapsed_time(e1) * 1e3 / (100 * STEPS_PER_LAUNCH), 4),
                    "plan": [int(x) for x in b.plan()[0]]}
        if with_tube:
            pos = b.rod_state(b.state_numpy(), 0)["pos"]
            off = np.hypot(np.hypot(pos[:, 0] - tube[0], pos[:, 1] - tube[1]) - tube[3], pos[:, 2] - tube[2])
            allow = tube[4] - rod.radius
            out[key]["nodes_on_wall"] = int(np.sum(off > allow * (1 - 1e-3)))
            out[key]["max_offset_over_allow"] = round(float(off.max() / allow), 6)
        b.close()
    return {"unit": "us/step", "workload": "512-node guidewire in a curved vessel (Rc 0.5 m, Rt 2 mm, mu 0.1), "
                                           "10 constraint iterations over distance and contact constraints",
            **out}


def run_knot(args, torch, corde, W):
    """Self-collision on a knot-like configuration: a 512-node guidewire laid on a (2, q)
    torus knot (two strands twisted together, 2.1 r apart, straight at rest), base pulled
    at 5 cm/s and twisted at 2 rad/s; 10 steps per launch, 100 launches timed after 30,
    beside the same rod without self-collision."""
    stream = torch.cuda.current_stream()
    drive = torch.as_tensor(np.array([[0.05, 0, 0, 0, 0, 0, 2.0, 0]], np.float32), device="cuda")
    out = {}
    for with_self in (True, False):
        rod = W.torus_knot(512, seed=21)
        b = corde.RodBatch([rod])
        if with_self:
            b.set_self_collision(0, 0.1)
        else:
            b.autotune(STEPS_PER_LAUNCH)
        for _ in range(30):
            b.step(STEPS_PER_LAUNCH, drive=drive)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(100):
            b.step(STEPS_PER_LAUNCH, drive=drive)
        e1.record(stream)
        torch.cuda.synchronize()
        key = "self_collision" if with_self else "free"
        out[key] = {"us_per_step": round(e0.elapsed_time(e1) * 1e3 / (100 * STEPS_PER_LAUNCH), 4),
                    "plan": [int(x) for x in b.plan()[0]]}
        if with_self:
            out[key].update(b.self_collision_stats(0))
        b.close()
    return {"unit": "us/step", "workload": "512-node guidewire on a (2, 15) torus knot, self-collision with "
                                           "mu 0.1 in each of 10 constraint iterations",
            "paper_context": {"us_per_step": 172.0, "what": "double fisherman's knot, 2 x 256 elements, ~300 "
                              "colliding sphere pairs, 10 steps per launch, GTX 560 (Section 3.5)"},
            **out}


def cpu_baseline_single(seconds=10.0):
    """The FP64 oracle as it stands, one host core, on the 512-element guidewire."""
    import oracle
    from paper_2509_04277_gb300 import workloads as W

    rod = W.guidewire(512, seed=2)
    drive = W.sinusoid_drive(2, 100000, STEPS_PER_LAUNCH * rod.dt)
    s = oracle.state_of(rod)
    oracle.step(rod, s, 10)
    steps = 0
    t0 = time.perf_counter()
    k = 0
    while steps == 0 or time.perf_counter() - t0 < seconds:
        s = oracle.step(rod, s, STEPS_PER_LAUNCH, drive=drive[k % len(drive)])
        steps += STEPS_PER_LAUNCH
        k += 1
    el = time.perf_counter() - t0
    return {"value": el * 1e6 / steps, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"512-element guidewire, {steps} time steps (10 per call, 1 kHz drive), FP64, serial"}


def cpu_baseline_batched(seconds=10.0):
    """The FP64 oracle over a sample of the 4096-rod batch, OpenMP over rods on all cores."""
    import oracle
    from paper_2509_04277_gb300 import workloads as W

    rods = W.batched_rods(4096, seed=4)[:256]
    states = [oracle.state_of(r) for r in rods]
    n_el = sum(r.n_nodes for r in rods)
    threads = oracle.step_batch(rods, states, 1)
    steps = 0
    t0 = time.perf_counter()
    while steps == 0 or time.perf_counter() - t0 < seconds:
        oracle.step_batch(rods, states, 10)
        steps += 10
    el = time.perf_counter() - t0
    return {"value": n_el * steps / el, "unit": "element-steps/s", "cores": threads, "kind": "oracle",
            "sample": f"first 256 of the 4096 rods ({n_el} elements), {steps} steps, FP64, OpenMP over rods"}


def _barrier(torch):
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def _max_over_ranks(torch, x: float) -> float:
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return x


def _sum_over_ranks(torch, x: float) -> float:
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())
    return x


def main_ours(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import __graft_entry__

    if rank == 0 or world == 1:
        __graft_entry__.build()
    _barrier(torch)
    from paper_2509_04277_gb300 import corde
    from paper_2509_04277_gb300 import workloads as W

    corde.load()
    if args.only is not None:
        part = {"single": lambda: run_single_rod(args, torch, corde, W, rank),
                "batched": lambda: run_batched(args, torch, corde, W, rank, world),
                "batched_inextensible": lambda: run_batched(args, torch, corde, W, rank, world,
                                                            n_iters=batch_iteration_table()),
                "pair": lambda: run_pair(args, torch, corde, W, measure_fp32_peak(corde)),
                "long": lambda: run_long_rods(args, torch, corde, W),
                "tube": lambda: run_tube(args, torch, corde, W),
                "knot": lambda: run_knot(args, torch, corde, W),
                "extensible": lambda: run_extensible(args, torch, corde, W),
                "adjoint": lambda: {"single": run_adjoint(args, torch, corde, W, 1),
                                "batched": run_adjoint(args, torch, corde, W, 256)}}[args.only]()
        if rank == 0:
            print(json.dumps({"only": args.only, "result": part}, default=str), flush=True)
        return
    single = run_single_rod(args, torch, corde, W, rank)
    batched = run_batched(args, torch, corde, W, rank, world) if not args.skip_batched else None
    batched_inext = None
    if not args.skip_batched and not args.skip_batched_inextensible:
        batched_inext = run_batched(args, torch, corde, W, rank, world, n_iters=batch_iteration_table())
    fp32 = measure_fp32_peak(corde)
    pair = run_pair(args, torch, corde, W, fp32) if not args.skip_pair else None
    long_rods = run_long_rods(args, torch, corde, W) if not args.skip_long else None
    tube = run_tube(args, torch, corde, W) if not args.skip_tube else None
    knot = run_knot(args, torch, corde, W) if not args.skip_knot else None
    extensible = run_extensible(args, torch, corde, W) if not args.skip_extensible else None
    adjoint = None
    if not args.skip_adjoint:
        adjoint = {"single": run_adjoint(args, torch, corde, W, 1), "batched": run_adjoint(args, torch, corde, W, 256)}
    value = _max_over_ranks(torch, single["us_per_step"])
    batched_totals = {}
    for key, part in (("batched", batched), ("batched_inextensible", batched_inext)):
        if part is not None:
            el_steps = part["n_elements"] * part["steps_per_launch"] * part["launches"]
            batched_totals[key] = (_sum_over_ranks(torch, el_steps), _max_over_ranks(torch, part["seconds"]))
    lock = single["e2e_lockstep"]
    e2e_path = "lockstep_persistent" if "us_per_step" in lock else "launch_per_tick"
    e2e = _max_over_ranks(torch, lock["us_per_step"] if "us_per_step" in lock else single["e2e_us"])
    out = None
    if rank == 0:
        peaks, which = _peaks()
        fp32_peak = fp32["burst_tflops"]  # the single rod's kernel is timed alone
        n_sms = fp32["n_sms"]
        flops_launch = flops_per_el_step(single["n_iters"]) * single["n_nodes"] * STEPS_PER_LAUNCH
        achieved = flops_launch / (single["kernel_ms_avg"] * 1e-3) / 1e12
        traffic, _ = _traffic("step_kernel_guidewire512")
        cpu = cpu_baseline_single(args.cpu_seconds)
        out = {
            "metric": METRIC,
            "value": round(value, 4),
            "unit": UNIT,
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(single["total_ms"] / args.steps, 4),
            "higher_is_better": False,
            "scaling": "weak",
            "vs_baseline": round(value / 32.0, 5),
            "dtype": "f32",
            "data": "synthetic (seeded guidewire, 1 kHz sinusoidal insertion/twist drive)",
            "config": workload_config(world),
            "gpu_launches": single["launches"],
            "e2e": {"value": round(e2e, 4), "unit": UNIT,
                    "h2d_bytes_per_step": 32 * LAUNCHES_PER_BENCH_STEP,
                    "d2h_bytes_per_step": 512 * 16 * LAUNCHES_PER_BENCH_STEP,
                    "path": e2e_path,
                    "what": {"lockstep_persistent": "one persistent launch in lock-step (rod_step once; per tick "
                                                    "one rod_mailbox_tick call: the host spins until the tick's "
                                                    "snapshot is published, writes the next tick's drive at once, "
                                                    "then copies the snapshot): the kernel waits for each drive, "
                                                    "runs 10 steps and publishes all 512 positions to pinned host "
                                                    "memory; the host's copy of tick k overlaps the kernel's tick "
                                                    "k + 1; host wall clock",
                             "launch_per_tick": "per tick one rod_step_io call (the kernel reads the drive from "
                                                "pinned host memory and writes the 512 positions to pinned host "
                                                "memory) + stream sync; host wall clock"}[e2e_path],
                    "launch_per_tick_us_per_step": round(single["e2e_launch_us"] / STEPS_PER_LAUNCH, 4),
                    "explicit_copies_per_launch_us": round(single["e2e_copies_launch_us"], 3),
                    "lockstep_persistent": single["e2e_lockstep"],
                    "persistent_mailbox": single["e2e_persistent"] if "us_per_step" not in single["e2e_persistent"]
                    else {
                        "us_per_step": round(single["e2e_persistent"]["us_per_step"], 4),
                        "ticks": single["e2e_persistent"]["ticks"], "steps": single["e2e_persistent"]["steps"],
                        "what": "one persistent launch; per host tick: drive written to the mailbox, newest "
                                "snapshot of all 512 positions pulled (published every 10 steps); the kernel "
                                "never waits for the host, so this is simulated steps over host wall time"}},
            "roofline": {"bound": "alu", "achieved": round(achieved, 6), "peak": round(fp32_peak, 2),
                         "unit": "TFLOP/s", "frac": round(achieved / fp32_peak, 8), "traffic": traffic,
                         "peak_source": "measured (rod_fp32_peak, burst: the kernel is timed alone)",
                         "fp32_peak": fp32,
                         "note": f"one rod = one thread block on one of {n_sms} SMs; latency-bound by design",
                         "kernel": "step_kernel<ept=%d, nt=%d>" % tuple(single["plan"]),
                         "frac_of_one_sm": round(achieved / (fp32_peak / n_sms), 6),
                         "kernel_us_per_launch": round(single["kernel_ms_avg"] * 1e3, 3),
                         "duration": "timed region / launches (includes launch gaps); one launch bracketed "
                                     "alone by events: %.3f us" % (single["kernel_ms_isolated"] * 1e3)},
            "latency": {"us_per_step": round(value, 4), "barriers_per_step": 2 + single["n_iters"],
                        "launch_overlap": "programmatic dependent launch (each launch waits in-kernel "
                                          "for the previous one's writes)",
                        "us_per_step_without_launch_overlap": round(single["us_per_step_without_launch_overlap"], 4),
                        "launch_rate_khz": round(1e3 / (value * STEPS_PER_LAUNCH), 2),
                        "haptic_1khz_realtime": bool(value * STEPS_PER_LAUNCH < 1000.0),
                        "floors_ns": {k: round(v, 2) for k, v in single["floors"].items()},
                        "step_over_grid_sync": round(value * 1e3 / single["floors"]["grid_sync_ns"], 3),
                        "step_over_block_barrier_floor": round(
                            value * 1e3 / ((2 + single["n_iters"]) * single["floors"]["block_ns"]), 3)},
            "cpu_baseline": cpu,
            "clocks": single["clocks"],
            "checks": {"max_len_err": single["diag"][0], "max_qnorm_err": single["diag"][1],
                       "nonfinite": single["diag"][2]},
            "paper_context": {"us_per_step_512_single_block_10tskl": 32.0, "hardware": "GeForce GTX 560 (Fermi)",
                              "note": "host-visible time incl. launch and D2H; compare with e2e",
                              "speedups_vs_cpu": {"extensible_10tskl": 40.0, "inextensible": 15.11,
                                                  "catheter_guidewire_2x512": 13.5},
                              "haptic_rate_khz": [0.5, 1.0],
                              "ours_vs_oracle_1core": round(cpu["value"] / value, 1) if cpu else None},
        }
        bw = peaks.get("hbm_gbs", 6800.0)
        for key, part in (("batched", batched), ("batched_inextensible", batched_inext)):
            if part is None:
                continue
            sec = part["seconds"] / part["launches"]
            # whole job: element-steps of every rank over the slowest rank's time
            tot_el_steps, max_seconds = batched_totals[key]
            part["element_steps_per_s"] = tot_el_steps / max_seconds
            out[key] = {
                "element_steps_per_s": part["element_steps_per_s"],
                "n_rods": part["n_rods"], "n_elements": part["n_elements"],
                "n_iters": part["n_iters_histogram"],
                "steps_per_launch": part["steps_per_launch"],
                "steps_per_launch_autotuned": part["steps_per_launch_autotuned"],
                "launches": part["launches"],
                "gpu_launches": part["gpu_launches"], "ms_per_launch": round(part["ms_per_launch"], 4),
                "plan": part["plan"], "max_len_err": part["max_len_err"],
                "roofline_alu": {"achieved": part["flops_per_launch"] / sec / 1e12,
                                 "peak": fp32["sustained_tflops"], "unit": "TFLOP/s",
                                 "peak_source": "measured (rod_fp32_peak, sustained: the batch runs for seconds)",
                                 "frac": part["flops_per_launch"] / sec / 1e12 / fp32["sustained_tflops"]},
                "roofline_hbm": {"achieved": part["bytes_per_launch"] / sec / 1e9, "peak": bw, "unit": "GB/s",
                                 "frac": part["bytes_per_launch"] / sec / 1e9 / bw},
            }
        if "batched" in out:
            out["batched"]["what"] = ("10 constraint iterations per rod (the paper's count); floppy long rods "
                                      "stretch beyond 1e-3 (max_len_err)")
            out["batched"]["cpu_baseline"] = (cpu_baseline_batched(args.cpu_seconds)
                                              if not args.skip_cpu_batched else None)
        if "batched_inextensible" in out:
            out["batched_inextensible"]["what"] = (
                "per-rod constraint iterations (10 to 640) for which the FP64 oracle holds every segment within "
                "1e-3 of its rest length over the 1000 steps (tests/golden/batch_iters_seed4.json)")
        if adjoint is not None:
            out["adjoint"] = adjoint
        if pair is not None:
            out["pair"] = pair
        if long_rods is not None:
            out["long_rods"] = {"unit": "us/step", "steps_per_launch": STEPS_PER_LAUNCH,
                                "by_nodes": long_rods}
        if tube is not None:
            out["vessel_contact"] = tube
        if knot is not None:
            out["self_collision"] = knot
        if extensible is not None:
            out["extensible"] = extensible
        print(json.dumps(out), flush=True)
    _barrier(torch)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


# --------------------------------------------------------------------------- reference arm


def workload_config(world=1):
    """The bench workload and its timing conditions, the same for both arms."""
    return {
        "workload": "guidewire: 1 inextensible rod, 512 elements, L=1.5 m, r=0.45 mm, E=60 GPa, "
                    "10 constraint iterations, dt=1e-4 s, 10 time steps per persistent launch",
        "n_rods": 1, "n_elements": 512, "steps_per_launch": STEPS_PER_LAUNCH,
        "time_steps_per_bench_step": STEPS_PER_LAUNCH * LAUNCHES_PER_BENCH_STEP,
        "l2": "flushed (256 MiB write) between bench steps, outside the timed intervals",
        "parallelism": f"replicas x{world}" if world > 1 else "single GPU, one thread block per rod",
    }


def main_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2509_04277_gb300 import workloads as W

    oracle.build()
    rod = W.guidewire(512, seed=2)
    steps_per_bench = 1000
    drive = W.sinusoid_drive(2, (args.warmup + args.steps) * steps_per_bench // STEPS_PER_LAUNCH,
                             STEPS_PER_LAUNCH * rod.dt)
    s = oracle.state_of(rod)
    k = 0
    for _ in range(args.warmup):
        for _ in range(steps_per_bench // STEPS_PER_LAUNCH):
            s = oracle.step(rod, s, STEPS_PER_LAUNCH, drive=drive[k])
            k += 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _ in range(steps_per_bench // STEPS_PER_LAUNCH):
            s = oracle.step(rod, s, STEPS_PER_LAUNCH, drive=drive[k])
            k += 1
    el = time.perf_counter() - t0
    value = el * 1e6 / (args.steps * steps_per_bench)
    out = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el * 1e3 / args.steps, 4),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.gpus),
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} x {steps_per_bench} time steps of the 512-element guidewire"},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batched-steps", type=int, default=1000)
    ap.add_argument("--batched-steps-per-launch", type=int, default=None,
                    help="steps per launch of the batch (default: autotuned among 10..200)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--skip-batched", action="store_true")
    ap.add_argument("--skip-batched-inextensible", action="store_true")
    ap.add_argument("--skip-cpu-batched", action="store_true")
    ap.add_argument("--skip-adjoint", action="store_true")
    ap.add_argument("--skip-pair", action="store_true")
    ap.add_argument("--skip-long", action="store_true")
    ap.add_argument("--skip-tube", action="store_true")
    ap.add_argument("--skip-knot", action="store_true")
    ap.add_argument("--skip-extensible", action="store_true")
    ap.add_argument("--only", choices=["single", "batched", "batched_inextensible", "pair", "adjoint", "long", "tube", "knot",
                             "extensible"], default=None,
                    help="run one part only and print its raw result (profiling aid, not a bench line)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="fixed kernel plan (single rod <2, 256>, batch default plan)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        main_reference(args)
    else:
        main_ours(args)


if __name__ == "__main__":
    main()
