"""Throughput of the IC time step on GB300: cell-updates/s and particle-steps/s.

Workload (default): 128^3 periodic staggered grid, FP32 state with FP64
accumulators, kT = 1e-3 (Philox stochastic stress), a standing wave of two
wavelengths along x held by the mode drive, 10^4 particles placed uniformly
at random with minimum separation 2h (m_p = 1.5 rho0 V, kappa_p = 0.5
kappa_f, free), thermal (Gibbs) initial state.

One step = the whole IC step (App. A.2 substeps 1-7: particle half step,
three RK3 fluid stages with particle-pressure corrections, impulse, spreading,
final position, accumulators), launched as one CUDA graph.  Inputs are resident
in HBM.  Between timed steps the L2 is flushed by writing a 512 MB buffer, and
each step is timed alone with CUDA events on the library's stream.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank runs its own box (box id = rank): weak scaling, no
collective in the data path; rank 0 prints one JSON line.
"""
import argparse
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

METRIC = "cell-updates/s and particle-steps/s (128^3, 1e4 particles); % of HBM roofline"
WORKLOAD = ("128^3 staggered grid FP32 state + FP64 accumulators, 1e4 free particles (min sep 2h), kT=1e-3, "
            "2-wavelength standing wave along x, thermal start")
# algorithmic bytes of the stage-wise SSP-RK3 sweep per cell and step (FP32):
# stage 1 reads U_s (4 words) and writes 4; stages 2-3 read U_s and U^n (8) and write 4
ALG_BYTES_PER_CELL_STEP = {"fp32": 128, "fp64": 256}
# The FP64 form is bound by GB300's FP64 units, not HBM: its roofline counts the
# floating-point operations of the three stages as written (an FMA is 2; a
# division, logarithm, square root, sine or cosine 1), 580 per cell and step,
# against the FP64 FMA rate measured on the GPU by the library's FMA-chain
# kernel (ic_fma64_rate); the nominal 1.25 TFLOP/s only if that fails.
ALG_FP64_FLOPS_PER_CELL_STEP = 580
# revision of the stage kernels: the ncu traffic in profiles/stage_traffic.json
# is reported only when it was captured on this revision
STAGE_KERNEL_REV = "pair-scaled-fluxes-ty13-idx"
FP64_PEAK_TFLOPS = 1.25   # nominal, the fallback


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi SM clock and throttle reasons, sampled every 50 ms; only the
    samples taken inside the timed window are summarised."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, bufsize=1)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self, window=None):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        lines = self.lines
        if window is not None:
            inside = [x for x in lines if window[0] <= x[0] <= window[1]]
            lines = inside if inside else lines
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], [], set()
        for _, ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[2:6]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        n_inside = 0 if window is None else sum(1 for x in self.lines if window[0] <= x[0] <= window[1])
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "samples_in_timed_region": n_inside}


def fp64_fma_peak(local):
    """The FP64 FMA rate of this GPU, measured by the library's FMA-chain
    kernel (ic_fma64_rate, CUDA events) with the SM clock sampled meanwhile."""
    import ctypes

    from paper_1307_0702_gb300 import _lib

    lib = _lib.load()
    rate, sec = ctypes.c_double(), ctypes.c_double()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    w0 = time.perf_counter()
    st = lib.ic_fma64_rate(200000, ctypes.byref(rate), ctypes.byref(sec))
    clocks = sampler.stop((w0, time.perf_counter()))
    if st != 0:
        return None
    out = {"tflops": rate.value / 1e12, "seconds": sec.value, "clocks": clocks,
           "how": "ic_fma64_rate: 8 independent FMA chains per thread, 8 CTAs x 256 threads per SM, CUDA events"}
    if clocks and clocks.get("sm_mhz"):
        out["tflops_per_ghz"] = out["tflops"] / (clocks["sm_mhz"] / 1e3)   # the rate scaled by the clock it ran at
    return out


def time_steps(grid, steps, warmup, flush, local):
    """Device time of `steps` single steps (CUDA events on the library's
    stream, the L2 flushed before each), the per-class kernel times of the
    same number of steps launched kernel by kernel, and the clocks."""
    import torch

    stream = grid.stream
    grid.step(warmup)
    grid.sync()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    sampler = ClockSampler(local)
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    w0 = time.perf_counter()
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
        grid.step(1)
        with torch.cuda.stream(stream):
            ev[i][1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop((w0, time.perf_counter()))
    t = float(np.sum([a.elapsed_time(b) for a, b in ev])) / 1e3
    grid.profile(True)
    for i in range(steps):
        if i % 8 == 0:
            with torch.cuda.stream(stream):
                torch.cuda._sleep(8_000_000)
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xFF)
        grid.step(1)
    prof = grid.profile_read()
    grid.profile(False)
    return t, prof, clocks


def sub_fp64(steps, warmup, local, flush, peak):
    """The plain FP64 form of the same workload (the precision the oracle
    matches to 1e-11): its throughput and its FP64-unit roofline."""
    from paper_1307_0702_gb300 import workloads as W

    gp, parts = W.large_box_config()
    gp["precision"] = "fp64"
    grid = setup_box(gp, parts, seed_thermal=1000)
    tiling = grid.autotune(reps=1)
    t, prof, clocks = time_steps(grid, steps, warmup, flush, local)
    grid.close()
    cells = gp["nx"] * gp["ny"] * gp["nz"]
    stage_ms = prof["fluid"][0] / steps
    tflops = ALG_FP64_FLOPS_PER_CELL_STEP * cells / (stage_ms * 1e-3) / 1e12
    peak_tf, kind = (peak["tflops"], "measured (ic_fma64_rate)") if peak else (FP64_PEAK_TFLOPS, "nominal")
    return {"value": cells * steps / t, "unit": "cell-updates/s", "ms_per_step": 1e3 * t / steps, "steps": steps,
            "particle_steps_per_s": parts["q"].shape[0] * steps / t, "stage_tiling": list(tiling),
            "roofline": {"bound": "alu", "achieved": tflops, "peak": peak_tf, "unit": "TFLOP/s",
                         "frac": tflops / peak_tf, "peak_kind": kind, "stage_ms_per_step": stage_ms,
                         "alg_flops_per_step": ALG_FP64_FLOPS_PER_CELL_STEP * cells},
            "clocks": clocks}


def sub_ensemble(steps, warmup, local, flush, boxes=256):
    """The FP32 batched ensemble (256 boxes of edges 16-48, ic_batch_step)."""
    import torch

    from paper_1307_0702_gb300 import Batch, workloads as W

    cfg = W.ensemble_config(boxes)
    grids = [setup_box(gp, parts, seed_thermal=5000 + b) for b, (gp, parts) in enumerate(cfg)]
    cells = sum(g.shape[0] * g.shape[1] * g.shape[2] for g in grids)
    npart = sum(g.n_particles for g in grids)
    s0 = grids[0].stream
    with Batch(grids) as batch:
        batch.autotune(reps=1)
        batch.step(warmup)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        sampler = ClockSampler(local)
        sampler.start()
        time.sleep(0.3)
        w0 = time.perf_counter()
        for i in range(steps):
            with torch.cuda.stream(s0):
                flush.fill_(i & 0xFF)
                ev[i][0].record(s0)
            batch.step(1)
            with torch.cuda.stream(s0):
                ev[i][1].record(s0)
        torch.cuda.synchronize()
        clocks = sampler.stop((w0, time.perf_counter()))
    t = float(np.sum([a.elapsed_time(b) for a, b in ev])) / 1e3
    for g in grids:
        g.close()
    return {"value": cells * steps / t, "unit": "cell-updates/s", "ms_per_step": 1e3 * t / steps, "steps": steps,
            "boxes": boxes, "cells": cells, "particles": npart, "particle_steps_per_s": npart * steps / t,
            "dtype": "f32", "clocks": clocks,
            "workload": "256 FP32 boxes, edges uniform in {16,24,32,48}, 1-200 particles each, kT=1e-3, Philox seed "
                        "= box index, one ic_batch_step per step"}


def sub_long_run(steps, local):
    """The headline box over a long run in one ic_step call (its graph
    replayed per step, no L2 flush): the amortised step time including the
    neighbour-list rebuilds the particles' motion triggers, and their count."""
    import torch

    from paper_1307_0702_gb300 import workloads as W

    gp, parts = W.large_box_config()
    grid = setup_box(gp, parts, seed_thermal=1000)
    grid.autotune(reps=1)
    grid.step(3)
    grid.sync()
    r0 = grid.neighbour_rebuilds()
    stream = grid.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    w0 = time.perf_counter()
    with torch.cuda.stream(stream):
        e0.record(stream)
    grid.step(steps)
    with torch.cuda.stream(stream):
        e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop((w0, time.perf_counter()))
    t = e0.elapsed_time(e1) / 1e3
    rebuilds = grid.neighbour_rebuilds() - r0
    grid.close()
    cells = gp["nx"] * gp["ny"] * gp["nz"]
    return {"value": cells * steps / t, "unit": "cell-updates/s", "ms_per_step": 1e3 * t / steps, "steps": steps,
            "rebuilds": rebuilds, "particle_steps_per_s": parts["q"].shape[0] * steps / t, "clocks": clocks,
            "how": "one ic_step call of all steps after 3 warm-up steps, CUDA events around it, L2 not flushed"}


def sub_force_accuracy():
    """The radiation force of the single tethered particle (32^3, h = 1,
    kT = 0, 8000 steps, Blackman-Harris window from step 3000) in FP32 and
    FP64 against the FP64 oracle's value stored in
    tests/golden/config1_force.json (written by the oracle alone)."""
    from paper_1307_0702_gb300 import Grid, workloads as W

    with open(os.path.join(ROOT, "tests", "golden", "config1_force.json")) as f:
        gold = json.load(f)
    out = {"workload": "one tethered particle at L/8 in the driven 32^3 box (h=1, kT=0, m_p=1.5 rho0 V, "
                       f"kappa_p=0.5 kappa_f), {gold['nsteps']} steps, window from step {gold['skip']}",
           "oracle_force": gold["f_spring"][0], "oracle_a2": gold["a2"]}
    for prec in ("fp32", "fp64"):
        gp, parts, _ = W.single_particle_config()
        gp["precision"] = prec
        rho, g = W.velocity_phase_wave_fields(gp)
        w = W.blackman_harris(gold["nsteps"], gold["skip"])
        with Grid(gp) as grid:
            grid.set_state(rho, g)
            grid.add_particles(parts["q"], parts["m_e"], parts["kappa_ratio"], parts["k_spring"])
            grid.step(len(w), w)
            fs, _, a2 = grid.time_average()
        out[prec] = {"force_rel_err": float(fs[0][0] / gold["f_spring"][0] - 1.0),
                     "a2_rel_err": float(a2 / gold["a2"] - 1.0)}
    return out


def setup_box(gp, parts, seed_thermal):
    from paper_1307_0702_gb300 import Grid, workloads as W

    grid = Grid(gp)
    rho, g = W.standing_wave_fields(gp)
    grid.set_state(rho, g)
    if gp["kT"] > 0:
        grid.init_thermal(seed_thermal, add=True)
    grid.add_particles(parts["q"], parts["m_e"], parts["kappa_ratio"], parts["k_spring"])
    return grid


def oracle_sample():
    """A 64^3 sub-box of the benchmark workload with the same particle density
    (1250 particles) and fluid parameters, as an oracle simulation."""
    from oracle import ic as oic
    from paper_1307_0702_gb300 import workloads as W

    gp, parts = W.many_particle_config(64, 1250, kT=1e-3, wave_amp=1e-3, wave_nlambda=1, seed=3, min_sep=2.0,
                                       fixed_contrast=(1.5, 0.5), k_spring=0.0)
    p = oic.GridParams(**{k: v for k, v in gp.items() if k in oic.GridParams.__dataclass_fields__})
    rho, g = W.standing_wave_fields(gp)
    th_drho, th_g = oic.thermal_fluctuation(p, 1000)
    sim = oic.Simulation(p, g=[g[a] + th_g[a] for a in range(3)], drho=rho - p.rho0 + th_drho)
    sim.add_particles(parts["q"], parts["m_e"], parts["kappa_ratio"], parts["k_spring"])
    return sim


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def _slab_worker(rank, world, port, warmup, steps, queue):
    """One process of the all-core oracle: its z-slab of the 128^3 workload."""
    import torch.distributed as dist

    from oracle import ic as oic
    from oracle import slabs
    from paper_1307_0702_gb300 import workloads as W

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    gp, parts = W.large_box_config()
    p = oic.GridParams(**{k: v for k, v in gp.items() if k in oic.GridParams.__dataclass_fields__})
    rho, g = W.standing_wave_fields(gp)
    th_drho, th_g = oic.thermal_fluctuation(p, 1000)
    sl = slabs.SlabSimulation(p, slabs.GlooComm(), rho - p.rho0 + th_drho, [g[a] + th_g[a] for a in range(3)])
    # particles start at rest (the no-slip start J v would need a serial pass)
    sl.add_particles(parts["q"], parts["m_e"], parts["kappa_ratio"], parts["k_spring"], np.zeros_like(parts["q"]))
    sl.run(warmup)
    dist.barrier()
    t0 = time.perf_counter()
    sl.run(steps)
    dist.barrier()
    el = time.perf_counter() - t0
    if rank == 0:
        queue.put(el)
    dist.destroy_process_group()


def oracle_all_cores(warmup, steps):
    """The oracle as it stands on every host core: the full 128^3 workload (10^4
    particles) split into z-slabs, one single-threaded process per core (the
    oracle's slab form, oracle/slabs.py, halo exchange over gloo).  Processes
    are spawned, not forked (this process may hold a CUDA context).
    Returns (seconds for the timed steps, processes)."""
    import socket

    import torch.multiprocessing as mp

    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    world = max(1, min(cores, 128 // 4))          # each slab keeps >= 4 planes beside its ghosts
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        queue = ctx.Queue()
        procs = [ctx.Process(target=_slab_worker, args=(r, world, port, warmup, steps, queue)) for r in range(world)]
        for pr in procs:
            pr.start()
        el = queue.get(timeout=900)
        for pr in procs:
            pr.join(timeout=120)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return el, world


def cpu_baseline(steps=10, single_budget=10.0):
    """The oracle as it stands: the full 128^3 workload on every host core
    (reported), and one thread on a 64^3 sub-box (beside it)."""
    el, world = oracle_all_cores(warmup=1, steps=steps)
    sim = oracle_sample()
    sim.step()   # warm-up (page-in, caches)
    t0 = time.perf_counter()
    n1 = 0
    while True:
        sim.step()
        n1 += 1
        el1 = time.perf_counter() - t0
        if el1 > single_budget or n1 >= 50:
            break
    cells = 128 ** 3
    return {"value": cells * steps / el, "unit": "cell-updates/s", "cores": world, "kind": "oracle",
            "sample": (f"the full 128^3 workload (1e4 particles, kT=1e-3), the oracle split into {world} z-slabs, one "
                       f"single-threaded numpy FP64 process per core (gloo halo exchange), {steps} steps in {el:.1f} s"),
            "cpu_model": cpu_model(), "particle_steps_per_s": 10000 * steps / el,
            "single_thread": {"value": 64 ** 3 * n1 / el1, "unit": "cell-updates/s", "cores": 1,
                              "sample": f"64^3 sub-box, 1250 particles, {n1} oracle steps in {el1:.1f} s"}}


def run_reference(args, rank, world):
    """The oracle as the reference arm: the full 128^3 workload on every host
    core (rank 0 only; other ranks exit without work)."""
    if rank != 0:
        return
    el, procs = oracle_all_cores(warmup=args.warmup, steps=args.steps)
    v = 128 ** 3 * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "cell-updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "same_config": True,
                       "sample": f"the full workload, oracle split into {procs} z-slabs, one process per core"},
            "particle_steps_per_s": 10000 * args.steps / el,
            "cpu_baseline": {"kind": "oracle", "cores": procs, "value": v, "cpu_model": cpu_model(),
                             "sample": f"each step: one oracle step of the full 128^3 workload on {procs} cores"},
            "e2e": {"value": v, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)



ADJOINT_METRIC = ("rollout-gradient steps/s (64^3, 16 tethered particles, 1000 steps, checkpoint every 50; "
                  "gradient of the time-averaged force w.r.t. m_e, kappa_p/kappa_f, A and the initial state)")
# the adjoint of the RK3 stage rates (the dominant adjoint kernel) per cell and launch:
# reads U_s (4 words) and the adjoint of U_{s+1} (4), writes gpart (3), rfbar (3), pibar (1)
ALG_ADJ_WORDS_PER_CELL = 15
# its floating-point operations as written once per cell (an FMA is 2, a division 1)
ALG_ADJ_FLOPS_PER_CELL = 280


def adjoint_record(prec, nsteps, warmup, flush, local, peak, peak_kind, peak64):
    """One differentiable rollout (the gradient of the time-averaged tether
    force, deterministic) timed forward and reversed: a unit of work is one
    step of the rollout run forward and reversed (checkpoints every 50 steps,
    each segment recomputed and its steps recorded and reversed)."""
    import torch

    from paper_1307_0702_gb300 import Grid, workloads as W
    from paper_1307_0702_gb300.adjoint import Rollout

    K = 50
    gp, rho, g, parts = W.line_config(64, 16, wave_amp=1e-3, precision=prec)
    cells = gp["nx"] * gp["ny"] * gp["nz"]
    grid = Grid(gp)
    grid.set_state(rho, g)
    grid.add_particles(parts["q"], parts["m_e"], parts["kappa_ratio"], parts["k_spring"], parts["u"])
    tiling = grid.autotune(reps=3)           # stage-kernel tiling for 64^3 (results do not depend on it)
    roll = Rollout(grid, parts["kappa_ratio"], checkpoint_every=K)
    roll.forward(np.ones(max(warmup, 3)))      # warm-up: graphs captured, snapshots allocated
    roll.backward()
    grid.snapshot_load(roll.checkpoints[0])
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    flush.fill_(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    phi = roll.forward(np.ones(nsteps))
    t1 = time.perf_counter()
    gr = roll.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    clocks = sampler.stop((t0, t2))
    # the same rollout once more with every kernel bracketed by events
    grid.snapshot_load(roll.checkpoints[0])
    grid.profile(True)
    roll.forward(np.ones(nsteps))
    roll.backward()
    prof = grid.profile_read()
    grid.profile(False)
    grid.close()
    st_ms, st_n = prof["adjoint_stage"]
    per_launch = st_ms / st_n * 1e-3
    words = 4 if prec == "fp32" else 8
    rec = {"value": nsteps / (t2 - t0), "unit": "rollout-gradient steps/s", "steps": nsteps, "phi": phi,
           "ms_per_step": 1e3 * (t2 - t0) / nsteps, "forward_ms_per_step": 1e3 * (t1 - t0) / nsteps,
           "reverse_ms_per_step": 1e3 * (t2 - t1) / nsteps,
           "cell_steps_per_s": cells * nsteps / (t2 - t0),
           "kernel_ms_per_step": {k: v[0] / nsteps for k, v in prof.items()},
           "launches_per_step": sum(v[1] for v in prof.values()) / nsteps,
           "grad_m_e_0": float(gr["m_e"][0]), "grad_A": float(gr["A"]), "clocks": clocks,
           "stage_tiling": list(tiling),
           "workload": "differentiable rollout: 64^3, 16 tethered particles on a line along x, A=1e-3, kT=0, "
                       "checkpoint every 50, wall time of the forward sweep and the reverse sweep"}
    if prec == "fp32":
        achieved = ALG_ADJ_WORDS_PER_CELL * words * cells / per_launch / 1e9
        rec["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                           "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                           "kernel": "k_adj_stage_rates (3 launches per reversed step)",
                           "alg_bytes_per_launch": ALG_ADJ_WORDS_PER_CELL * words * cells,
                           "note": "the 64^3 working set (15 fields, 16 MB) is L2-resident"}
    else:
        tflops = ALG_ADJ_FLOPS_PER_CELL * cells / per_launch / 1e12
        peak_tf, kind = (peak64["tflops"], "measured (ic_fma64_rate)") if peak64 else (FP64_PEAK_TFLOPS, "nominal")
        rec["roofline"] = {"bound": "alu", "achieved": tflops, "peak": peak_tf, "unit": "TFLOP/s",
                           "frac": tflops / peak_tf, "traffic": None, "peak_kind": kind,
                           "kernel": "k_adj_stage_rates (3 launches per reversed step)",
                           "alg_flops_per_launch": ALG_ADJ_FLOPS_PER_CELL * cells}
    return rec


def run_adjoint(args):
    """Differentiable rollout: FP32 is the line's value; FP64 rides along."""
    import torch

    nsteps = args.adj_steps
    peak, peak_kind = load_peaks()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device="cuda")
    peak64 = fp64_fma_peak(local) if "fp64" in args.adj_precision else None
    out = {prec: adjoint_record(prec, nsteps, args.warmup, flush, local, peak, peak_kind, peak64)
           for prec in args.adj_precision}
    r = out[args.adj_precision[0]]
    line = {
        "metric": ADJOINT_METRIC, "value": r["value"], "unit": r["unit"], "n_gpus": 1, "steps": nsteps,
        "warmup": max(args.warmup, 3), "ms_per_step": r["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.adj_precision[0] == "fp32" else "f64",
        "data": "synthetic",
        "config": {"workload": f"differentiable rollout: 64^3, 16 tethered particles on a line along x, A=1e-3, "
                               f"kT=0, {nsteps} steps, checkpoint every 50 ({args.adj_precision[0]}; "
                               f"each precision run in its own key)",
                   "l2": "flushed before the timed rollout; the 64^3 state stays L2-resident within it"},
        "roofline": r["roofline"], "gpu_launches": int(round(r["launches_per_step"] * nsteps)),
        "clocks": r["clocks"], **out,
    }
    if peak64:
        line["fp64_fma_peak"] = peak64
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = adjoint_cpu_baseline()
    print(json.dumps(line), flush=True)


def adjoint_cpu_baseline(nsteps=12):
    """The oracle's checkpointed reverse sweep on the same 64^3 line, a
    bounded number of steps."""
    from oracle import adjoint as oadj, ic as oic
    from paper_1307_0702_gb300 import workloads as W

    gp, rho, g, parts = W.line_config(64, 16, wave_amp=1e-3, precision="fp64")
    p = oic.GridParams(**{k: v for k, v in gp.items() if k in oic.GridParams.__dataclass_fields__})
    op = oadj.make_parts(parts["q"], parts["u"], parts["m_e"], parts["kappa_ratio"], parts["k_spring"], p.c)
    d = np.tile([1.0, 0.0, 0.0], (16, 1))
    t0 = time.perf_counter()
    oadj.rollout_gradient(p, rho - p.rho0, g, op, np.ones(nsteps), d, checkpoint_every=6)
    el = time.perf_counter() - t0
    return {"value": nsteps / el, "unit": "rollout-gradient steps/s", "cores": 1, "kind": "oracle",
            "sample": f"the same 64^3 line, {nsteps} steps, checkpoint every 6, {el:.1f} s (numpy FP64, 1 thread)"}


ENSEMBLE_METRIC = "cell-updates/s and particle-steps/s (ensemble of 256 boxes, edges 16/24/32/48, 1-200 particles)"


def run_ensemble(args):
    """Batched ensemble: 256 FP32 boxes advanced by ic_batch_step after
    ic_batch_autotune; beside it the same ensemble with the default tiling,
    as one captured graph per ensemble step, and unbatched (one ic_step per
    box per step)."""
    import torch

    from paper_1307_0702_gb300 import Batch, workloads as W

    cfg = W.ensemble_config(args.boxes)
    grids = [setup_box(gp, parts, seed_thermal=5000 + b) for b, (gp, parts) in enumerate(cfg)]
    cells = sum(g.shape[0] * g.shape[1] * g.shape[2] for g in grids)
    npart = sum(g.n_particles for g in grids)
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device="cuda")
    s0 = grids[0].stream

    def timed(step_fn, steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        for i in range(steps):
            with torch.cuda.stream(s0):
                flush.fill_(i & 0xFF)
                ev[i][0].record(s0)
            step_fn()
            with torch.cuda.stream(s0):
                ev[i][1].record(s0)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        return float(np.sum([a.elapsed_time(b) for a, b in ev])) / 1e3, wall

    def unbatched():
        for g in grids:
            g.step(1)
        # the end event waits for every box
        for g in grids[1:]:
            e = torch.cuda.Event()
            e.record(g.stream)
            s0.wait_event(e)

    batch = Batch(grids)
    batch.step(args.warmup)
    t_default, wall_default = timed(lambda: batch.step(1), args.steps)
    tiles = batch.autotune(reps=3)
    batch.step(args.warmup)
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    time.sleep(0.3)
    w0 = time.perf_counter()
    t_batch, wall_batch = timed(lambda: batch.step(1), args.steps)
    clocks = sampler.stop((w0, time.perf_counter()))
    os.environ["IC_BATCH_GRAPH"] = "1"        # the whole ensemble step as one graph
    batch.step(args.warmup)
    t_one, wall_one = timed(lambda: batch.step(1), args.steps)
    os.environ.pop("IC_BATCH_GRAPH")
    for g in grids:
        g.step(args.warmup)
    t_unb, wall_unb = timed(unbatched, args.steps)
    by_edge = {}
    for g, t in zip(grids, tiles):
        by_edge.setdefault(str(g.shape[2]), [list(t)])
    line = {
        "metric": ENSEMBLE_METRIC, "value": cells * args.steps / t_batch, "unit": "cell-updates/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_batch / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "ensemble: 256 FP32 boxes, edges uniform in {16,24,32,48}, 1-200 particles each "
                               "(min sep 2h), kT=1e-3, Philox seed = box index, ic_batch_step",
                   "boxes": len(grids), "cells": cells, "particles": npart,
                   "l2": "flushed between timed steps (512 MB write, outside the step events)"},
        "particle_steps_per_s": npart * args.steps / t_batch,
        "tiles_by_edge": {k: v[0] for k, v in sorted(by_edge.items(), key=lambda kv: int(kv[0]))},
        "default_tiling": {"value": cells * args.steps / t_default, "ms_per_step": 1e3 * t_default / args.steps},
        "one_graph_per_step": {"value": cells * args.steps / t_one, "ms_per_step": 1e3 * t_one / args.steps,
                               "wall_ms_per_step": 1e3 * wall_one / args.steps},
        "unbatched": {"value": cells * args.steps / t_unb, "ms_per_step": 1e3 * t_unb / args.steps,
                      "wall_ms_per_step": 1e3 * wall_unb / args.steps},
        "wall_ms_per_step": 1e3 * wall_batch / args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    batch.close()
    for g in grids:
        g.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--particles", type=int, default=10000)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sub", action="store_true", help="skip the FP64 and ensemble records beside the headline")
    ap.add_argument("--sub-steps", type=int, default=20)
    ap.add_argument("--long-steps", type=int, default=2000,
                    help="steps of the long-run sub-record (amortised rebuilds)")
    ap.add_argument("--adj-steps", type=int, default=1000)
    ap.add_argument("--sub-adj-steps", type=int, default=1000,
                    help="steps of the FP32 differentiable-rollout record beside the headline")
    ap.add_argument("--adj-precision", nargs="+", default=["fp32", "fp64"], choices=["fp32", "fp64"])
    ap.add_argument("--workload", default="box", choices=["box", "ensemble", "adjoint"],
                    help="box: the 128^3 single box (default); ensemble: the batched 256-box ensemble")
    ap.add_argument("--boxes", type=int, default=256)
    ap.add_argument("--tile", type=int, nargs=2, metavar=("TILE_X", "ZCHUNK"), default=None,
                    help="fixed stage-kernel tiling instead of the autotuner's (e.g. for profiling)")
    ap.add_argument("--stage-copy", default="auto", choices=["auto", "thread", "bulk", "rows16"],
                    help="loads of the FP32 wide stage tile: the autotuner's choice, per-thread copies, "
                         "TMA bulk row copies or 16-byte row copies")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if args.workload == "ensemble":
        if rank == 0:
            run_ensemble(args)
        return
    if args.workload == "adjoint":
        if rank == 0:
            run_adjoint(args)
        return
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1307_0702_gb300 import workloads as W

    gp, parts = W.large_box_config(args.n, args.particles)
    gp["precision"] = args.precision
    gp["box"] = rank
    grid = setup_box(gp, parts, seed_thermal=1000 + rank)
    cells = gp["nx"] * gp["ny"] * gp["nz"]
    npart = parts["q"].shape[0]
    stream = grid.stream
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    # stage-kernel tiling picked by the library's autotuner, then warm-up (captures the graphs)
    if args.tile:
        grid.set_tile(*args.tile)
        tiling = grid.tile()
    else:
        tiling = grid.autotune(reps=3)
    if args.stage_copy != "auto":
        grid.set_stage_copy(args.stage_copy)
    stage_copy = grid.stage_copy()
    grid.step(args.warmup)
    grid.sync()

    # timed region: K steps, each bracketed by events on the library's stream, L2 flushed in between
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    barrier()
    sampler.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
        grid.step(1)
        with torch.cuda.stream(stream):
            ev[i][1].record(stream)
    barrier()
    wall1 = time.perf_counter()
    wall = wall1 - wall0
    clocks = sampler.stop((wall0, wall1))
    grid.sync()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_local = float(np.sum(step_ms)) / 1e3
    t = torch.tensor([t_local], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t_max = float(t.item())
    value = world * cells * args.steps / t_max
    pvalue = world * npart * args.steps / t_max

    # kernel timing pass: same steps with events around every kernel (graphs
    # off).  Launching kernel by kernel, the host is slower than the GPU; a
    # 4 ms sleep on the stream before every 8 steps lets the host queue them
    # first, so that no event pair also times a launch gap.
    grid.profile(True)
    for i in range(args.steps):
        if i % 8 == 0:
            with torch.cuda.stream(stream):
                torch.cuda._sleep(8_000_000)
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xFF)
        grid.step(1)
    prof = grid.profile_read()
    grid.profile(False)
    fluid_ms, fluid_launches = prof["fluid"]
    part_ms, part_launches = prof["particles"]
    end_ms, end_launches = prof["end"]
    launches_per_step = (fluid_launches + part_launches + end_launches) / args.steps
    peak, peak_kind = load_peaks()
    alg_bytes = ALG_BYTES_PER_CELL_STEP[args.precision] * cells       # per step = per 3 stage launches
    stage_ms_per_step = fluid_ms / args.steps
    achieved = alg_bytes / (stage_ms_per_step * 1e-3) / 1e9
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "stage_traffic.json")
    if os.path.exists(tfile):
        with open(tfile) as f:
            tj = json.load(f)
        # ncu DRAM bytes of the same kernel (same precision, size and tile width)
        if (tj.get("precision") == args.precision and tj.get("cells") == cells
                and tj.get("tile_x") == tiling[0] and tj.get("kernel_rev") == STAGE_KERNEL_REV
                and tj.get("stage_copy", "thread") == stage_copy):
            traffic = tj.get("bytes_per_launch")

    # end-to-end through the public API with host buffers: one step per call,
    # its averaging weight uploaded from pinned memory, the step's result -- the
    # constraint force lambda on every particle, and the device status word --
    # copied back every step (ic_forces_async into one of two pinned slots) and
    # read on the host while the next step runs (ic_forces_collect)
    e2e = None
    if not args.no_e2e:
        pinned_w = torch.ones(1, dtype=torch.float64).pin_memory().numpy()
        lam = np.empty((npart, 3))
        grid.step(1, pinned_w)
        grid.forces_async(0)
        grid.forces_collect(0, lam)
        barrier()
        t0 = time.perf_counter()
        for i in range(args.steps):
            grid.step(1, pinned_w)
            grid.forces_async(i & 1)
            if i:
                grid.forces_collect((i - 1) & 1, lam)
        grid.forces_collect((args.steps - 1) & 1, lam)
        barrier()
        el = time.perf_counter() - t0
        tt = torch.tensor([el], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        el = float(tt.item())
        # bytes the library moves: weight + (first step, count) header in; lambda
        # in the state precision + the device status word out
        e2e = {"value": world * cells * args.steps / el, "unit": "cell-updates/s",
               "h2d_bytes_per_step": 8 + 16,
               "d2h_bytes_per_step": 3 * npart * (4 if args.precision == "fp32" else 8) + 4,
               "particle_steps_per_s": world * npart * args.steps / el}

    # beside the headline: the plain FP64 form of the same box and the FP32
    # batched ensemble, each timed like the headline (rank 0 of a 1-GPU run)
    subs = {}
    if rank == 0 and world == 1 and args.precision == "fp32" and not args.no_sub:
        peak64 = fp64_fma_peak(local)
        subs["fp64_fma_peak"] = peak64
        subs["fp64"] = sub_fp64(args.sub_steps, 3, local, flush, peak64)
        subs["ensemble"] = sub_ensemble(args.sub_steps, 3, local, flush)
        subs["long_run"] = sub_long_run(args.long_steps, local)
        pk, pk_kind = load_peaks()
        subs["adjoint"] = adjoint_record("fp32", args.sub_adj_steps, 3, flush, local, pk, pk_kind, peak64)
        subs["force_accuracy"] = sub_force_accuracy()

    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline()

    if args.precision == "fp32":
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": traffic, "peak_kind": peak_kind, "traffic_unit": "bytes per launch",
                    "alg_bytes_per_launch": alg_bytes / 3, "alg_bytes_per_step": alg_bytes}
    else:
        tflops = ALG_FP64_FLOPS_PER_CELL_STEP * cells / (stage_ms_per_step * 1e-3) / 1e12
        pk = fp64_fma_peak(local)
        peak_tf, peak_kind64 = (pk["tflops"], "measured (ic_fma64_rate)") if pk else (FP64_PEAK_TFLOPS, "nominal")
        roofline = {"bound": "alu", "achieved": tflops, "peak": peak_tf, "unit": "TFLOP/s",
                    "frac": tflops / peak_tf, "traffic": None, "peak_kind": peak_kind64, "fp64_fma_peak": pk,
                    "alg_flops_per_step": ALG_FP64_FLOPS_PER_CELL_STEP * cells,
                    "hbm_frac_for_reference": achieved / peak}
    kname = "k_stage_rows" if tiling[0] == gp["nx"] and args.precision == "fp32" else "k_rk3_stage"
    roofline.update({"kernel": f"{kname} (3 launches per step)", "stage_ms_per_step": stage_ms_per_step,
                     "particle_ms_per_step": part_ms / args.steps, "end_ms_per_step": end_ms / args.steps})
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": cells, "particles": npart, "precision": args.precision,
                       "parallelism": f"{world} independent boxes (one per GPU)",
                       "l2": "flushed between timed steps (512 MB write, outside the step events)",
                       "stage_tiling": list(tiling), "stage_copy": stage_copy, "particle_steps_per_s": pvalue},
            "particle_steps_per_s": pvalue,
            "roofline": roofline,
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": base,
            "wall_s_timed": wall,
        }
        line.update(subs)
        print(json.dumps(line), flush=True)
    grid.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
