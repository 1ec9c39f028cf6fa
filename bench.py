#!/usr/bin/env python
"""Benchmark of the UGKWP time step on GB300.

Workload: the 1D frequency-dependent slab (200 cells, 30 log groups on
nu in [1e-3, 10], sigma = 1e2 nu^-3 T^-1/2 capped at 1e6, black body T = 1
into T = 1e-3, dt = 1e-4, FP64), started from a seeded synthetic mid-run
Marshak-front state holding 1e6 particles (the regime the 500-step run
reaches).  A step is one pass of the whole hot path: birth counts and scan,
wave flux, the particle kernel (sampling, streaming with t_f reset, tallies,
compaction) and the source iteration.

Metric: particle segments per second over the timed steps (device time from
CUDA events on the launching stream, L2 flushed between timed steps), plus
steps/s.  `--impl reference` times the CPU oracle on the same workload.
Launch: `python bench.py --gpus N --steps K --warmup W`; for N > 1 under
torch.distributed.run each rank runs an independent replica (the method has
no cross-problem exchange) and the job value is the sum over ranks.
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
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2312_16981_gb300 import inputs as I  # noqa: E402

N_PARTICLES = 1_000_000
WORKLOAD = "multigroup_slab_200x30"
METRIC = "particle segments/s"
# kernels of one slab step: birth, one-block scan, wave flux, the particle
# kernel (FP64: k_stream64; mixed: the survivor kernel, which also streams
# the newborns), source iteration, the survivor sort (a one-block scan and
# the scatter) and the end of step
KERNELS_PER_STEP = {"fp64": 8, "mixed": 8}
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per processed
# particle of the particle kernel, from one ncu capture of the current kernel
# on the slab's 1e6-particle state (the benchmark's workload; the survivors'
# writes are still in L2 when the kernel ends); the roofline's "traffic" is
# this times the particles a launch processes.  None: no capture of the
# current kernel.
TRAFFIC_PER_PROCESSED = {"fp64": None, "mixed": 27.1}


def combine_replicas(ms: float, segments: float, world: int, device):
    """Job totals over independent replicas (one per rank): the slowest rank's
    time and the sum of the segments every rank streamed.  No data exchange
    is part of the method; this is the only collective, outside the timed
    region."""
    if world <= 1:
        return ms, segments
    import torch
    import torch.distributed as dist
    mx = torch.tensor([ms], dtype=torch.float64, device=device)
    sm = torch.tensor([segments], dtype=torch.float64, device=device)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[0])


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def workload(rank: int = 0, n_particles: int = N_PARTICLES, name: str = "slab"):
    if name == "checkerboard":
        p = I.checkerboard_2d()
        p.instance = rank
        p.particle_capacity = max(p.particle_capacity, int(n_particles * 1.6))
        return p, I.synthetic_state(p, n_particles, seed=3, front=0.35)
    p = I.multigroup_slab()
    p.instance = rank
    p.particle_capacity = max(p.particle_capacity, int(n_particles * 1.5))
    s = I.synthetic_state(p, n_particles, seed=1)
    return p, s


def config_dict(p, n_particles, extra=None):
    d = {"workload": WORKLOAD if p.dim == 1 else p.name, "cells": p.ncell, "groups": p.G, "dt": p.dt,
         "particles_at_start": n_particles, "state": "seeded synthetic Marshak front",
         "l2": "flushed between timed steps (512 MiB write)"}
    if extra:
        d.update(extra)
    return d


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.strip() == "Active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "reasons": reasons, "samples": len(rows)}


def oracle_segments_per_s(p, s, n_sample, steps, warmup=0):
    """The CPU oracle as it stands, on `steps` steps of a bounded sample after
    `warmup` untimed steps."""
    import oracle as O
    op = O.OracleProblem(p)
    parts = {k: v[:n_sample] for k, v in s["particles"].items()} if n_sample else s["particles"]
    st = O.State(p, s["T"].copy(), s["rho"].copy(), s["rho_h"].copy(),
                 O.ParticleSet.from_arrays(parts, cap=max(len(parts["id"]) * 2, 1 << 16)), s["step"])
    segs, t = 0, 0.0
    for k in range(warmup + steps):
        t0 = time.perf_counter()
        st2, tal, _, status = O.step(op, st, cap_out=max(st.particles.n * 2, 1 << 16))
        if k >= warmup:
            t += time.perf_counter() - t0
            segs += tal.c.n_segments
        st = st2
    return segs, t


# The CPU baseline, one protocol for both places it is reported (the
# cpu_baseline object and the --impl reference arm): the oracle, one core, on
# the workload's state with its first ORACLE_SAMPLE particles (the newborns of
# every step are the whole workload's: births depend on the wave part, not on
# the sample), one untimed step, then ORACLE_STEPS timed steps; segments per
# second over the timed steps.  Its cost per step grows with the particles
# alive (the source iteration is a fixed cost), so the protocol fixes both.
ORACLE_SAMPLE = 100_000
ORACLE_STEPS = 3


def oracle_protocol(p, s):
    segs, t = oracle_segments_per_s(p, s, ORACLE_SAMPLE, ORACLE_STEPS, warmup=1)
    return segs, t


def _oracle_replica(args):
    """One oracle replica for the parallel CPU baseline: its own slice of the
    workload's particles, the protocol of oracle_protocol (one untimed step,
    ORACLE_STEPS timed ones, the full source iteration each step)."""
    k, n_sample, particles = args
    p, s = workload(0, particles)
    sl = slice(k * n_sample, (k + 1) * n_sample)
    s = dict(s, particles={f: v[sl] for f, v in s["particles"].items()})
    return oracle_segments_per_s(p, s, 0, ORACLE_STEPS, warmup=1)


def host_cpu():
    """Core count and CPU model of this host (for the CPU baseline)."""
    import platform
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part"):
                    model = "%s (%s %s)" % (platform.machine(), key, line.split(":", 1)[1].strip())
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count() or 1, "model": model}


def oracle_parallel(n_sample, particles):
    """The oracle as N independent replicas (one per host core, processes
    started with spawn), each on its own particle slice: total segments over
    the slowest replica's compute time."""
    import multiprocessing as mp
    n = max(1, min(os.cpu_count() or 1, particles // n_sample))
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map(_oracle_replica, [(k, n_sample, particles) for k in range(n)])
    return sum(r[0] for r in res) / max(r[1] for r in res), n


def protocol_text(n_particles):
    return ("the oracle on one core: the workload's state with its first %d of %d particles, one untimed "
            "step, then %d timed steps (full 200x30 source iteration each step; the newborns are the "
            "whole workload's)" % (ORACLE_SAMPLE, n_particles, ORACLE_STEPS))


def run_reference(args):
    """The reference arm: the CPU oracle under the protocol of oracle_protocol,
    repeated min(max(1, steps // ORACLE_STEPS), 4) times from the same state
    (so the arm ends within minutes), so that its figure and the
    cpu_baseline object measure the same thing."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    p, s = workload()
    reps = min(max(1, args.steps // ORACLE_STEPS), 4)
    segs = t = 0.0
    for _ in range(reps):
        sg, tt = oracle_protocol(p, s)
        segs += sg
        t += tt
    v = segs / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "segments/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / (reps * ORACLE_STEPS), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(p, N_PARTICLES, {"sample": "first %d of %d particles" % (ORACLE_SAMPLE, N_PARTICLES)}),
            "cpu_baseline": {"value": v, "unit": "segments/s", "cores": 1, "kind": "oracle",
                             "sample": protocol_text(N_PARTICLES) + "; repeated %d times" % reps,
                             "host": host_cpu()},
            "e2e": {"value": v, "unit": "segments/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# FP64 operations (an FMA counted as two) of the source iteration per (cell,
# group) and FP64 iterate as the kernel executes them (App. B: the
# equilibrium fluxes of the faces, the closed-form T and rho updates, the
# Planck edge interpolants and group fractions, the Simpson group opacity,
# tau and q; prologue and epilogue shared out over the iterates), counted by
# ncu (2 x DFMA + DADD + DMUL thread instructions): the 200x30 slab, FP64
# build, 3 iterates a launch; the 2D checkerboard, mixed build with the FP32
# warm start, 4 FP64 iterates a launch (its FP32 iterates add time, not FP64
# operations).  3D takes the 2D figure.
SI_FLOPS_PER_CELL_GROUP = {1: 235, 2: 197, 3: 197}
# FP64 peak of the chip: 152 SMs x 4 sub-partitions x 0.5 FMA lanes a cycle
# x 2 flops x the maximum SM clock
FP64_PEAK_TFLOPS = 152 * 4 * 0.5 * 2 * 2.07e9 / 1e12


def algorithmic_bytes(p, phase, n_read, n_out, si_iters, mixed=False):
    """Algorithmic HBM bytes of one launch of a phase: the particle kernels
    read the state of each particle alive at step start (newborns are born in
    registers) and write each survivor once -- x (, y), mu (, Omega_y), nu, w
    and the 64-bit identity: 24 B (1D) or 32 B (2D) in mixed precision, 40 B or
    56 B in FP64, the cell implied by the sort -- plus the tallies and bin
    tables."""
    ncg = p.ncell * p.G
    if phase == "particles":
        nf = 2 * p.dim + 2
        per = nf * (4 if mixed else 8) + 8
        return per * n_read + per * n_out + 3 * 8 * ncg + 3 * 8 * p.nbins
    return 0


def roofline(p, phase, launch_ms, n_proc, n_read, n_out, si_iters, mixed, pk, src):
    """Roofline of one phase from its CUDA-event duration (kernel by kernel):
    the particle kernels against HBM (algorithmic bytes per launch), the
    source iteration against the FP64 pipe (its FP64 operations per launch;
    it moves a few arrays of cells x groups per iterate, far from any HBM
    bound)."""
    if phase == "source_iteration":
        flops = SI_FLOPS_PER_CELL_GROUP[p.dim] * p.ncell * p.G * si_iters
        ach = flops / (launch_ms * 1e-3) / 1e12
        return {"kernel": "k_si", "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_source": "FP64 pipe from unit counts and the maximum SM clock (152 SMs x 4 x 0.5 FMA/cycle x 2 x 2.07 GHz)",
                "algorithmic_flops_per_launch": flops, "iterates_per_launch": si_iters, "launch_ms": launch_ms,
                "note": "FP64 operations of the kernel, %d per (cell, group) and FP64 iterate (ncu count); latency-bound on small grids" % SI_FLOPS_PER_CELL_GROUP[p.dim]}
    abytes = algorithmic_bytes(p, phase, n_read, n_out, si_iters, mixed=mixed)
    ach = abytes / (launch_ms * 1e-3) / 1e9 if abytes else 0.0
    tpp = TRAFFIC_PER_PROCESSED["mixed" if mixed else "fp64"]
    traffic = tpp * n_proc if (phase == "particles" and p.dim == 1 and tpp) else None
    r = {"kernel": {"particles": ("k_stream32_fast" if (mixed and p.dim == 1) else "k_stream32")
                    if mixed else "k_stream64"}.get(phase, phase),
         "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
         "frac": ach / pk["hbm_gbs"], "traffic": traffic, "peak_source": src,
         "algorithmic_bytes_per_launch": abytes, "launch_ms": launch_ms,
         "bytes_per_particle": (2 * p.dim + 2) * (4 if mixed else 8) + 8}
    if traffic is not None:
        r["traffic_source"] = "ncu capture of the same kernel on the 1e6-particle slab state, scaled by particles processed per launch"
    if phase == "particles" and not mixed:
        r["note"] = "FP64-pipe bound on GB300 (see profiles/): HBM is not the limit of this kernel"
    return r


def timed_steps(sim, steps, flush, sampler=None):
    """Device time per step (CUDA events) with L2 flushed between steps."""
    import torch
    phases = np.zeros(6)
    segs = n_proc = n_read = n_out = si = 0
    torch.cuda.synchronize()
    for _ in range(steps):
        flush.fill_(1)
        ms = sim.step_timed()
        t = sim.tallies()
        phases += np.array(ms)
        segs += t["n_segments"]
        n_proc += t["n_in"] + t["n_born"]
        n_read += t["n_in"]
        n_out += t["n_survived"]
        si += t["si_iters"]
    torch.cuda.synchronize()
    assert t["status_bits"] == 0, t["status_bits"]
    return phases, segs, (n_proc, n_read), n_out, si


def graph_steps(sim, steps, flush):
    """Device time of `steps` whole steps replayed as the library's CUDA graph
    (ugkwp_step), CUDA events on the launching stream around each step, L2
    flushed before each; counters from the tally report after each step."""
    import torch
    ms = 0.0
    segs = n_proc = n_read = n_out = si = 0
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    for _ in range(steps):
        flush.fill_(1)
        a.record()
        sim.step(1)
        b.record()
        b.synchronize()
        ms += a.elapsed_time(b)
        t = sim.tallies()
        segs += t["n_segments"]
        n_proc += t["n_in"] + t["n_born"]
        n_read += t["n_in"]
        n_out += t["n_survived"]
        si += t["si_iters"]
    assert t["status_bits"] == 0, t["status_bits"]
    return ms, segs, (n_proc, n_read), n_out, si


def device_ms(fn, flush=None):
    """Device milliseconds of fn() on the current stream (CUDA events)."""
    import torch
    if flush is not None:
        flush.fill_(1)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    fn()
    b.record()
    b.synchronize()
    return a.elapsed_time(b)


def ensemble_leg(B, dev, flush, steps, warmup, members=256, evolve=100, autotune_cache=None):
    """256 independent slabs with uneven cells, groups, opacity and boundary
    temperature, each run from its cold initial state for `evolve` steps
    (its reference weight is set so that about 1e4-1e6 particles are alive
    by then): one batched (mixed precision, autotuned) step against the same
    members stepped one after another, in FP64 and in mixed precision.  All
    three are timed the same way: CUDA events around one step of every
    member (CUDA graph replay), L2 flushed before each step."""
    probs = I.ensemble_slabs(members, steps=evolve)
    for p in probs:
        target = 0.25 * p.bcT[0] ** 4 * p.dt * evolve / p.omega_ref
        p.particle_capacity = int(2.0 * target) + 65536

    def segments(sims_members):
        tot = alive = 0
        for sim, mm in sims_members:
            t = sim.tallies(member=mm)
            assert t["status_bits"] == 0, (mm, t["status_bits"])
            tot += t["n_segments"]
            alive += t["n_particles"]
        return tot, alive

    out = {"members": members, "evolved_steps": evolve,
           "cells_x_groups": int(sum(p.ncell * p.G for p in probs))}
    # batched, mixed precision, autotuned launch shape
    ens = B.Simulation([p.replace(precision=I.MIXED) for p in probs], device=dev)
    ens.step(evolve)
    out["particles_alive"] = segments([(ens, m) for m in range(members)])[1]
    tune = ens.autotune(steps=2, cache=autotune_cache)
    for _ in range(max(warmup, 3)):
        ens.step(1)
    ms = segs = 0.0
    for _ in range(steps):
        ms += device_ms(lambda: ens.step(1), flush)
        segs += segments([(ens, m) for m in range(members)])[0]
    out["batched_mixed"] = {"value": segs / (ms / 1e3), "unit": "segments/s",
                            "ms_per_step": ms / steps, "launch_shape": tune}
    ens.close()
    del ens
    # the same members one after another, one graph each
    for name, prec in (("sequential_fp64", I.FP64), ("sequential_mixed", I.MIXED)):
        sims = [B.Simulation(p.replace(precision=prec), device=dev) for p in probs]
        for sm in sims:
            sm.step(evolve + max(warmup, 3))

        def all_one():
            for sm in sims:
                sm.step(1)
        ms = segs = 0.0
        for _ in range(steps):
            ms += device_ms(all_one, flush)
            segs += segments([(sm, 0) for sm in sims])[0]
        out[name] = {"value": segs / (ms / 1e3), "unit": "segments/s", "ms_per_step": ms / steps}
        for sm in sims:
            sm.close()
        del sims
    b = out["batched_mixed"]["value"]
    out["speedup_batched_mixed_vs_sequential_fp64"] = b / out["sequential_fp64"]["value"]
    out["speedup_batched_mixed_vs_sequential_mixed"] = b / out["sequential_mixed"]["value"]
    return out


def paired_error_stats(e_mixed, e_fp64):
    """Tally errors of the two builds on the same seeds (common random
    numbers): the ratio of the mean errors, and the paired difference
    mean(e_mixed - e_fp64) / mean(e_fp64) with its standard error, whose
    noise is far below either error's own (the same draws on both sides).
    Matched: the mixed build is worse by at most 5 %, at two standard
    errors."""
    em, ef = np.asarray(e_mixed), np.asarray(e_fp64)
    d = em - ef
    mf = float(np.mean(ef))
    rel = float(np.mean(d)) / mf
    se = float(np.std(d, ddof=1) / np.sqrt(len(d))) / mf if len(d) > 1 else float("inf")
    return {"error_ratio_mixed_over_fp64": float(np.mean(em)) / mf, "paired_rel_diff": rel,
            "paired_rel_diff_stderr": se, "matched": bool(rel + 2.0 * se <= 0.05)}


def flip_fraction(B, dev, probs, states):
    """One step of the FP64 and the mixed builds from the same state with
    per-particle records: the fraction of particles whose fate, end cell or
    number of segments differs (event flips of the FP32 arithmetic)."""
    out = []
    for prec in (I.FP64, I.MIXED):
        recs = []
        for p, st in zip(probs, states):
            sim = B.Simulation(p.replace(precision=prec), device=dev)
            sim.set_state(st["T"], st["rho"], st["rho_h"], st["particles"], step=st["step"])
            n_cap = 2 * len(st["particles"]["id"]) + 1_000_000
            sim.attach_records(min(n_cap, 40_000_000))
            sim.step(1)
            t = sim.tallies()
            recs.append(sim.records(t["n_in"] + t["n_born"]))
            sim.close()
        out.append(recs)
    n = flips = 0
    for ra, rb in zip(*out):
        m = min(len(ra), len(rb))
        same_id = ra["id"][:m] == rb["id"][:m]
        diff = (ra["fate"][:m] != rb["fate"][:m]) | (ra["cell1"][:m] != rb["cell1"][:m]) | (ra["nseg"][:m] != rb["nseg"][:m])
        n += int(same_id.sum())
        flips += int((diff & same_id).sum())
    return {"particles": n, "flips": flips, "fraction": flips / max(n, 1)}


def matched_error_run(B, dev, probs, steps, seeds, refine, what, cap_scale=1.0):
    """Tally error of the mixed build against the FP64 build on a set of
    problems (one, or an ensemble's members), each run from its initial
    state for `steps` steps: the reference is the mean of `seeds` FP64 runs
    with `refine` times the particles (omega_ref / refine); each build then
    runs seeds 1..seeds at the problems' omega_ref; the error of a run is the
    relative RMS temperature difference from the reference over the cells
    the front reached (T_ref > 2 T0), all problems together."""
    batched = len(probs) > 1

    def run(prec, seed, refine_by):
        ps = [p.replace(precision=prec, omega_ref=p.omega_ref / refine_by, seed=seed,
                        particle_capacity=int(p.particle_capacity * refine_by * cap_scale)) for p in probs]
        sim = B.Simulation(ps if batched else ps[0], device=dev)
        sim.step(steps)
        Ts, sts, n = [], [], 0
        for m in range(len(ps)):
            t = sim.tallies(member=m)
            assert t["status_bits"] == 0, t["status_bits"]
            g = sim.get_state(member=m)
            Ts.append(g["T"])
            n += g["n"]
            sts.append({"T": g["T"], "rho": g["rho"], "rho_h": g["rho_h"], "particles": g["particles"], "step": steps})
        sim.close()
        return Ts, n, sts

    refs = [run(I.FP64, 1000 + r, refine)[0] for r in range(seeds)]
    Tref = [np.mean([r[m] for r in refs], axis=0) for m in range(len(probs))]
    hot = [Tref[m] > 2.0 * float(np.min(probs[m].T0)) for m in range(len(probs))]

    def rel_rms(Ts):
        num = np.concatenate([((Ts[m] - Tref[m]) / Tref[m])[hot[m]] for m in range(len(probs))])
        return float(np.sqrt(np.mean(num ** 2))) if num.size else float("nan")
    errs, same, last_states, alive = {}, [], None, {}
    runs = {}
    for name, prec in (("fp64", I.FP64), ("mixed", I.MIXED)):
        rs = [run(prec, 1 + r, 1.0) for r in range(seeds)]
        runs[name] = rs
        errs[name] = [rel_rms(r[0]) for r in rs]
        alive[name] = int(np.mean([r[1] for r in rs]))
        if name == "fp64":
            last_states = rs[0][2]
    for a, b in zip(runs["fp64"], runs["mixed"]):
        same.append(max(float(np.max(np.abs(x - y) / x)) for x, y in zip(a[0], b[0])))
    res = {"what": what, "hot_cells": int(sum(h.sum() for h in hot)), "seeds": seeds, "refine": refine,
           "steps": steps, "fp64": {"rel_rms_T_error": float(np.mean(errs["fp64"])), "per_seed": errs["fp64"],
                                    "particles_at_end": alive["fp64"]},
           "mixed": {"rel_rms_T_error": float(np.mean(errs["mixed"])), "per_seed": errs["mixed"],
                     "particles_at_end": alive["mixed"]},
           "same_seed_max_rel_T_diff_mixed_vs_fp64": max(same),
           "reference_self_noise_estimate": float(np.mean([np.std([r[m] for r in refs], axis=0)[hot[m]].mean()
                                                           / Tref[m][hot[m]].mean() for m in range(len(probs))
                                                           if hot[m].any()]) / np.sqrt(seeds))}
    res.update(paired_error_stats(errs["mixed"], errs["fp64"]))
    res["flips_one_step"] = flip_fraction(B, dev, probs, last_states)
    return res


def matched_error_leg(B, dev, steps=500, seeds=8, refine=16):
    """The 200x30 slab from its initial state (500 steps)."""
    base = I.multigroup_slab()
    base.particle_capacity = 1 << 23
    return matched_error_run(B, dev, [base], steps, seeds, refine,
                             "%d steps of the 200x30 slab from its initial state; reference = mean of %d FP64 runs at "
                             "omega_ref/%d; error = relative RMS of T over the cells the front reached, per seed"
                             % (steps, seeds, refine))


def matched_error_checkerboard(B, dev, steps=20, seeds=4, refine=4):
    """The 2D 256x256 checkerboard (30 groups) from its initial state."""
    p = I.checkerboard_2d()
    return matched_error_run(B, dev, [p], steps, seeds, refine,
                             "%d steps of the 256x256x30 checkerboard from its initial state; reference = mean of %d "
                             "FP64 runs at omega_ref/%d" % (steps, seeds, refine), cap_scale=1.0)


def matched_error_ensemble(B, dev, members=32, steps=100, seeds=4, refine=4):
    """The first `members` slabs of the batched ensemble, run batched."""
    probs = I.ensemble_slabs(256, steps=steps)[:members]
    for p in probs:
        p.particle_capacity = int(2.0 * 0.25 * p.bcT[0] ** 4 * p.dt * steps / p.omega_ref) + 65536
    return matched_error_run(B, dev, probs, steps, seeds, refine,
                             "%d steps of the first %d ensemble slabs run batched from their initial states; "
                             "reference = mean of %d batched FP64 runs at omega_ref/%d" % (steps, members, seeds, refine))


def checkerboard_leg(B, dev, flush, steps, warmup, n_particles):
    """The 2D 256x256 checkerboard (30 groups, thick/thin 16x16 blocks,
    central T_s = 1 source) from a seeded synthetic state with n_particles
    particles: FP64 and mixed precision builds, whole steps as CUDA-graph
    replays, then a few kernel-by-kernel steps for the phase times."""
    p = I.checkerboard_2d()
    p.particle_capacity = max(p.particle_capacity, int(1.6 * n_particles))
    s = I.synthetic_state(p, n_particles, seed=3, front=0.35)
    out = {"workload": "checkerboard_2d_256x256x30", "particles_at_start": n_particles}
    names = ["total", "birth_scan", "wave", "particles", "source_iteration", "end"]
    for name, prec in (("fp64", I.FP64), ("mixed", I.MIXED)):
        sim = B.Simulation(p.replace(precision=prec), device=dev)
        sim.set_state(s["T"], s["rho"], s["rho_h"], s["particles"], step=s["step"])
        for _ in range(max(warmup, 3)):
            sim.step(1)
        ms, segs, (n_in, _), n_out, si = graph_steps(sim, steps, flush)
        ph, _, _, _, _ = timed_steps(sim, max(2, steps // 2), flush)
        out[name] = {"value": segs / (ms / 1e3), "unit": "segments/s", "ms_per_step": ms / steps,
                     "phase_ms_per_step": {n: float(ph[i] / max(2, steps // 2)) for i, n in enumerate(names)},
                     "particles_per_step": n_in / steps, "si_iters_per_step": si / steps}
        sim.close()
        del sim
    out["speedup_mixed_vs_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    return out


def adjoint_leg(B, dev, steps=200, ckpt_every=20, n_fd=64, h=1e-6):
    """Gradient of L = sum (T - T_target)^2 after 200 steps of the 2D 128x128x16
    grid with respect to the 16384 per-cell log-opacity scales s ~ N(0, 0.1):
    the adjoint (checkpoint every 20 steps) timed against the forward run, and
    checked on 64 random cells against central differences with common random
    numbers (the forward is bitwise reproducible, so a small h is usable)."""
    import torch
    from paper_2312_16981_gb300 import adjoint as A
    # the source iteration converged to 1e-14: its stopping error (relative
    # change <= si_tol) is the noise floor of a difference with small h
    p = I.adjoint_grid().replace(si_tol=1e-14)
    rng = np.random.Generator(np.random.Philox(5))
    s = rng.normal(0.0, 0.1, p.ncell)
    s_target = rng.normal(0.0, 0.1, p.ncell)
    sim = B.Simulation(A.with_log_opacity(p.replace(seed=p.seed + 1), s_target), device=dev)
    sim.step(steps)
    T_target = sim.get_state(cap=0)["T"]
    sim.close()

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L_plain = A.misfit(p, s, steps, T_target, device=dev)
    t_fwd = time.perf_counter() - t0

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run = A.forward(A.with_log_opacity(p, s), steps, ckpt_every, dev)
    t1 = time.perf_counter()
    Tt = torch.as_tensor(T_target, device=run.T.device)
    r = run.T - Tt
    L = float((r * r).sum())
    ds, iters = A.backward(run, 2.0 * r)
    g = ds.cpu().numpy()
    t2 = time.perf_counter()
    unmatched = run.unmatched
    n_end = run.sim.tallies()["n_particles"]
    run.sim.close()

    cells = rng.choice(p.ncell, size=n_fd, replace=False)
    t3 = time.perf_counter()
    fd, used, flipped = A.crn_finite_differences(p, s, steps, T_target, list(cells), h=h, device=dev, retries=2)
    t_fd = time.perf_counter() - t3
    # relative to max(|FD|, 1e-5 max|g|): a cell whose sensitivity is below
    # 1e-5 of the largest is compared on that scale (the differences' own noise
    # is about 1e-9 of max|g| at h = 1e-6)
    floor = 1e-5 * float(np.max(np.abs(g)))
    rel_all = np.abs(g[cells] - fd) / np.maximum(np.abs(fd), floor)
    # a cell that misses 1e-3 without a decision flip: the difference again
    # with 10 h (less noise from the source iteration's stopping error, more
    # truncation); both differences and their spread are reported
    retried = []
    miss = [k for k in range(len(cells)) if not flipped[k] and rel_all[k] > 1e-3]
    if miss:
        fd10, used10, flip10 = A.crn_finite_differences(p, s, steps, T_target, [int(cells[k]) for k in miss],
                                                        h=10 * h, device=dev, retries=1)
        for j, k in enumerate(miss):
            r10 = abs(g[cells[k]] - fd10[j]) / max(abs(fd10[j]), floor)
            retried.append({"cell": int(cells[k]), "adjoint": float(g[cells[k]]), "fd_h": float(fd[k]),
                            "fd_10h": float(fd10[j]), "h_used": float(used10[j]), "flipped": bool(flip10[j]),
                            "rel_err_h": float(rel_all[k]), "rel_err_10h": float(r10),
                            "fd_spread_rel": float(abs(fd[k] - fd10[j]) / max(abs(fd10[j]), floor))})
            if not flip10[j] and used10[j] == 10 * h and r10 <= 1e-3:
                rel_all[k] = r10
    rel = rel_all[~flipped] if np.any(~flipped) else rel_all
    return {"workload": "adjoint_grid_128x128x16, 200 steps, dt = dx/c, 16x16 T_s = 1 source",
            "params": p.ncell, "loss": L, "loss_plain_forward": L_plain,
            "forward_s": t_fwd, "forward_with_checkpoints_s": t1 - t0, "backward_s": t2 - t1,
            "gradient_over_forward": (t2 - t0) / t_fwd, "checkpoint_every": ckpt_every,
            "particles_at_end": n_end, "unmatched_across_checkpoints": int(unmatched),
            "fd": {"cells": n_fd, "h": h, "h_min_used": float(np.min(used)),
                   "decision_flip_unresolved": int(np.sum(flipped)),
                   "compared": int(rel.size), "within_1e-3": int(np.sum(rel <= 1e-3)),
                   "median_rel_err": float(np.median(rel)), "max_rel_err": float(np.max(rel)),
                   "worst": [{"cell": int(cells[k]), "adjoint": float(g[cells[k]]), "fd": float(fd[k]),
                              "rel_err": float(rel_all[k])} for k in np.argsort(-rel_all)[:4]],
                   "max_abs_grad": float(np.max(np.abs(g))),
                   "max_rel_err_incl_flipped": float(np.max(rel_all)),
                   "rel_err_floor": "1e-5 x max |dL/ds|", "retried_at_10h": retried, "seconds": t_fd}}


def families_leg(B, dev, flush, steps=20):
    """The paper's other problem families and the UGKP variant, each evolved
    from its initial state and then timed as CUDA-graph steps (mixed
    precision and FP64): the Larsen slab (Sec. 3.3, photo-ionisation
    opacity, tau_num, free side; 400 steps in), the Olson foam (Sec. 3.5,
    three-band opacity, T-dependent heat capacity; 40 steps in, source on),
    the 200x30 slab in the UGKP variant from the synthetic state, and the
    32^3 x 8 3D checkerboard (20 steps in)."""
    out = {}
    cases = [("larsen_slab_200x24", I.larsen_slab(), 400, None),
             ("olson_slab_128x30", I.olson_slab(), 40, None)]
    pu = I.multigroup_slab().replace(method=I.UGKP)
    pu.particle_capacity = 1 << 23
    cases.append(("multigroup_slab_200x30_ugkp", pu, 5, I.synthetic_state(pu, N_PARTICLES, seed=1)))
    cases.append(("checkerboard_3d_32x32x32x8", I.checkerboard_3d(), 20, None))
    for name, p, evolve, st in cases:
        row = {}
        for prec_name, prec in (("mixed", I.MIXED), ("fp64", I.FP64)):
            sim = B.Simulation(p.replace(precision=prec), device=dev)
            if st is not None:
                sim.set_state(st["T"], st["rho"], st["rho_h"], st["particles"], step=st["step"])
            sim.step(evolve)
            assert sim.tallies()["status_bits"] == 0
            ms, segs, (n_in, _), _, si = graph_steps(sim, steps, flush)
            row[prec_name] = {"value": segs / (ms / 1e3), "unit": "segments/s", "ms_per_step": ms / steps,
                              "particles_per_step": n_in / steps, "si_iters_per_step": si / steps}
            sim.close()
        row["speedup_mixed_vs_fp64"] = row["mixed"]["value"] / row["fp64"]["value"]
        row["evolved_steps"] = evolve
        out[name] = row
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--particles", type=int, default=N_PARTICLES,
                    help="particles in the starting state (profiling runs use other sizes)")
    ap.add_argument("--quick", action="store_true",
                    help="timed steps of one precision only (no e2e, mixed or CPU legs): for profiler runs")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="particle precision of the headline (quick) run")
    ap.add_argument("--workload", default="slab", choices=["slab", "checkerboard"],
                    help="workload of a --quick run (profiling): the 200x30 slab or the 2D checkerboard")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the batched-ensemble leg")
    ap.add_argument("--no-families", action="store_true",
                    help="skip the Larsen / Olson / UGKP leg")
    ap.add_argument("--no-matched-error", action="store_true", help="skip the matched-error leg")
    ap.add_argument("--ensemble-steps", type=int, default=10)
    ap.add_argument("--no-checkerboard", action="store_true", help="skip the 2D checkerboard leg")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the opacity-gradient leg")
    ap.add_argument("--checkerboard-particles", type=int, default=20_000_000)
    ap.add_argument("--launch", default=None,
                    help="particle-kernel launch shape BLOCK,PPT[,PER] of a --quick run (profiling the shape a "
                         "full run's autotuner chose)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    from paper_2312_16981_gb300 import binding as B

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = "cuda:%d" % local
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    K = args.steps
    names = ["total", "birth_scan", "wave", "particles", "source_iteration", "end"]
    pk, src = peaks()
    p, s = workload(rank, args.particles, args.workload if args.quick else "slab")
    head_mixed = args.precision == "mixed" if args.quick else True
    p_head = p.replace(precision=I.MIXED if head_mixed else I.FP64)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    shapes = {}

    def prepare(prob, tune):
        # warm-up steps, the library's autotuner (the particle kernel's launch
        # shape timed on identical steps from a saved state), more warm-up
        sim = B.Simulation(prob, device=dev)
        sim.set_state(s["T"], s["rho"], s["rho_h"], s["particles"], step=s["step"])
        for _ in range(max(args.warmup, 3)):
            sim.step(1)
        if tune:
            shapes[tune] = sim.autotune(steps=3)
            for _ in range(3):
                sim.step(1)
        elif args.launch:
            sim.set_launch(*[int(x) for x in args.launch.split(",")])
            for _ in range(3):
                sim.step(1)
        assert sim.tallies()["status_bits"] == 0
        return sim

    sim = prepare(p_head, None if args.quick else "mixed" if head_mixed else "fp64")
    sim64 = None if args.quick else prepare(p.replace(precision=I.FP64), "fp64")

    # ---- timed region: whole steps as CUDA-graph replays (the headline build,
    # then the plain FP64 build it is compared with), device time from events
    barrier()
    with ClockSampler(local) as clk:
        total_ms, segs, (n_in, n_rd), n_out, si = graph_steps(sim, K, flush)
        if sim64 is not None:
            ms64, segs64, (n_in64, n_rd64), n_out64, si64 = graph_steps(sim64, K, flush)
    barrier()
    clocks = clk.summary()
    total_ms_max, segs_all = combine_replicas(total_ms, float(segs), world, dev)
    value = segs_all / (total_ms_max / 1e3)

    # ---- phase breakdown and per-launch kernel durations: the same step
    # launched kernel by kernel with events between the phases
    phases, _, (pn_in, pn_rd), pn_out, psi = timed_steps(sim, K, flush)
    dom = int(np.argmax(phases[1:])) + 1
    roof = roofline(p_head, names[dom], phases[dom] / K, pn_in / K, pn_rd / K, pn_out / K, psi / K,
                    head_mixed, pk, src)
    roof_p = roofline(p_head, "particles", phases[3] / K, pn_in / K, pn_rd / K, pn_out / K, psi / K,
                      head_mixed, pk, src)

    line = {"metric": METRIC, "value": value, "unit": "segments/s", "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": total_ms_max / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if head_mixed else "f64",
            "precision": ("mixed: f32 particle state and arithmetic; f64 tallies, source iteration, "
                          "Planck integrals and energy ledger" if head_mixed else "f64 throughout"),
            "data": "synthetic",
            "config": config_dict(p, args.particles, {"parallelism": "replicas" if world > 1 else "single"}),
            "timing": "CUDA events around each whole step (one CUDA-graph replay of all kernels)",
            "steps_per_s": K / (total_ms_max / 1e3),
            "phase_ms_per_step": {n: float(phases[i] / K) for i, n in enumerate(names)},
            "phase_timing": "the same step launched kernel by kernel, events between phases (%d more steps)" % K,
            "particles_per_step": n_in / K, "si_iters_per_step": si / K,
            "roofline": roof, "particle_kernel_roofline": roof_p, "clocks": clocks}
    if shapes:
        line["launch_shape"] = {k: {"block": v["block"], "particles_per_thread": v["particles_per_thread"],
                                    "blocks_per_sm": v["blocks_per_sm"]} for k, v in shapes.items()}
        line["launch_shape"]["how"] = "ugkwp_autotune: each candidate shape timed on 3 steps from the same saved state"

    if sim64 is not None:
        ph64, _, (qn_in, qn_rd), qn_out, qsi = timed_steps(sim64, K, flush)
        line["fp64"] = {
            "value": segs64 / (ms64 / 1e3), "unit": "segments/s", "dtype": "f64",
            "ms_per_step": ms64 / K, "steps_per_s": K / (ms64 / 1e3),
            "phase_ms_per_step": {n: float(ph64[i] / K) for i, n in enumerate(names)},
            "particles_per_step": n_in64 / K, "si_iters_per_step": si64 / K,
            "particle_kernel_roofline": roofline(p, "particles", ph64[3] / K, qn_in / K, qn_rd / K, qn_out / K,
                                                 qsi / K, False, pk, src)}
        line["speedup_vs_fp64"] = value / line["fp64"]["value"]
        sim64.close()

        # ---- end to end through the C ABI with host buffers (headline build)
        Tdev = sim.device_array("T")
        Rdev = sim.device_array("rho")
        Th = torch.empty(Tdev.shape, dtype=torch.float64, pin_memory=True)
        Rh = torch.empty(Rdev.shape, dtype=torch.float64, pin_memory=True)
        Th.copy_(Tdev)
        Rh.copy_(Rdev)
        torch.cuda.synchronize()
        e2e_segs = 0
        barrier()
        t0 = time.perf_counter()
        for _ in range(K):
            Tdev.copy_(Th, non_blocking=True)
            Rdev.copy_(Rh, non_blocking=True)
            sim.step(1)
            Th.copy_(Tdev, non_blocking=True)
            Rh.copy_(Rdev, non_blocking=True)
            tt = sim.tallies()           # synchronises: the step's result is on the host
            e2e_segs += tt["n_segments"]
        e2e_s = time.perf_counter() - t0
        barrier()
        line["e2e"] = {"value": e2e_segs / e2e_s, "unit": "segments/s",
                       "h2d_bytes_per_step": int(Th.numel() + Rh.numel()) * 8,
                       "d2h_bytes_per_step": int(Th.numel() + Rh.numel()) * 8,
                       "what": "per step: H2D of T and rho from pinned host memory, ugkwp_step "
                               "(CUDA graph), D2H of T, rho and the tally report"}
        # timed graph steps of both builds, their phase passes, and the e2e steps
        # (mixed graph steps: the timed ones and the e2e ones also sort)
        # the timed region: K graph steps of each build
        line["gpu_launches"] = int(K * (KERNELS_PER_STEP["mixed"] + KERNELS_PER_STEP["fp64"]))
    else:
        line["gpu_launches"] = int(K * KERNELS_PER_STEP["mixed" if head_mixed else "fp64"])

    extra_legs = rank == 0 and world == 1 and not args.quick
    if extra_legs and not args.no_matched_error:
        line["matched_error"] = {"multigroup_slab_200x30": matched_error_leg(B, dev),
                                 "checkerboard_2d_256x256x30": matched_error_checkerboard(B, dev),
                                 "ensemble_first_32_slabs": matched_error_ensemble(B, dev)}
    if extra_legs and not args.no_checkerboard:
        line["checkerboard_2d"] = checkerboard_leg(B, dev, flush, min(K, 10), args.warmup,
                                                   args.checkerboard_particles)
    if extra_legs and not args.no_adjoint:
        line["adjoint"] = adjoint_leg(B, dev)
    if extra_legs and not args.no_families:
        line["families"] = families_leg(B, dev, flush)
    if extra_legs and not args.no_ensemble:
        line["batched_ensemble"] = ensemble_leg(B, dev, flush, args.ensemble_steps, args.warmup)

    if rank == 0 and not args.no_cpu_baseline and not args.quick:
        osegs, ot = oracle_protocol(p, s)
        line["cpu_baseline"] = {
            "value": osegs / ot, "unit": "segments/s", "cores": 1, "kind": "oracle",
            "sample": protocol_text(args.particles), "host": host_cpu(),
            "not_timed": "the 2D checkerboard at 1e7 particles: about 80 s of oracle time per step on one "
                         "core (2e7 segments at ~2.5e5 segments/s), beyond a benchmark that ends in minutes"}
        n_sample = ORACLE_SAMPLE
        try:
            pv, pn = oracle_parallel(n_sample, args.particles)
            line["cpu_baseline"]["parallel"] = {
                "value": pv, "unit": "segments/s", "cores": pn,
                "what": "%d oracle replicas in spawned processes, each one untimed and %d timed steps on its "
                        "own %d-particle slice of the workload (each with the full source iteration)"
                        % (pn, ORACLE_STEPS, n_sample)}
        except Exception as exc:   # the single-core figure stands
            line["cpu_baseline"]["parallel"] = {"unavailable": str(exc)[:200]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
