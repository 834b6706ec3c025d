#!/usr/bin/env python3
"""Benchmark of the GLISSE test-particle map on GB300 (one JSON line on stdout).

Metric: FP64 particle-steps/s (and the fraction of the measured FP64 peak).
Workload (default): 131072 test particles between Uranus-like and Neptune-like
orbits under a 4-planet system (a in U[20, 29] AU, e in U[0, 0.1], Rayleigh
inclinations sigma = 2 deg, dt = 0.5 yr), chunk 1024 steps, live-particle
compaction after every chunk; seeded synthetic data (glisse_inputs).

One benchmark step = one pass of the whole path over one chunk: the planet
ephemeris for the next chunk (side stream), the particle map over 1024 steps,
and compaction.  W untimed steps, then K steps each bracketed by CUDA events on
the library's stream, with an L2 flush (256 MiB write) between steps outside
the events; barrier + synchronize around the timed region; max over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload longrun|belt|tiny]
  python bench.py --impl reference ...   # the plain FP64 CPU oracle on host cores
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FP64 particle-steps/s at 1 GB300 (4 planets, 1e5-1e6 particles); % FP64 peak"
UNIT = "particle-steps/s"

# FP64 work of one interior particle-step in the kernel's formulation (static count of
# the source; ncu's executed DADD:DMUL:DFMA mix matches it): the fast Kepler drift with
# the degree-3 Stumpff tier (3 DADD, 13 DMUL, 42 DFMA), the h0 term (3 DFMA), and per
# planet 3 DADD + 1 DMUL + 8 DFMA (separation, |d|^2, k |d|^-3 with the seed's square
# and k times its cube formed in integer arithmetic, velocity update).
def fp64_instr_per_step(np_: int) -> int:
    return 58 + 3 + 12 * np_


def flop_per_step(np_: int) -> int:
    # DFMA counts 2 FLOP, DADD / DMUL 1
    return (3 + 13 + 2 * 42) + 2 * 3 + np_ * (3 + 1 + 2 * 8)


# GB300 FP64 pipe: 2 DFMA per clock per SM (ncu: sm__sass_thread_inst_executed_op_dfma_pred_on
# peak_sustained = 2 inst/cycle/SM), 152 SMs.
DFMA_PER_CLK_PER_SM = 2


PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "particle_tasks_kernel_longrun.txt")
KERNEL_SOURCES = ["particle_map.cuh", "particles.cu", "kepler.cuh", "device_math.cuh", "glisse_internal.h"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2011_03484_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_traffic():
    """DRAM bytes per particle-kernel launch from the committed ncu summary, if it was
    taken on the current kernel source (its hash line must match), else None."""
    try:
        vals = {}
        for line in open(PROFILE_TRAFFIC):
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
        if vals.get("kernel_source_hash") != kernel_hash():
            return None
        return float(vals["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.proc = None
        self.path = None
        self.index = index

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self):
        if self.proc is None or not self.path:
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        try:
            sm = [float(r[1]) for r in rows]
            smax = max(float(r[2]) for r in rows)
        except ValueError:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": reasons, "samples": len(rows)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_particles(w, rank: int):
    """Particles of rank `rank` under weak scaling: rank 0 uses the workload itself, every
    other rank an independent seeded replica of the same shape (no data is exchanged)."""
    import numpy as np

    import glisse_inputs as gi

    if rank == 0:
        return gi.make(w.name)["particles"]
    rng = np.random.Generator(np.random.PCG64(w.seed + 1000 * rank))
    return gi.particle_belt(rng, w.n, w.a_range, w.e_range, w.sigma_i_deg, w.star_mass)


def reduce_over_ranks(total_ms: float, particle_steps: float, device=None):
    """(max over ranks of the timed milliseconds, sum over ranks of particle-steps).
    The only cross-rank traffic of the benchmark; with one process it is the identity."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return total_ms, particle_steps
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    n = torch.tensor([particle_steps], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item())


def workload_desc(w, n):
    return (f"{w.name}: {n} test particles, 4 planets (a 5.2-30.1 AU), a in U[{w.a_range[0]:g},{w.a_range[1]:g}] AU, "
            f"e in U[{w.e_range[0]:g},{w.e_range[1]:g}], sigma_i {w.sigma_i_deg:g} deg, dt {w.dt:g} yr, "
            f"chunk {w.chunk}, compaction every chunk")


def cpu_oracle_rate(w, planets, particles, steps_per_chunk, chunks, threads=0, warmup=0, kepler_iters=0):
    """Oracle particle-steps/s on host cores over `chunks` timed chunks of a particle
    sample, after `warmup` untimed chunks of the same run (kepler_iters > 0: the
    paper's fixed-iteration Kepler solve)."""
    import oracle

    oracle.build()
    rc = oracle.rcrit(w.star_mass, planets, 0, w.k_hill)
    run = oracle.ParticleRun(w.star_mass, planets[:, 0], particles, rc, w.r_max, kepler_iters=kepler_iters)
    pl = planets.copy()
    done, busy = 0, 0.0
    for c in range(warmup + chunks):
        pl2, log, _ = oracle.planet_wh(w.star_mass, pl, w.dt, steps_per_chunk)
        alive0 = int((run.removal_step < 0).sum())
        t0 = time.perf_counter()
        run.advance(log, w.dt, threads)
        el = time.perf_counter() - t0
        pl = pl2
        alive1 = int((run.removal_step < 0).sum())
        if c >= warmup:
            busy += el
            # removed particles counted with half a chunk (their steps stop mid-chunk)
            done += alive1 * steps_per_chunk + (alive0 - alive1) * steps_per_chunk // 2
    cores = threads if threads > 0 else oracle.max_threads()
    return done / busy, cores, busy


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    import glisse_inputs as gi

    w = gi.WORKLOADS[args.workload]
    full = gi.make(args.workload)
    ids = gi.subset_ids(args.workload, args.ref_particles)
    sample = full["particles"][ids]
    rate_t, cores, busy_t = cpu_oracle_rate(w, full["planets"], sample, w.chunk, args.steps, warmup=args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": rate_t, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * busy_t / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(w, w.n), "sample_particles": len(ids), "steps_per_bench_step": w.chunk},
        "cpu_baseline": {"value": rate_t, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{len(ids)} random ids of the {w.n}-particle workload, {w.chunk} steps per bench step"},
        "e2e": {"value": rate_t, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def time_batched(G, torch, dev, stream, b, C, steps, warmup, tune=False):
    """W untimed chunks, then `steps` graph-replayed chunks of the batch, each bracketed by CUDA
    events with an L2 flush outside them; exact particle-steps from the device counter."""
    args_b = (b["star_mass"], b["n_planets"], b["planets"], b["n_particles"], b["particles"], b["dt"])
    sim = G.BatchSimulation(*args_b, chunk_steps=C, cuda_stream=stream.cuda_stream)
    tuned = sim.tune(256) if tune else None
    C_run = tuned[0] if tuned else C
    for _ in range(warmup):
        sim.advance(C_run)
    torch.cuda.synchronize(dev)
    live0 = sim.status()[0]
    steps0 = sim.steps_done()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    with ClockSampler(dev.index or 0) as clocks:
        for k in range(steps):
            flush.zero_()
            starts[k].record(stream)
            sim.advance(C_run)
            ends[k].record(stream)
        torch.cuda.synchronize(dev)
    done = sim.steps_done() - steps0  # exact: each particle counts the steps it advanced
    total_ms = sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends))
    live1 = sim.status()[0]
    sim.close()
    del flush
    return {"value": done / (total_ms * 1e-3), "total_ms": total_ms, "clocks": clocks.summary(), "live0": live0,
            "live1": live1, "tuned": tuned, "C_run": C_run, "args_b": args_b}


def batched_arm(args):
    """256 independent systems (N_p 2..8, ~3.4e6 particles, dt = P_inner / 20) in one
    context: planet chunks of all systems, the persistent particle kernel, compaction
    and task rebuild replayed as a captured CUDA graph per chunk."""
    import numpy as np
    import torch

    import glisse_inputs as gi
    import paper_2011_03484_gb300 as G

    rank, world, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    G._build.build()
    G.load()
    b = gi.make_batched(seed=4 + 1000 * rank, n_systems=args.batched_systems)
    C = 1024
    stream = torch.cuda.current_stream(dev)
    rb = time_batched(G, torch, dev, stream, b, C, args.steps, args.warmup, tune=args.tune)
    value, total_ms, tuned, C_run, args_b = rb["value"], rb["total_ms"], rb["tuned"], rb["C_run"], rb["args_b"]
    live0, live1 = rb["live0"], rb["live1"]
    # per-stage device times from a timing-mode copy (direct launches with events)
    simt = G.BatchSimulation(*args_b, chunk_steps=C_run, timing=1, cuda_stream=stream.cuda_stream)
    if tuned:
        simt.set_launch(tuned[1], tuned[2])
    for _ in range(args.warmup):
        simt.advance(C_run)
    simt.timings(reset=True)
    for _ in range(min(args.steps, 3)):
        simt.advance(C_run)
    tm = simt.timings()
    simt.close()
    # end to end through the C ABI with host buffers in pinned memory: create (H2D of every
    # system's planets and particles) + one chunk + read (D2H of states, flags, steps, reasons)
    e2e = None
    if args.e2e_steps > 0:
        def pinned(a, dtype):
            t = torch.empty(np.shape(a), dtype=dtype).pin_memory().numpy()
            t[...] = a
            return t

        pl_h = pinned(b["planets"], torch.float64)
        pa_h = pinned(b["particles"], torch.float64)
        n_all = int(np.sum(b["n_particles"]))
        out_h = {"state": pinned(np.zeros((n_all, 6)), torch.float64),
                 "alive": pinned(np.zeros(n_all), torch.uint8),
                 "removal_step": pinned(np.zeros(n_all), torch.int64),
                 "removal_reason": pinned(np.zeros(n_all), torch.int32)}
        times, done_e = [], 0
        for k in range(args.e2e_steps + 1):
            t0 = time.perf_counter()
            se = G.BatchSimulation(b["star_mass"], b["n_planets"], pl_h, b["n_particles"], pa_h, b["dt"],
                                   chunk_steps=C_run, cuda_stream=stream.cuda_stream)
            if tuned:
                se.set_launch(tuned[1], tuned[2])
            se.advance(C_run)
            se.read(out_h)
            steps_k = se.steps_done()
            se.close()
            el = time.perf_counter() - t0
            if k > 0:
                times.append(el)
                done_e += steps_k
        e2e = {"value": done_e / sum(times), "unit": UNIT,
               "h2d_bytes_per_step": int(pl_h.nbytes + pa_h.nbytes),
               "d2h_bytes_per_step": int(sum(a.nbytes for a in out_h.values())),
               "host_buffers": "pinned"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = batched_cpu_baseline(b, C_run)

    csum = rb["clocks"]
    mhz = csum["sm_mhz"] if csum else 2070.0
    n_sm, dfma_peak = fp64_peak(torch, dev, mhz)
    w_np = float(np.sum(b["n_planets"] * b["n_particles"]) / np.sum(b["n_particles"]))
    kernel_ms = tm["particle_ms"] / max(tm["particle_launches"], 1)
    spl = tm["particle_steps"] / max(tm["particle_launches"], 1)
    flop = flop_per_step(0) + (flop_per_step(1) - flop_per_step(0)) * w_np
    instr = fp64_instr_per_step(0) + (fp64_instr_per_step(1) - fp64_instr_per_step(0)) * w_np
    achieved = flop * spl / (kernel_ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"batched: {len(b['star_mass'])} systems, N_p 2..8, {int(b['n_particles'].sum())} "
                               f"particles, dt = P_inner/20, chunk {C_run}, one graph per chunk",
                   "live_at_start": live0, "live_at_end": live1, "tuned": tuned,
                   "particle_weighted_planets": w_np},
        "roofline": {"bound": "alu", "achieved": achieved * 1e-9, "peak": 2 * dfma_peak * 1e-9, "unit": "GFLOP/s",
                     "frac": achieved / (2 * dfma_peak), "traffic": None, "kernel": "batch_particle_kernel",
                     "kernel_ms_avg": kernel_ms,
                     "fp64_pipe_frac": instr * spl / (kernel_ms * 1e-3) / dfma_peak,
                     "flop_per_particle_step": flop},
        "stage_ms_per_step": {"particle": tm["particle_ms"] / max(tm["particle_launches"], 1),
                              "ephemeris": tm["ephemeris_ms"] / max(tm["ephemeris_launches"], 1),
                              "compaction": tm["compact_ms"] / max(tm["compact_launches"], 1)},
        "gpu_launches": 7 * args.steps,
        "clocks": csum,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def batched_cpu_baseline(b, n_steps, n_sys=64, per_sys=2048, seed=0):
    """The oracle on the host cores over a bounded sample of the batched workload: n_sys
    random systems, up to per_sys random particles of each, n_steps steps of each system's
    own map (its planets integrated by the oracle too)."""
    import numpy as np

    import oracle

    oracle.build()
    rng = np.random.default_rng(seed)
    n_systems = len(b["star_mass"])
    pl_off = np.concatenate([[0], np.cumsum(b["n_planets"])])
    pa_off = np.concatenate([[0], np.cumsum(b["n_particles"])])
    done, busy, taken = 0, 0.0, 0
    for s in sorted(rng.choice(n_systems, size=min(n_sys, n_systems), replace=False)):
        pl = b["planets"][pl_off[s]:pl_off[s + 1]]
        pa = b["particles"][pa_off[s]:pa_off[s + 1]]
        if len(pa) > per_sys:
            pa = pa[np.sort(rng.choice(len(pa), size=per_sys, replace=False))]
        t0 = time.perf_counter()
        o = oracle.run(float(b["star_mass"][s]), pl, pa, float(b["dt"][s]), n_steps)
        busy += time.perf_counter() - t0
        rs = o["removal_step"]
        done += int(np.where(rs >= 0, rs, n_steps).sum())
        taken += len(pa)
    cores = oracle.max_threads()
    return {"value": done / busy, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{min(n_sys, n_systems)} random systems, {taken} particles (up to {per_sys} per system), "
                      f"{n_steps} steps each ({busy:.1f} s wall on {cores} threads)"}


def time_diff(G, torch, dev, stream, n_particles=0, n_steps=0, K=256):
    """Differentiation workload: 65536 particles (a 22-28 AU, e < 0.05, sigma_i 1 deg),
    10^4 steps (n_steps > 0: fewer), checkpoints every K steps.  Times the plain map, the
    differentiable forward pass (without and with one tangent vector), the adjoint pass, the
    growth gradient and tape mode, and returns each as particle-steps/s and as a cost ratio
    to the plain map."""
    import glisse_inputs as gi

    w = gi.WORKLOADS["diff"]
    full = gi.make("diff")
    pl, s0 = full["planets"], full["particles"]
    if n_particles > 0:
        s0 = s0[:n_particles]  # a prefix of the same seeded set (small cases for ncu)
    n, n_steps = s0.shape[0], (n_steps if n_steps > 0 else w.n_steps)

    def timed(fn):
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1), out

    # plain map over the same steps (chunk 1024, compaction every chunk)
    sim = G.Simulation(1.0, pl, s0, w.dt, cuda_stream=stream.cuda_stream, timing=1)
    sim.advance(w.chunk)  # warm-up
    sim.timings(reset=True)
    ms_map, _ = timed(lambda: sim.advance(n_steps))
    steps_map = sim.timings()["particle_steps"]
    sim.close()
    x0 = torch.as_tensor(s0, dtype=torch.float64, device=dev)
    warm = G.DiffMap(1.0, pl, n, w.dt, 64, K)
    warm.forward(x0)
    warm.backward(torch.ones_like(x0))
    warm.close()
    dm = G.DiffMap(1.0, pl, n, w.dt, n_steps, K)
    ms_fwd, out = timed(lambda: dm.forward(x0))
    live = int((out[3] < 0).sum().item())
    ms_bwd, _ = timed(lambda: dm.backward(torch.ones_like(x0)))
    tan = G._growth_seed(x0)
    ms_fwd_t, out_t = timed(lambda: dm.forward(x0, tan))
    # gradient of the growth indicator: one reverse sweep of the map extended by its
    # tangent (after the forward pass with the tangent), and forward mode over the
    # 6 state coordinates
    ones = torch.ones(n, dtype=torch.float64, device=dev)
    ms_grow_rev, _ = timed(lambda: dm.backward_growth(torch.ones_like(x0), ones, out_t[1][0]))
    ms_grow, _ = timed(lambda: dm.growth_gradient(x0, tan[0].contiguous()))
    dm.close()
    # the memory-aware default (GLISSE_DIFF_AUTO): tape mode -- the forward pass records every
    # step, the backward pass only sweeps back -- when the record fits in half of the free
    # device memory, else checkpoints every 256 steps
    da = G.DiffMap(1.0, pl, n, w.dt, n_steps, G.GLISSE_DIFF_AUTO)
    ms_fwd_auto, _ = timed(lambda: da.forward(x0))
    ms_bwd_auto, _ = timed(lambda: da.backward(torch.ones_like(x0)))
    auto_k = da.checkpoint_every
    da.close()
    tape = {"checkpoint_every": auto_k, "forward_ms": ms_fwd_auto, "adjoint_ms": ms_bwd_auto,
            "record_bytes": 8 * (14 + 2 * len(pl)) * n * n_steps if auto_k == 0 else None,
            "forward_plus_adjoint_ratio": (ms_fwd_auto + ms_bwd_auto) / ms_map}
    # the growth gradient with a tape that keeps tangent 0 (GLISSE_DIFF_TAPE_TANGENT): the forward
    # pass with the tangent records every step, the reverse sweep recomputes nothing; run when
    # the record fits in half of the free device memory
    tt_bytes = 8 * (23 + 2 * len(pl)) * n * n_steps
    growth_tape = None
    if tt_bytes <= 0.5 * torch.cuda.mem_get_info(dev)[0]:
        dt_ = G.DiffMap(1.0, pl, n, w.dt, n_steps, G.GLISSE_DIFF_TAPE_TANGENT)
        ms_fwd_tt, out_tt = timed(lambda: dt_.forward(x0, tan))
        ms_grow_tt, _ = timed(lambda: dt_.backward_growth(torch.ones_like(x0), ones, out_tt[1][0]))
        dt_.close()
        growth_tape = {"forward_with_tangent_ms": ms_fwd_tt, "reverse_sweep_ms": ms_grow_tt,
                       "record_bytes": tt_bytes, "ratio": (ms_fwd_tt + ms_grow_tt) / ms_map}
    ps = n * n_steps  # particle-steps of the differentiable run (removed particles stop early)
    line = {
        "metric": "FP64 particle-steps/s of the differentiable map (forward, adjoint) vs the plain map",
        "value": ps / ((ms_fwd + ms_bwd) * 1e-3), "unit": "particle-steps/s (forward + adjoint)",
        "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": ms_fwd + ms_bwd, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"diff: {n} particles, 4 planets, a 22-28 AU, e<0.05, {n_steps} steps, "
                               f"checkpoints every {K} steps", "live_at_end": live},
        "plain_map": {"ms": ms_map, "particle_steps_per_s": steps_map / (ms_map * 1e-3)},
        "diff_forward": {"ms": ms_fwd, "particle_steps_per_s": ps / (ms_fwd * 1e-3)},
        "diff_forward_with_tangent": {"ms": ms_fwd_t, "particle_steps_per_s": ps / (ms_fwd_t * 1e-3)},
        "adjoint": {"ms": ms_bwd, "particle_steps_per_s": ps / (ms_bwd * 1e-3)},
        "growth_gradient": {"reverse_sweep_ms": ms_grow_rev,
                            "forward_with_tangent_plus_reverse_ratio": (ms_fwd_t + ms_grow_rev) / ms_map,
                            "forward_mode_ms": ms_grow, "forward_mode_ratio": ms_grow / ms_map},
        "cost_ratio_to_plain_map": {"forward": ms_fwd / ms_map, "forward_with_tangent": ms_fwd_t / ms_map,
                                    "forward_plus_adjoint": (ms_fwd + ms_bwd) / ms_map},
        "auto_mode": tape,
        "growth_gradient_tangent_tape": growth_tape,
    }
    return line


def diff_arm(args):
    import torch

    import paper_2011_03484_gb300 as G

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    G._build.build()
    G.load()
    line = time_diff(G, torch, dev, torch.cuda.current_stream(dev), args.diff_particles, args.diff_steps)
    print(json.dumps(line), flush=True)
    return 0


def time_single(G, torch, dev, stream, w, planets, particles, steps, warmup, kmode=0, kepler_iters=5, sort=False,
                sample_every=0, one_call=False, dist=None):
    """W untimed chunks, then `steps` chunks of w.chunk steps, each bracketed by CUDA events on the
    library's stream with an L2 flush (256 MiB write) outside the events; clocks sampled during
    the timed region.  Returns the handle (caller destroys it) and the measurements."""
    np_ = planets.shape[0]
    o = G.glisse_opts_default()
    o.chunk_steps = w.chunk
    o.resync_chunks = w.resync
    o.enc_value = w.k_hill
    o.r_max = w.r_max
    o.timing = 1
    o.cuda_stream = stream.cuda_stream
    o.kepler_mode = kmode
    o.kepler_iters = kepler_iters
    o.sort_mode = G.GLISSE_SORT_COST if sort else G.GLISSE_SORT_NONE
    h = G.glisse_create(w.star_mass, planets, particles, w.dt, o)
    if sample_every > 0:
        G.glisse_set_sampling(h, sample_every, frame=G.GLISSE_FRAME_BARY, max_samples=0, res_planet=np_ - 1,
                              res_p=3, res_q=2, avoid_deg=10.0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(warmup):
        G.glisse_advance(h, w.chunk)
    torch.cuda.synchronize(dev)
    G.glisse_timings(h, reset=True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    live_before = G.glisse_status(h)[0]
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    chunk_live, chunk_steps = [], []  # host-side counters, read between chunks (no GPU work)
    with ClockSampler(dev.index or 0) as clocks:
        t_wall0 = time.perf_counter()
        if one_call:
            # the whole timed run as one glisse_advance call (the planets may run ahead of
            # the particles up to its last chunk)
            flush.zero_()
            chunk_live.append(G.glisse_status(h)[0])
            starts[0].record(stream)
            G.glisse_advance(h, w.chunk * steps)
            ends[0].record(stream)
            chunk_steps.append(G.glisse_timings(h)["particle_steps"])
            starts, ends = starts[:1], ends[:1]
        else:
            for k in range(steps):
                flush.zero_()
                chunk_live.append(G.glisse_status(h)[0])
                starts[k].record(stream)
                G.glisse_advance(h, w.chunk)
                ends[k].record(stream)
                chunk_steps.append(G.glisse_timings(h)["particle_steps"])
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter() - t_wall0
    if dist:
        dist.barrier()
    del flush
    step_ms = [s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)]
    tm = G.glisse_timings(h)
    return h, {"step_ms": step_ms, "total_ms": sum(step_ms), "chunk_live": chunk_live, "chunk_steps": chunk_steps,
               "tm": tm, "live_before": live_before, "live_after": G.glisse_status(h)[0],
               "clocks": clocks.summary(), "t_wall": t_wall}


def fp64_peak(torch, dev, mhz):
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    return n_sm, n_sm * DFMA_PER_CLK_PER_SM * mhz * 1e6


def belt_record(G, torch, dev, stream, steps=5, warmup=3):
    """A few chunks of the 1048576-particle resonant belt (a in 40-50 AU, e < 0.4), in the
    benchmark's launch configuration: particle-steps/s and the particle kernel's FP64 fraction."""
    import glisse_inputs as gi

    w = gi.WORKLOADS["belt"]
    full = gi.make("belt")
    h, r = time_single(G, torch, dev, stream, w, full["planets"], full["particles"], steps, warmup)
    G.glisse_destroy(h)
    tm = r["tm"]
    mhz = r["clocks"]["sm_mhz"] if r["clocks"] else 2070.0
    _, dfma_peak = fp64_peak(torch, dev, mhz)
    kernel_ms = tm["particle_ms"] / max(tm["particle_launches"], 1)
    spl = tm["particle_steps"] / max(tm["particle_launches"], 1)
    np_ = full["planets"].shape[0]
    return {"workload": workload_desc(w, w.n), "steps": steps, "warmup": warmup,
            "value": tm["particle_steps"] / (r["total_ms"] * 1e-3), "unit": UNIT,
            "ms_per_step": r["total_ms"] / steps, "live_at_start": r["live_before"], "live_at_end": r["live_after"],
            "frac": flop_per_step(np_) * spl / (kernel_ms * 1e-3) / (2.0 * dfma_peak),
            "fp64_pipe_frac": fp64_instr_per_step(np_) * spl / (kernel_ms * 1e-3) / dfma_peak,
            "kernel_ms_avg": kernel_ms, "clocks": r["clocks"]}


def batched_record(G, torch, dev, stream, plain_value, steps=3, warmup=3):
    """A few chunks of the 256-system batched workload (graph-replayed chunks, default launch
    shape): particle-steps/s and its per-particle-step cost against the plain map's."""
    import numpy as np

    import glisse_inputs as gi

    b = gi.make_batched()
    r = time_batched(G, torch, dev, stream, b, 1024, steps, warmup)
    mhz = r["clocks"]["sm_mhz"] if r["clocks"] else 2070.0
    _, dfma_peak = fp64_peak(torch, dev, mhz)
    w_np = float(np.sum(b["n_planets"] * b["n_particles"]) / np.sum(b["n_particles"]))
    flop = flop_per_step(0) + (flop_per_step(1) - flop_per_step(0)) * w_np
    return {"workload": f"batched: {len(b['star_mass'])} systems, N_p 2..8, {int(b['n_particles'].sum())} particles, "
                        f"dt = P_inner/20, chunk 1024, one graph per chunk",
            "steps": steps, "warmup": warmup, "value": r["value"], "unit": UNIT, "ms_per_step": r["total_ms"] / steps,
            "frac_of_chunk_time": flop * r["value"] / (2.0 * dfma_peak),
            "cost_ratio_to_plain_map": plain_value / r["value"], "clocks": r["clocks"]}


def diff_record(G, torch, dev, stream, n_steps=2048, K=256):
    """The differentiation workload (65536 particles) over a reduced number of steps: the plain
    map, the differentiable forward pass, the adjoint pass (checkpoints every K steps, and the
    memory-aware default, which on this GPU records every step), the growth gradient; each as
    a cost ratio to the plain map over the same steps."""
    r = time_diff(G, torch, dev, stream, 0, n_steps, K)
    m = r["plain_map"]["ms"]
    out = {"workload": r["config"]["workload"], "plain_map_ms": m,
           "ratio": {"forward": r["diff_forward"]["ms"] / m, "adjoint": r["adjoint"]["ms"] / m,
                     "forward_plus_adjoint": (r["diff_forward"]["ms"] + r["adjoint"]["ms"]) / m,
                     "forward_with_tangent": r["diff_forward_with_tangent"]["ms"] / m,
                     "growth_gradient_reverse_sweep_with_tangent_forward":
                         r["growth_gradient"]["forward_with_tangent_plus_reverse_ratio"],
                     "growth_gradient_forward_mode": r["growth_gradient"]["forward_mode_ratio"]}}
    t = r["auto_mode"]
    out["ratio"]["auto_forward"] = t["forward_ms"] / m
    out["ratio"]["auto_adjoint"] = t["adjoint_ms"] / m
    out["ratio"]["auto_forward_plus_adjoint"] = t["forward_plus_adjoint_ratio"]
    out["auto_checkpoint_every"] = t["checkpoint_every"]
    out["auto_record_bytes"] = t["record_bytes"]
    gt = r.get("growth_gradient_tangent_tape")
    out["ratio"]["growth_gradient_tangent_tape"] = gt["ratio"] if gt else None
    return out


ORACLE_OPCOUNT = os.path.join(ROOT, "profiles", "oracle_op_count_tiny.txt")


def oracle_op_count():
    """FLOP per particle-step of the map as the oracle computes it (its op-counting build on the
    1024-particle workload, written by oracle/opcount.py), or None."""
    try:
        for line in open(ORACLE_OPCOUNT):
            if line.startswith("flop_per_particle_step:"):
                return float(line.split(":", 1)[1])
    except (OSError, ValueError):
        pass
    return None


def oracle_timings():
    """The oracle on the host's cores, on one thread and on all: the 1024-particle workload in
    full (10^4 steps) and a 4096-particle random subset of the 1048576-particle belt over 10^4
    steps (particle-steps/s each)."""
    import numpy as np

    import glisse_inputs as gi
    import oracle

    oracle.build()
    out = {}
    for name, k in (("tiny", None), ("belt", 4096)):
        w = gi.WORKLOADS[name]
        full = gi.make(name)
        pa = full["particles"] if k is None else full["particles"][gi.subset_ids(name, k)]
        pl = full["planets"]
        rc = oracle.rcrit(w.star_mass, pl, 0, w.k_hill)
        _, log, _ = oracle.planet_wh(w.star_mass, pl, w.dt, 10_000)
        rec = {"particles": len(pa), "steps": 10_000}
        for label, threads in (("one_core", 1), ("all_cores", 0)):
            run = oracle.ParticleRun(w.star_mass, pl[:, 0], pa, rc, w.r_max)
            t0 = time.perf_counter()
            run.advance(log, w.dt, threads)
            el = time.perf_counter() - t0
            rs = run.removal_step
            rec[label] = int(np.where(rs >= 0, rs, 10_000).sum()) / el
        rec["cores"] = oracle.max_threads()
        out[name] = rec
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="longrun",
                    choices=["longrun", "belt", "tiny", "batched", "diff", "eccentric"])
    ap.add_argument("--sort", action="store_true",
                    help="order live particles by expected Kepler-solve cost at every compaction")
    ap.add_argument("--tune", action="store_true", help="batched: run the autotuner before timing")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--batched-systems", type=int, default=256, help="batched: number of systems (small cases for ncu)")
    ap.add_argument("--one-call", action="store_true",
                    help="single-system: time the whole run as one glisse_advance call of steps x chunk steps")
    ap.add_argument("--diff-particles", type=int, default=0, help="diff: first N particles only (0 = all)")
    ap.add_argument("--diff-steps", type=int, default=0, help="diff: steps (0 = the workload's)")
    ap.add_argument("--ref-particles", type=int, default=8192)
    ap.add_argument("--cpu-particles", type=int, default=32768)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-subrecords", action="store_true",
                    help="leave out the belt / batched / diff sub-records of the default line")
    ap.add_argument("--kepler", default="converge", choices=["converge", "paper"],
                    help="paper: the paper's fixed-iteration Kepler solve (GLISSE_KEPLER_PAPER_FIXED)")
    ap.add_argument("--kepler-iters", type=int, default=5)
    ap.add_argument("--sample-every", type=int, default=0,
                    help="take barycentric element samples with a 3:2 libration test against the outermost "
                         "planet every K steps (flags only, no element log)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "batched":
        return batched_arm(args)
    if args.workload == "diff":
        return diff_arm(args)

    import numpy as np
    import torch

    import glisse_inputs as gi
    import paper_2011_03484_gb300 as G

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    G._build.build()
    G.load()

    w = gi.WORKLOADS[args.workload]
    full = gi.make(args.workload)
    # weak scaling: every rank integrates its own seeded replica of the workload
    planets, particles = full["planets"], replica_particles(w, rank)
    n = particles.shape[0]
    np_ = planets.shape[0]

    stream = torch.cuda.current_stream(dev)
    paper = args.kepler == "paper"
    kmode = G.GLISSE_KEPLER_PAPER_FIXED if paper else G.GLISSE_KEPLER_CONVERGE
    h, r = time_single(G, torch, dev, stream, w, planets, particles, args.steps, args.warmup, kmode=kmode,
                       kepler_iters=args.kepler_iters, sort=args.sort, sample_every=args.sample_every,
                       one_call=args.one_call, dist=dist)
    G.glisse_destroy(h)
    step_ms, total_ms, tm = r["step_ms"], r["total_ms"], r["tm"]
    # particle-steps/s of each chunk against the fraction of particles live at its start
    chunk_steps = r["chunk_steps"]
    done = [b - a for a, b in zip([0] + chunk_steps[:-1], chunk_steps)]
    vs_alive = [[round(lv / n, 5), round(ps / (ms * 1e-3), 1)] for lv, ps, ms in zip(r["chunk_live"], done, step_ms)]
    psteps = tm["particle_steps"]
    total_ms_all, psteps_all = reduce_over_ranks(total_ms, float(psteps), dev)
    value = psteps_all / (total_ms_all * 1e-3)

    # roofline of the particle kernel: FP64 work / its own device time, against the FP64 pipe
    # peak from the unit counts (152 SMs x 2 DFMA/clk) at the clock sampled during the timed
    # region (max clock if no sample)
    csum = r["clocks"]
    mhz = csum["sm_mhz"] if csum else 2070.0
    n_sm, dfma_peak = fp64_peak(torch, dev, mhz)
    probe_rate, probe_mhz = G.glisse_fp64_peak(20000)
    kernel_ms = tm["particle_ms"] / max(tm["particle_launches"], 1)
    steps_per_launch = psteps / max(tm["particle_launches"], 1)
    achieved = flop_per_step(np_) * steps_per_launch / (kernel_ms * 1e-3)
    peak = 2.0 * dfma_peak
    pipe = fp64_instr_per_step(np_) * steps_per_launch / (kernel_ms * 1e-3) / dfma_peak
    traffic = profile_traffic()
    orc_flop = oracle_op_count()

    # end to end through the C ABI with host buffers in pinned memory: create (H2D of the
    # planets and particles) + one chunk + read (D2H of states, flags, steps, reasons)
    e2e = None
    if args.e2e_steps > 0:
        def pinned(shape, dtype):
            return torch.empty(shape, dtype=dtype).pin_memory().numpy()

        pl_h = pinned(planets.shape, torch.float64)
        pl_h[...] = planets
        pa_h = pinned(particles.shape, torch.float64)
        pa_h[...] = particles
        out_h = {"state": pinned((n, 6), torch.float64), "alive": pinned((n,), torch.uint8),
                 "removal_step": pinned((n,), torch.int64), "removal_reason": pinned((n,), torch.int32)}
        times, done_e = [], 0
        phases = np.zeros(4)  # create (with the H2D copy), advance, read (with the D2H copy), destroy
        for k in range(args.e2e_steps + 1):
            t0 = time.perf_counter()
            sim = G.Simulation(w.star_mass, pl_h, pa_h, w.dt, chunk_steps=w.chunk, enc_value=w.k_hill,
                               r_max=w.r_max, kepler_mode=kmode, kepler_iters=args.kepler_iters,
                               sort_mode=G.GLISSE_SORT_COST if args.sort else G.GLISSE_SORT_NONE)
            t1 = time.perf_counter()
            sim.advance(w.chunk)
            t2 = time.perf_counter()
            out = sim.read(out_h)
            t3 = time.perf_counter()
            sim.close()
            t4 = time.perf_counter()
            if k > 0:
                times.append(t4 - t0)
                phases += np.array([t1 - t0, t2 - t1, t3 - t2, t4 - t3])
                # steps each particle advanced: up to its removal step, else the whole chunk
                rs = out["removal_step"]
                done_e += int(np.where(rs >= 0, rs, w.chunk).sum())
        e2e = {"value": done_e / sum(times), "unit": UNIT,
               "ms_per_step": {name: 1e3 * v / max(len(times), 1)
                               for name, v in zip(("create_h2d", "advance", "read_d2h", "destroy"), phases)},
               "h2d_bytes_per_step": int(particles.nbytes + planets.nbytes),
               "d2h_bytes_per_step": int(out["state"].nbytes + out["removal_step"].nbytes +
                                         out["removal_reason"].nbytes + n),
               "host_buffers": "pinned",
               "note": "each e2e step: create from pinned host buffers, the first 1024-step chunk (all "
                       "particles live), read into pinned host buffers, destroy"}

    subrecords = {}
    if rank == 0 and world == 1 and not args.no_subrecords and args.workload == "longrun" and not paper:
        subrecords["belt"] = belt_record(G, torch, dev, stream)
        subrecords["batched"] = batched_record(G, torch, dev, stream, value)
        subrecords["diff"] = diff_record(G, torch, dev, stream)

    cpu = None
    orc_t = None
    if rank == 0 and not args.no_cpu_baseline:
        ids = gi.subset_ids(args.workload, args.cpu_particles)
        rate, cores, busy = cpu_oracle_rate(w, planets, particles[ids], w.chunk, 2,
                                            kepler_iters=args.kepler_iters if paper else 0)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{len(ids)} random ids of the workload, 2 chunks of {w.chunk} steps "
                         f"({busy:.1f} s wall on {cores} threads)"}
        if not paper:
            orc_t = oracle_timings()

    launches = tm["particle_launches"] + tm["ephemeris_launches"] + 3 * tm["compact_launches"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_all / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(w, n), "particles_per_gpu": n, "planets": np_,
                   "steps_per_bench_step": w.chunk, "live_at_start": r["live_before"], "live_at_end": r["live_after"],
                   "fraction_alive_at_end": r["live_after"] / n, "l2": "flushed (256 MiB write) between timed steps",
                   "parallelism": f"replicas x{world} (independent particle sets, no collective)",
                   "wall_s": r["t_wall"]},
        "kepler": (f"paper fixed-iteration solve, {args.kepler_iters} Newton iterations (library sin/cos)"
                   if paper else "converged (FP32 pre-solve + FP64 Halley step)"),
        "sampling": (f"barycentric elements + 3:2 libration test every {args.sample_every} steps"
                     if args.sample_every > 0 else None),
        "sort": "by expected Kepler-solve cost, costliest first" if args.sort else None,
        "roofline": None if paper else {
            "bound": "alu", "achieved": achieved * 1e-9, "peak": peak * 1e-9, "unit": "GFLOP/s",
            "frac": achieved / peak, "traffic": traffic,
            "kernel": "particle_tasks_kernel<4> (the task launch AUTO picks for this workload)",
            "kernel_ms_avg": kernel_ms, "flop_per_particle_step": flop_per_step(np_),
            "flop_count": "the kernel's own FP64 work per particle-step (static count, equal to ncu's "
                          "executed DADD/DMUL/DFMA mix); the oracle's count is given beside it",
            "flop_per_particle_step_oracle": orc_flop,
            "frac_at_oracle_count": (orc_flop * steps_per_launch / (kernel_ms * 1e-3) / peak) if orc_flop else None,
            "fp64_instr_per_particle_step": fp64_instr_per_step(np_), "fp64_pipe_frac": pipe,
            "peak_source": f"unit counts: {n_sm} SMs x {DFMA_PER_CLK_PER_SM} DFMA/clk x 2 FLOP x "
                           f"{mhz:.0f} MHz (SM clock sampled during the timed region)",
            "probe_dfma_per_s": probe_rate,
            "probe_frac_of_peak": probe_rate / dfma_peak},
        "stage_ms_per_step": {"particle": tm["particle_ms"] / args.steps, "ephemeris": tm["ephemeris_ms"] / args.steps,
                              "compaction": tm["compact_ms"] / args.steps},
        "throughput_vs_alive": {"columns": ["fraction live at chunk start", "particle-steps/s of the chunk"],
                                "chunks": vs_alive},
        "e2e": e2e,
        "cpu_baseline": cpu,
        "oracle_timings": orc_t,
        "gpu_launches": int(launches),
        "clocks": csum,
    }
    line.update(subrecords)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
