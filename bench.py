"""Benchmark: subcycled Z4c zone-updates/s on one GB300.

Workload (one "step" = one subcycled coarse step, Sec. II steps 1-7 on every
level): Z4c head-on Brill-Lindquist data (m = 0.5 at z = +-1, lapse psi^-2),
7 nested levels, level 0 64^3 over [-32,32]^3 (h = 1), finest h = 1/64,
radiative outer boundary, KO sigma 0.3, eta 2.  Zone updates are counted as if
every cell took the finest time step (Sec. IV.C): 1.594e8 per coarse step.

Arms:
  default            the CUDA library (state resident in HBM, ~5 GB > L2)
  --impl reference   the CPU oracle on the machine's host cores, each step one
                     coarse step of a bounded sample of the same workload
                     (5 nested levels of 20^3, same physics and parameters).

The default JSON line also carries: the roofline of the dominant kernel and
of the others against FP64 peaks read and measured on the device; e2e through
the C ABI with host buffers and the transfer split; the uniform-step mode and
the plain per-box form of the same hierarchy; the scalar-wave workloads in the
plain, graph and persistent forms; the 256-request serving ensemble in four
arms; the CPU oracle on one core and on every core.  --study runs one study
instead (moving boxes, the wave stage kernel, the FP64 issue rates, the small
Z4c case of the ncu captures).

Multi-GPU (torchrun): independent replicas, one per GPU ("weak" scaling);
the path has no exchange step on one hierarchy per GPU.
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "subcycled Z4c zone-updates/s on 1 GB300, % roofline; ensemble p50/p99 latency"
UNIT = "zone-updates/s (finest-equivalent)"
# The FP64 roofline denominators are read from the device at run time
# (sc_measure_fp64_peak): the nominal rate (SMs x maximum SM clock x 2 DFMA
# per SM per clock x 2 flops) and the measured issue rates of a general DFMA
# and of a DADD (a DFMA with a unit multiplier issues at the DADD rate).


def _measured_hbm_gbs() -> float:
    """HBM copy bandwidth measured on this machine (MEASURED_PEAKS.json), else
    the profiling recipe's fallback figure (6.8 TB/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except Exception:
        return 6800.0


HBM_GBS = _measured_hbm_gbs()
# Algorithmic FP64 flops per interior cell of each Z4c pass: adds,
# multiplies and fused multiply-adds (2 flops) of the formulation as first
# written, counted by ncu (z4c_derivs = row-segment D_x/D_y pass 133 +
# per-cell pass 1047).  Later rewrites evaluate the same right-hand side with
# fewer FP64 instructions (FP64_INSTR_PER_CELL); the flop counts stay fixed so
# that achieved rates measure the method's work, and the issue fractions
# measure the current instruction stream.
FLOPS_PER_CELL = {"z4c_derivs": 1180.0, "z4c_stage": 1971.0}
# DRAM bytes (read + write) per interior cell of each kernel from a
# cold-cache ncu capture of a 262,144-cell launch (ncu flushes the caches
# before the launch; profiles/z4c_kernels_bl3level64_ncu.md), scaled to a
# launch by its cell count; None once the kernel has changed since the
# counters were taken.
DRAM_BYTES_PER_CELL = {"z4c_derivs": (32.003584e6 + 5.960192e6 + 150.886144e6 + 247.183104e6) / 262144,
                       "z4c_stage": (525.380608e6 + 289.159168e6) / 262144}
# FP64 instructions (DFMA + DMUL + DADD, thread-level / cell) per interior
# cell of each pass, counted by ncu on the 3-level 64^3 case
# (profiles/z4c_kernels_bl3level64_ncu.md, profiles/z4c_fp64_op_classes_bl3level64_ncu.md).
FP64_INSTR_PER_CELL = {4: {"z4c_derivs": 72.1875 + 693.0, "z4c_stage": 1072.0},
                       8: {"z4c_derivs": 209.0 + 1210.0, "z4c_stage": 1072.0}}
# The same passes split by issue rate (general FMAs, DADD-rate operations:
# additions, multiplications, unit-multiplier FMAs), counted by ncu on their
# op-class build (sc_run_op_class_pass, which issues every such operation as
# a DADD or DMUL; profiles/z4c_fp64_op_classes_bl3level64_ncu.md).
FP64_OP_CLASSES = {4: {"z4c_derivs": (48.125 + 451.0, 24.0625 + 242.0), "z4c_stage": (830.559, 13.0 + 235.445)},
                   8: {"z4c_derivs": (156.75 + 429.0, 52.25 + 781.0), "z4c_stage": (830.559, 13.0 + 235.445)}}
# Kernel with the largest share of a coarse step in the ncu launch list
# (profiles/z4c_bl_7level_launch_list.md).
DOMINANT = "z4c_stage"


def sample_hierarchy(nlev: int = 5, n: int = 20):
    """Bounded CPU sample of the benchmark workload: nlev nested cubes of n^3
    cells (each level the central n cells of its index space), same Z4c
    physics, Brill-Lindquist data and parameters."""
    from paper_2503_09629_gb300 import workloads as W
    boxes = [[W.cube(0, n)]]
    for l in range(1, nlev):
        lo = boxes[-1][0][0][0] * 2 + n // 2
        boxes.append([W.cube(lo, n)])
    L = 2.0
    return W.Hierarchy(system=W.Z4C, boxes=boxes, ncells0=(n, n, n), origin=(-L, -L, -L), h0=2 * L / n,
                       bc=W.BC_RADIATIVE, id_kind=W.ID_BRILL_LINDQUIST,
                       id_params=[0.5, 0.0, 0.0, 1.0, 0.5, 0.0, 0.0, -1.0],
                       name=f"z4c BL {nlev}-level {n}^3 sample")


def oracle_step_rate(h, steps: int, warmup: int):
    """Time the oracle (single thread) over `steps` coarse steps of h."""
    import oracle
    from paper_2503_09629_gb300 import workloads as W
    o = oracle.Oracle(h.system, h.boxes, h.ncells0, h.origin, h.h0, **h.kwargs())
    for l in range(h.nlevels):
        a = W.initial_fields(h, l, 0, ghosted=True)
        for f in range(a.shape[0]):
            o.set_field(l, 0, f, a[f], ghosted=True)
    if warmup:
        o.advance(warmup)
    t0 = time.perf_counter()
    o.advance(steps)
    dt = time.perf_counter() - t0
    fin, _ = h.zone_updates_per_coarse_step()
    return fin * steps / dt, dt


def _oracle_worker(job):
    """One oracle process of the aggregate CPU baseline: (kind, coarse steps)
    -> finest-equivalent zone-updates/s of that process."""
    kind, steps = job
    from paper_2503_09629_gb300 import workloads as W
    if kind == "z4c":
        return oracle_step_rate(sample_hierarchy(), steps, 0)[0]
    import oracle
    h = W.standing_wave_2level(32)
    o = oracle.Oracle(h.system, h.boxes, h.ncells0, h.origin, h.h0, **h.kwargs())
    for l in range(h.nlevels):
        a = W.initial_fields(h, l, 0)
        for f in range(2):
            o.set_field(l, 0, f, a[f])
    t0 = time.perf_counter()
    o.advance(steps)
    fin, _ = h.zone_updates_per_coarse_step()
    return fin * steps / (time.perf_counter() - t0)


def cpu_aggregate(cores: int):
    """The oracle on every host core at once (one process per core, started
    with spawn): aggregate zone-updates/s = the sum of the concurrent
    processes' rates, for the Z4c sample and for the 2-level standing wave."""
    import multiprocessing as mp
    out = {}
    with mp.get_context("spawn").Pool(cores) as pool:
        for kind, steps, label in (("z4c", 1, "z4c BL 5-level 20^3 sample, 1 coarse step per process"),
                                   ("wave", 32, "standing wave 2-level 32^3, 32 coarse steps per process")):
            t0 = time.perf_counter()
            rates = pool.map(_oracle_worker, [(kind, steps)] * cores)
            out[kind] = {"value": sum(rates), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": label,
                         "per_process_mean": sum(rates) / cores, "wall_s": time.perf_counter() - t0}
    return out


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        exe = shutil.which("nvidia-smi")
        if not exe:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.proc = subprocess.Popen([exe, f"--id={self.device}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                      "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL,
                                     stderr=subprocess.DEVNULL)
        time.sleep(0.3)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(dist, x: float, device: str) -> float:
    """Max of a per-rank float over all ranks (identity without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_step_per_rank: float, steps: int, t_max_ms: float) -> float:
    """Units processed by all ranks / the slowest rank's time (weak scaling:
    every replica does the same work)."""
    return world * units_per_step_per_rank * steps / (t_max_ms * 1e-3)


def run_ensemble(sc, W, n: int, seed: int, burst: bool, mean_interarrival: float, arm: str,
                 budget: int = 48 << 30, max_active: int = 8):
    """Serve the seeded request ensemble in one arm; returns latency and throughput.

    arms: "plain_per_box" -- one request at a time in arrival order, kernels
    launched box by box without graphs; "plain_graph" -- one request at a
    time, one CUDA graph per coarse step; "served_streams" -- continuous
    batching, max_active slots with one stream and one graph per request;
    "served_merged" -- continuous batching with the scalar-wave requests of a
    tick merged into one persistent cooperative launch (Z4c requests keep
    their graphs on their own streams)."""
    reqs = sorted(W.serving_requests(n, seed, burst=burst, mean_interarrival=mean_interarrival), key=lambda r: r[0])
    served = arm.startswith("served")
    srv = sc.Server(budget, max_active if served else 1, 2)
    srv.sc_server_set_merge(arm == "served_merged")
    mode = sc.SC_EXEC_PER_BOX if arm == "plain_per_box" else sc.SC_EXEC_GRAPH
    lat = []
    nxt = 0
    t0 = time.perf_counter()
    unfinished = []
    while nxt < len(reqs) or unfinished:
        now = time.perf_counter() - t0
        if now > 600.0:
            raise RuntimeError("serving ensemble did not finish within 600 s")
        while nxt < len(reqs) and reqs[nxt][0] <= now:
            _t, h, steps = reqs[nxt]
            unfinished.append(srv.sc_server_submit(h, steps, exec_mode=mode))
            nxt += 1
        srv.sc_server_tick()
        still = []
        for t in unfinished:
            done, l = srv.sc_server_poll(t)
            if done:
                lat.append(l)
                srv.sc_server_release(t)
            else:
                still.append(t)
        unfinished = still
    wall = time.perf_counter() - t0
    st = srv.sc_server_stats()
    srv.close()
    lat.sort()
    pct = lambda q: lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]
    return {"requests": n, "arrivals": "burst" if burst else f"poisson mean {mean_interarrival * 1e3:.1f} ms",
            "arm": arm, "max_active": max_active if served else 1,
            "p50_s": pct(0.5), "p99_s": pct(0.99), "wall_s": wall,
            "zone_updates_per_s": st["zu_finest"] / wall, "actual_zone_updates_per_s": st["zu_actual"] / wall,
            "gpu_launches": st["launches"]}


def run_serving_arms(sc, W, n: int, max_active: int = 8):
    """The seeded ensemble (60% wave, 40% Z4c requests) in every arm, burst
    arrivals and Poisson arrivals at 0.9 of the plain per-box service rate."""
    import torch
    torch.cuda.empty_cache()
    burst = {arm: run_ensemble(sc, W, n, 0, True, 0.0, arm, max_active=max_active)
             for arm in ("plain_per_box", "plain_graph", "served_streams", "served_merged")}
    ia = burst["plain_per_box"]["wall_s"] / n / 0.9
    poisson = {arm: run_ensemble(sc, W, n, 0, False, ia, arm, max_active=max_active)
               for arm in ("plain_per_box", "plain_graph", "served_streams")}
    return {"requests": n, "burst": burst, "poisson_load_0.9_of_plain_per_box": poisson}


def time_form(sc, h, mode, steps, warm=2):
    """Zone-updates/s of one hierarchy in one execution form, CUDA events on
    the context's stream over `steps` coarse steps after `warm` untimed ones."""
    import torch
    ctx = sc.Context(h, exec_mode=mode)
    ctx.sc_set_initial_data(h.id_kind, h.id_params)
    ctx.sc_advance(warm)
    ctx.sc_synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.sc_advance(steps)
    e1.record(stream)
    ctx.sc_synchronize()
    ms = e0.elapsed_time(e1) / steps
    launches = ctx.sc_launches_per_step()
    ctx.close()
    fin, _act = h.zone_updates_per_coarse_step()
    return {"ms_per_coarse_step": ms, "zone_updates_per_s": fin / (ms * 1e-3), "launches_per_coarse_step": launches}


def run_wave_forms(sc, W, scale: float = 1.0):
    """The scalar-wave workloads in the three execution forms: plain per-box
    launches, one CUDA graph per coarse step (one launch per level and phase
    over all boxes), and the persistent cooperative kernel (one launch per
    coarse step, grid barriers between phases)."""
    cases = [("standing wave 2-level 32^3 (state 10 MB, L2-resident)", W.standing_wave_2level(32), 200),
             ("gaussian 3-level 64^3, seeded uneven boxes", W.gaussian_3level(64, 0), 100),
             ("gaussian 3-level 128^3, seeded uneven boxes", W.gaussian_3level(128, 0), 40)]
    out = {}
    for name, h, steps in cases:
        steps = max(4, int(steps * scale))
        r = {"plain_per_box": time_form(sc, h, sc.SC_EXEC_PER_BOX, steps),
             "graph": time_form(sc, h, sc.SC_EXEC_GRAPH, steps),
             "persistent": time_form(sc, h, sc.SC_EXEC_PERSISTENT, steps)}
        base = r["plain_per_box"]["zone_updates_per_s"]
        for k in ("graph", "persistent"):
            r[k]["speedup_vs_plain"] = r[k]["zone_updates_per_s"] / base
        r["steps"] = steps
        out[name] = r
    return out


def run_serving(args):
    import torch

    import paper_2503_09629_gb300 as sc
    from paper_2503_09629_gb300 import workloads as W
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    sc.build()
    return run_serving_arms(sc, W, args.requests, args.max_active)


def study_moving(sc, W, steps: int):
    """Moving-box run of the 9-level binary-black-hole layout: each coarse
    step interpolates the shift at the punctures, moves them along dx/dt =
    -beta (forward Euler over the coarse step), regrids levels 3-8 around
    them and advances one coarse step."""
    import torch
    h, pos, radii, fm = W.moving_9level(32)
    ctx = sc.Context(h)
    ctx.sc_autotune()
    ctx.sc_set_initial_data(h.id_kind, h.id_params)
    dt0 = h.cfl * h.h0
    t_regrid = t_step = fin = 0.0
    track, cells = [pos], []
    for _ in range(steps):
        t0 = time.perf_counter()
        pos = W.track_punctures(ctx, pos, dt0)
        ctx.sc_regrid(W.moving_layout(ctx.h, pos, radii, fm))
        t1 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.sc_advance(1)
        e1.record()
        torch.cuda.synchronize()
        t_regrid += t1 - t0
        t_step += e0.elapsed_time(e1) * 1e-3
        fin += ctx.h.zone_updates_per_coarse_step()[0]
        track.append(pos)
        cells.append(sum(ctx.h.interior_cells(l) for l in range(ctx.h.nlevels)))
    out = {"workload": h.name, "coarse_steps": steps, "zone_updates_per_s_incl_regrid": fin / (t_step + t_regrid),
           "zone_updates_per_s_step_only": fin / t_step, "regrid_share": t_regrid / (t_step + t_regrid),
           "mean_step_ms": t_step / steps * 1e3, "mean_regrid_ms": t_regrid / steps * 1e3,
           "interior_cells_first_last": [cells[0], cells[-1]],
           "puncture_x_first_last": [track[0][1][0], track[-1][1][0]], "state_finite": bool(ctx.sc_check_finite()),
           "final_boxes_per_level": [len(b) for b in ctx.h.boxes]}
    ctx.close()
    return out


def study_wavekernel(sc, W, n: int = 256):
    """The scalar-wave stage kernel alone on one periodic n^3 level: CUDA-event
    time per launch against the FP64-issue and HBM bounds (15 FP64
    instructions and 64 algorithmic bytes per cell: u, Pi and y_n read, k and
    the next stage input written)."""
    h = W.Hierarchy(system=W.WAVE, boxes=[[W.cube(0, n)]], ncells0=(n, n, n), origin=(0.0, 0.0, 0.0), h0=1.0 / n,
                    id_kind=W.ID_STANDING_WAVE, id_params=[1.0, 1.0, 1.0, 1.0], name=f"wave 1-level {n}^3")
    ctx = sc.Context(h)
    ctx.sc_autotune()
    ctx.sc_set_initial_data(h.id_kind, h.id_params)
    ms, _ = ctx.sc_time_stage_kernels(0, 20)
    ctx.close()
    pk = sc.sc_measure_fp64_peak()
    cells, ipc, bpc = n ** 3, 15, 64
    issue = cells * ipc / (ms * 1e-3) / 1e9
    return {"workload": h.name, "ms_per_launch": ms, "cells": cells, "fp64_issue_g_per_s": issue,
            "frac_of_measured_dfma_issue": issue / pk["dfma_g_per_s"],
            "frac_of_measured_dadd_issue": issue / pk["dadd_g_per_s"],
            "algorithmic_gb_per_s": cells * bpc / (ms * 1e-3) / 1e9,
            "hbm_frac": cells * bpc / (ms * 1e-3) / 1e9 / HBM_GBS, "peaks": pk}


def study_z4c3level(sc, W, steps: int, n: int = 64, fd_order: int = 4):
    """Brill-Lindquist head-on on 3 nested levels of n^3 (n = 64: about 1.3 GB
    of device state, more than L2): the small case the ncu captures of the
    Z4c and refinement-boundary kernels run on.  One untimed coarse step,
    then `steps` timed ones, then the op-class pass of level 0 (the
    derivative pass and stage kernel with additions and multiplications as
    DADD/DMUL, for instruction counters that split the FP64 stream by issue
    rate; kernel names carry PlainK)."""
    import torch
    h = W.bl_3level(n)
    h.fd_order = fd_order
    ctx = sc.Context(h)
    ctx.sc_set_initial_data(h.id_kind, h.id_params)
    ctx.sc_advance(1)
    ctx.sc_synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ctx.sc_advance(steps)
    e1.record()
    ctx.sc_synchronize()
    out = {"workload": h.name, "coarse_steps": steps, "ms_per_coarse_step": e0.elapsed_time(e1) / max(steps, 1),
           "launches_per_coarse_step": ctx.sc_launches_per_step()}
    ctx.sc_run_op_class_pass(0)
    out["op_class_pass"] = {"level": 0, "interior_cells": h.interior_cells(0)}
    ctx.close()
    return out


def run_study(args):
    import torch

    import paper_2503_09629_gb300 as sc
    from paper_2503_09629_gb300 import workloads as W
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    sc.build()
    if args.study == "moving":
        return study_moving(sc, W, args.study_steps)
    if args.study == "wavekernel":
        return study_wavekernel(sc, W)
    if args.study == "z4c3level":
        return study_z4c3level(sc, W, args.study_steps, fd_order=args.fd_order)
    return sc.sc_measure_fp64_peak()


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    h = sample_hierarchy()
    value, dt = oracle_step_rate(h, args.steps, args.warmup)
    ms = dt / args.steps * 1e3
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": h.name, "note": "CPU oracle, single thread; bounded sample of the 7-level workload"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} coarse steps of {h.name}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args, rank: int, world: int):
    import numpy as np
    import torch

    import paper_2503_09629_gb300 as sc
    from paper_2503_09629_gb300 import workloads as W

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))
    sc.build()
    h = W.bl_7level()
    h.fd_order = args.fd_order
    fin_per_step, act_per_step = h.zone_updates_per_coarse_step()
    ctx = sc.Context(h)
    tile, _tune_ms = ctx.sc_autotune()
    tuning = ctx.sc_get_tuning()
    ctx.sc_set_initial_data(h.id_kind, h.id_params)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        ctx.sc_advance(1)
    ctx.sc_synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()

    clocks = ClockSampler(dev)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.sc_advance(1)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    t_max = max_over_ranks(dist, ms, "cuda")
    ms_per_step = t_max / args.steps
    value = whole_job_rate(world, fin_per_step, args.steps, t_max)
    launches = ctx.sc_launches_per_step() * args.steps
    state_finite = ctx.sc_check_finite()

    # Roofline of the dominant kernels: FP64-ALU bound.  Per-launch durations
    # from CUDA events on the library's stream, on the finest level; peaks
    # read from this device (nominal from its SM count and clock, and the
    # measured DFMA and DADD issue rates).
    pk = sc.sc_measure_fp64_peak(stream.cuda_stream)
    nominal_tflops = pk["sms"] * pk["sm_clock_mhz"] * 4 / 1e6
    dfma_tflops = 2 * pk["dfma_g_per_s"] / 1e3
    fin_level = h.nlevels - 1
    cells = h.interior_cells(fin_level)
    t_der, t_stage = ctx.sc_time_stage_kernels(fin_level, 5)
    roof = {}
    for name, t in (("z4c_derivs", t_der), ("z4c_stage", t_stage)):
        fpc = FLOPS_PER_CELL[name] if (h.fd_order == 4 or name == "z4c_stage") else None
        ipc = FP64_INSTR_PER_CELL[h.fd_order][name]
        issue = cells * ipc / (t * 1e-3) / 1e9
        gen, slow = FP64_OP_CLASSES[h.fd_order][name]
        # shortest time of this instruction mix at the measured issue rates
        t_mix = cells * (gen / pk["dfma_g_per_s"] + slow / pk["dadd_g_per_s"]) / 1e9 * 1e3
        r = {"ms_per_launch": t, "cells_per_launch": cells, "flops_per_cell": fpc,
             "fp64_issue": {"achieved_g_instr_per_s": issue, "instr_per_cell": ipc,
                            "general_fma_per_cell": gen, "dadd_rate_ops_per_cell": slow,
                            "frac_of_nominal_dfma_issue": issue / (nominal_tflops * 1e3 / 2),
                            "frac_of_measured_dfma_issue": issue / pk["dfma_g_per_s"],
                            "frac_of_measured_dadd_issue": issue / pk["dadd_g_per_s"],
                            "mix_ceiling_ms": t_mix, "frac_of_mix_ceiling": t_mix / t}}
        if fpc is not None:
            ach = cells * fpc / (t * 1e-3) / 1e12
            tb = DRAM_BYTES_PER_CELL.get(name) if h.fd_order == 4 else None
            r.update({"bound": "alu", "achieved": ach, "peak": nominal_tflops, "unit": "TFLOP/s",
                      "frac": ach / nominal_tflops, "frac_of_measured_dfma": ach / dfma_tflops,
                      "traffic": (tb * cells if tb else None)})
        roof[name] = r
    # Refinement-boundary ghost fill on the finest level: the tile-separable
    # prolongation (FP64: the FMAs its tiles execute, counted by the library)
    # and the dense-output apply (HBM: 5 reads + 1 write per ghost value, plus
    # the 12-byte cell record per ghost cell).
    t_pro, t_app, (n_amr, n_tiles, n_slow, tile_fmas) = ctx.sc_time_ghost_kernels(fin_level, 5)
    F = 22
    nvec = 5
    pro_flops = 2 * nvec * F * (tile_fmas + n_slow * 258)
    pro_ach = pro_flops / (t_pro * 1e-3) / 1e12
    roof["amr_prolong"] = {"bound": "alu", "achieved": pro_ach, "peak": nominal_tflops, "unit": "TFLOP/s",
                           "frac": pro_ach / nominal_tflops, "frac_of_measured_dfma": pro_ach / dfma_tflops,
                           "ms_per_launch": t_pro, "ghost_cells": n_amr, "tiles": n_tiles, "fallback_cells": n_slow,
                           "fmas_per_ghost_value": (tile_fmas + n_slow * 258) / max(n_amr, 1),
                           "ghost_values_per_s": n_amr * nvec * F / (t_pro * 1e-3),
                           "frac_at_42_fma_per_value": 2 * 42 * n_amr * nvec * F / (t_pro * 1e-3) / 1e12 / nominal_tflops}
    app_bytes = n_amr * F * 6 * 8 + n_amr * 12
    roof["amr_apply"] = {"bound": "hbm", "achieved": app_bytes / (t_app * 1e-3) / 1e9, "peak": HBM_GBS,
                         "unit": "GB/s", "frac": app_bytes / (t_app * 1e-3) / 1e9 / HBM_GBS, "ms_per_launch": t_app}
    dominant = DOMINANT
    roofline = dict(roof[dominant])
    roofline["kernel"] = dominant
    roofline["peak_source"] = (f"nominal from this device: {pk['sms']} SMs x {pk['sm_clock_mhz']:.0f} MHz x 4 FP64 "
                               f"flop/clk/SM; measured issue rates: DFMA {pk['dfma_g_per_s']:.1f} G/s, "
                               f"DADD {pk['dadd_g_per_s']:.1f} G/s (sc_measure_fp64_peak)")
    roofline["measured_peaks"] = {"dfma_tflops": dfma_tflops, "dadd_g_instr_per_s": pk["dadd_g_per_s"],
                                  "dfma_g_instr_per_s": pk["dfma_g_per_s"], "nominal_tflops": nominal_tflops}
    # the whole coarse step against the FP64 peak: RHS flops of both Z4c
    # passes per cell and stage, over every actual cell update
    if h.fd_order == 4:
        step_tflops = (FLOPS_PER_CELL["z4c_derivs"] + FLOPS_PER_CELL["z4c_stage"]) * 4 * act_per_step / (
            ms_per_step * 1e-3) / 1e12
        roofline["step_level"] = {"achieved": step_tflops, "unit": "TFLOP/s", "frac": step_tflops / nominal_tflops,
                                  "frac_of_measured_dfma": step_tflops / dfma_tflops,
                                  "flops_per_cell_stage": FLOPS_PER_CELL["z4c_derivs"] + FLOPS_PER_CELL["z4c_stage"]}
    roofline["other_kernels"] = {k: v for k, v in roof.items() if k != dominant}

    # End to end through the public API with host buffers: each step uploads
    # the whole state from page-locked host memory (sc_set_state: level 0
    # with its evolved ghost shell), advances one coarse step and reads the
    # state back (sc_get_state: interiors).
    n_in = ctx.sc_state_bytes(True) // 8
    n_out = ctx.sc_state_bytes(False) // 8
    host_in = torch.empty(n_in, dtype=torch.float64).pin_memory()
    host_out = torch.empty(n_out, dtype=torch.float64).pin_memory()
    ctx.sc_get_state(host_in.data_ptr(), ghosted_level0=True)
    h2d, d2h = n_in * 8, n_out * 8
    ne2e = max(1, min(args.steps, 5))
    barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(ne2e)]
    t0 = time.perf_counter()
    t_set = t_get = 0.0
    xfer = {"set": [0.0, 0.0], "get": [0.0, 0.0]}  # [DMA ms, pack/unpack kernel ms], CUDA events in the library
    direct = True
    for q in range(ne2e):
        ta = time.perf_counter()
        ctx.sc_set_state(host_in.data_ptr(), ghosted_level0=True)
        st = ctx.sc_transfer_stats()
        xfer["set"][0] += st["copy_ms"]
        xfer["set"][1] += st["kernel_ms"]
        direct = direct and st["direct"]
        tb = time.perf_counter()
        ev[q][0].record(stream)
        ctx.sc_advance(1)
        ev[q][1].record(stream)
        ev[q][1].synchronize()
        tc = time.perf_counter()
        ctx.sc_get_state(host_out.data_ptr())
        st = ctx.sc_transfer_stats()
        xfer["get"][0] += st["copy_ms"]
        xfer["get"][1] += st["kernel_ms"]
        direct = direct and st["direct"]
        t_set += tb - ta
        t_get += time.perf_counter() - tc
    torch.cuda.synchronize()
    barrier()
    e2e_s = max_over_ranks(dist, time.perf_counter() - t0, "cuda")
    e2e_value = whole_job_rate(world, fin_per_step, ne2e, e2e_s * 1e3)
    e2e_step_ms = sum(a.elapsed_time(b) for a, b in ev) / ne2e  # device time of the step inside the e2e loop
    split = {}
    for k, nbytes in (("set", h2d), ("get", d2h)):
        dma, ker = xfer[k][0] / ne2e, xfer[k][1] / ne2e
        split[k] = {"dma_ms": dma, "kernel_ms": ker, "gb_per_s": nbytes / ((dma + ker) * 1e-3) / 1e9}
    # The other transfer form once, for comparison: one DMA to a device
    # staging buffer plus unpack/pack kernels (the form pageable memory takes).
    ctx.sc_set_transfer_mode(sc.SC_XFER_STAGED)
    staged = {}
    for k, fn, ptr, g0, nbytes in (("set", ctx.sc_set_state, host_in, True, h2d),
                                   ("get", ctx.sc_get_state, host_out, False, d2h)):
        ta = time.perf_counter()
        fn(ptr.data_ptr(), ghosted_level0=g0)
        wall = time.perf_counter() - ta
        st = ctx.sc_transfer_stats()
        staged[k] = {"dma_ms": st["copy_ms"], "kernel_ms": st["kernel_ms"], "host_ms": wall * 1e3,
                     "gb_per_s": nbytes / ((st["copy_ms"] + st["kernel_ms"]) * 1e-3) / 1e9}
    ctx.sc_set_transfer_mode(sc.SC_XFER_AUTO)

    # The method's saving: the same hierarchy with every level at the finest
    # time step (uniform-step mode), timed the same way.
    uniform = None
    if rank == 0 and args.uniform_steps > 0:
        hu = W.bl_7level()
        hu.subcycle = False
        hu.fd_order = args.fd_order
        cu = sc.Context(hu)
        cu.sc_autotune()
        cu.sc_set_initial_data(hu.id_kind, hu.id_params)
        cu.sc_advance(1)
        torch.cuda.synchronize()
        u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        u0.record(stream)
        cu.sc_advance(args.uniform_steps)
        u1.record(stream)
        torch.cuda.synchronize()
        ums = u0.elapsed_time(u1) / args.uniform_steps
        fin_u, act_u = hu.zone_updates_per_coarse_step()
        uniform = {"ms_per_coarse_step": ums, "zone_updates_per_s": fin_u / (ums * 1e-3),
                   "actual_zone_updates_per_coarse_step": act_u, "subcycling_speedup": ums / ms_per_step,
                   "steps": args.uniform_steps}
        cu.close()

    # The same hierarchy in the plain per-box form: every kernel launched box
    # by box directly on the stream, no CUDA graph (same arithmetic, so the
    # same fields), timed the same way.
    per_box = None
    if rank == 0 and args.per_box_steps > 0:
        hp = W.bl_7level()
        hp.fd_order = args.fd_order
        cp = sc.Context(hp, exec_mode=sc.SC_EXEC_PER_BOX)
        cp.sc_autotune()
        cp.sc_set_initial_data(hp.id_kind, hp.id_params)
        cp.sc_advance(1)
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_host = time.perf_counter()
        p0.record(stream)
        cp.sc_advance(args.per_box_steps)
        p1.record(stream)
        torch.cuda.synchronize()
        t_host = time.perf_counter() - t_host
        pms = p0.elapsed_time(p1) / args.per_box_steps
        per_box = {"ms_per_coarse_step": pms, "zone_updates_per_s": fin_per_step / (pms * 1e-3),
                   "host_ms_per_coarse_step": t_host * 1e3 / args.per_box_steps,
                   "launches_per_coarse_step": cp.sc_launches_per_step(), "graph_speedup": pms / ms_per_step,
                   "steps": args.per_box_steps}
        cp.close()

    # The scalar-wave workloads in the plain, graph and persistent forms.
    wave_forms = None
    if rank == 0 and args.wave_forms:
        wave_forms = run_wave_forms(sc, W)

    # Served form vs plain per-box form on a seeded ensemble (60% wave, 40% Z4c requests).
    serving = None
    if rank == 0 and args.serving_requests > 0:
        ctx.close()
        ctx = None
        serving = run_serving_arms(sc, W, args.serving_requests, args.max_active)

    cpu = None
    if rank == 0 and world == 1:
        hs = sample_hierarchy()
        v, dt = oracle_step_rate(hs, 1, 0)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"1 coarse step of {hs.name} ({dt:.1f} s)"}
        if args.cpu_aggregate:
            cpu["aggregate_all_cores"] = cpu_aggregate(os.cpu_count() or 1)
    if ctx is not None:
        ctx.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": h.name, "levels": h.nlevels, "base_cells": 64 ** 3,
                           "fd_order": h.fd_order,
                           "interior_cells": sum(h.interior_cells(l) for l in range(h.nlevels)),
                           "finest_equiv_zone_updates_per_step": fin_per_step,
                           "actual_zone_updates_per_step": act_per_step,
                           "actual_zone_updates_per_s": world * act_per_step / (ms_per_step * 1e-3),
                           "l2": "state ~5 GB per replica > 129 MB L2: inputs larger than L2, no flush",
                           "stencil_tile": list(tile), "tuning": tuning,
                           "state_finite_after_timed_steps": state_finite,
                           "parallelism": f"replicas{world}"},
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "steps": ne2e, "ms_per_step": e2e_s * 1e3 / ne2e, "device_ms_per_step": e2e_step_ms,
                        "set_state_ms": t_set * 1e3 / ne2e, "get_state_ms": t_get * 1e3 / ne2e,
                        "transfer_form": "direct (kernels access page-locked host memory)" if direct else "staged",
                        "transfer_split": split, "staged_form_once": staged},
                "gpu_launches": launches, "clocks": clk, "serving": serving, "uniform_step_mode": uniform,
                "per_box_form": per_box, "wave_forms": wave_forms}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--serving", action="store_true", help="only the 256-request serving ensemble, one JSON line")
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--uniform-steps", type=int, default=2,
                    help="coarse steps of the same hierarchy in uniform-step mode (0: skip)")
    ap.add_argument("--per-box-steps", type=int, default=2,
                    help="coarse steps of the same hierarchy in the plain per-box form, no graph (0: skip)")
    ap.add_argument("--fd-order", type=int, default=4, choices=[4, 8],
                    help="finite-difference order of the Z4c right-hand side (8: the paper's production setting)")
    ap.add_argument("--cpu-aggregate", type=int, default=1,
                    help="1: also time the oracle on every host core at once (aggregate CPU baseline)")
    ap.add_argument("--study", choices=["moving", "wavekernel", "fp64", "z4c3level"],
                    help="one study instead of the benchmark (moving: 9-level moving boxes; wavekernel: the wave "
                         "stage kernel on one 256^3 level; fp64: the measured FP64 issue rates; z4c3level: "
                         "3-level 64^3 Brill-Lindquist, the small case of the ncu captures)")
    ap.add_argument("--study-steps", type=int, default=32)
    ap.add_argument("--wave-forms", type=int, default=1,
                    help="1: time the scalar-wave workloads in the plain, graph and persistent forms")
    ap.add_argument("--serving-requests", type=int, default=256,
                    help="requests of the served-vs-plain ensemble embedded in the default line (0: skip)")
    ap.add_argument("--max-active", type=int, default=8,
                    help="slots of the served arms (8: best p50, p99 and throughput of 4/8/16/32/64 on this ensemble)")
    args = ap.parse_args()
    if args.study:
        print(json.dumps(run_study(args)), flush=True)
        return
    if args.serving:
        res = run_serving(args)
        print(json.dumps({"metric": "ensemble p50/p99 latency and zone-updates/s (served vs plain per-box form)",
                          "unit": "s / zone-updates/s", "data": "synthetic", "dtype": "f64", "serving": res}),
              flush=True)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world)


if __name__ == "__main__":
    main()
