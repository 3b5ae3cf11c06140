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
# FP64 peak derived from the unit counts and clocks: 152 SMs x 2070 MHz x
# 2 DFMA lanes per SM per clock x 2 flops per DFMA.
FP64_PEAK_GFLOPS = 152 * 2.070 * 2 * 2


def _measured_hbm_gbs() -> float:
    """HBM copy bandwidth measured on this machine (MEASURED_PEAKS.json), else
    the profiling recipe's fallback figure (6.8 TB/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except Exception:
        return 6800.0


HBM_GBS = _measured_hbm_gbs()
# Algorithmic FP64 flops per interior cell of each Z4c pass in this
# formulation: adds, multiplies and fused multiply-adds (2 flops) counted by
# ncu on the kernels before their additions were re-expressed as FMAs with a
# unit multiplier (that rewrite changes the instruction, not the arithmetic).
# z4c_derivs = row-segment D_x/D_y pass (133) + per-cell pass (1047);
# profiles/z4c_kernels_bl3level64_ncu.md.
FLOPS_PER_CELL = {"z4c_derivs": 1180.0, "z4c_stage": 1971.0}
# DRAM bytes (read + write) per interior cell of each kernel from an ncu
# capture of a 262,144-cell launch without cache flushes (--cache-control
# none; profiles/z4c_kernels_bl3level64_ncu.md), scaled to a launch by its
# cell count; None once the kernel has changed since the counters were taken.
DRAM_BYTES_PER_CELL = {"z4c_derivs": None,
                       "z4c_stage": (514.633984e6 + 278.21952e6) / 262144}
# FP64 instructions (DFMA + DMUL + DADD, thread-level / cell) per interior
# cell of the derivative pass (D_x/D_y row pass + per-cell pass), counted by
# ncu on the 3-level 64^3 case (profiles/z4c_kernels_bl3level64_ncu.md,
# profiles/z4c_derivs_fd8_bl3level64_ncu.md).  The pass issues its additions
# as DFMAs, so its bound is the DFMA issue rate: 152 SMs x 2070 MHz x 2.
FP64_INSTR_PER_CELL = {4: {"z4c_derivs": 103.0 + 807.0}, 8: {"z4c_derivs": 242.0 + 1324.0}}
FP64_ISSUE_PEAK_G = 152 * 2.070 * 2
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


def run_ensemble(sc, W, n: int, seed: int, burst: bool, mean_interarrival: float, served: bool,
                 budget: int = 48 << 30, max_active: int = 32):
    """Serve the seeded request ensemble; returns latency and throughput.

    served=True: continuous batching (max_active slots, one stream each, CUDA
    graph per coarse step); served=False: the plain per-box form, one request
    at a time in arrival order, kernels launched box by box without graphs."""
    reqs = sorted(W.serving_requests(n, seed, burst=burst, mean_interarrival=mean_interarrival), key=lambda r: r[0])
    srv = sc.Server(budget, max_active if served else 1, 2)
    mode = sc.SC_EXEC_GRAPH if served else sc.SC_EXEC_PER_BOX
    tickets, lat = [], []
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
            "form": "served (continuous batching, graphs)" if served else "plain (FIFO, per-box launches)",
            "p50_s": pct(0.5), "p99_s": pct(0.99), "wall_s": wall,
            "zone_updates_per_s": st["zu_finest"] / wall, "actual_zone_updates_per_s": st["zu_actual"] / wall,
            "gpu_launches": st["launches"]}


def run_serving(args):
    import torch

    import paper_2503_09629_gb300 as sc
    from paper_2503_09629_gb300 import workloads as W
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    sc.build()
    n = args.requests
    plain_burst = run_ensemble(sc, W, n, 0, True, 0.0, served=False)
    served_burst = run_ensemble(sc, W, n, 0, True, 0.0, served=True)
    mean_service = plain_burst["wall_s"] / n
    ia = mean_service / 0.9  # arrival rate 0.9 / mean plain service time
    plain_poisson = run_ensemble(sc, W, n, 0, False, ia, served=False)
    served_poisson = run_ensemble(sc, W, n, 0, False, ia, served=True)
    return {"burst": {"served": served_burst, "plain": plain_burst},
            "poisson": {"served": served_poisson, "plain": plain_poisson,
                        "mean_plain_service_s": mean_service}}


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
    # from CUDA events on the library's stream, on the finest level.
    fin_level = h.nlevels - 1
    cells = h.interior_cells(fin_level)
    t_der, t_stage = ctx.sc_time_stage_kernels(fin_level, 5)
    roof = {}
    for name, t in (("z4c_derivs", t_der), ("z4c_stage", t_stage)):
        fpc = FLOPS_PER_CELL[name] if (h.fd_order == 4 or name == "z4c_stage") else None
        if fpc is None:
            roof[name] = {"ms_per_launch": t, "cells_per_launch": cells, "flops_per_cell": None}
            continue
        ach = cells * fpc / (t * 1e-3) / 1e12
        tb = DRAM_BYTES_PER_CELL.get(name) if h.fd_order == 4 else None
        roof[name] = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_GFLOPS / 1e3, "unit": "TFLOP/s",
                      "frac": ach * 1e3 / FP64_PEAK_GFLOPS, "traffic": (tb * cells if tb else None),
                      "ms_per_launch": t, "cells_per_launch": cells, "flops_per_cell": fpc}
    ipc = FP64_INSTR_PER_CELL[h.fd_order]["z4c_derivs"]
    issue = cells * ipc / (t_der * 1e-3) / 1e9
    roof["z4c_derivs"]["fp64_issue"] = {"achieved": issue, "peak": FP64_ISSUE_PEAK_G, "unit": "G FP64 instr/s",
                                        "frac": issue / FP64_ISSUE_PEAK_G, "instr_per_cell": ipc}
    # Refinement-boundary ghost fill on the finest level: the separable
    # prolongation (FP64: 42 FMAs per fine position of a 4x4x4 block and
    # vector-field, 2688 FMAs per block and vector-field) and the
    # dense-output apply (HBM: 5 reads + 1 write per ghost value, plus the
    # 12-byte cell record per ghost cell).
    t_pro, t_app, (n_amr, n_blk, n_slow) = ctx.sc_time_ghost_kernels(fin_level, 5)
    F = 22
    pro_flops = n_blk * 5 * F * 2688 * 2 + n_slow * 5 * F * 258 * 2
    app_bytes = n_amr * F * 6 * 8 + n_amr * 12
    roof["amr_prolong"] = {"bound": "alu", "achieved": pro_flops / (t_pro * 1e-3) / 1e12,
                           "peak": FP64_PEAK_GFLOPS / 1e3, "unit": "TFLOP/s",
                           "frac": pro_flops / (t_pro * 1e-3) / 1e9 / FP64_PEAK_GFLOPS, "ms_per_launch": t_pro,
                           "ghost_cells": n_amr, "blocks": n_blk, "fallback_cells": n_slow}
    roof["amr_apply"] = {"bound": "hbm", "achieved": app_bytes / (t_app * 1e-3) / 1e9, "peak": HBM_GBS,
                         "unit": "GB/s", "frac": app_bytes / (t_app * 1e-3) / 1e9 / HBM_GBS, "ms_per_launch": t_app}
    dominant = DOMINANT
    roofline = dict(roof[dominant])
    roofline["kernel"] = dominant
    roofline["peak_source"] = "derived: 152 SMs x 2070 MHz x 4 FP64 flop/clk/SM (nominal 1.25 TFLOP/s)"
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

    # Served form vs plain per-box form on a seeded ensemble (60% wave, 40% Z4c requests).
    serving = None
    if rank == 0 and args.serving_requests > 0:
        ctx.close()
        ctx = None
        torch.cuda.empty_cache()
        n = args.serving_requests
        plain = run_ensemble(sc, W, n, 0, True, 0.0, served=False)
        served = run_ensemble(sc, W, n, 0, True, 0.0, served=True)
        ia = plain["wall_s"] / n / 0.9
        plain_p = run_ensemble(sc, W, n, 0, False, ia, served=False)
        served_p = run_ensemble(sc, W, n, 0, False, ia, served=True)
        serving = {"requests": n, "burst": {"served": served, "plain": plain},
                   "poisson_load_0.9": {"served": served_p, "plain": plain_p}}

    cpu = None
    if rank == 0 and world == 1:
        hs = sample_hierarchy()
        v, dt = oracle_step_rate(hs, 1, 0)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"1 coarse step of {hs.name} ({dt:.1f} s)"}
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
                           "stencil_tile": list(tile),
                           "state_finite_after_timed_steps": state_finite,
                           "parallelism": f"replicas{world}"},
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "steps": ne2e, "ms_per_step": e2e_s * 1e3 / ne2e, "device_ms_per_step": e2e_step_ms,
                        "set_state_ms": t_set * 1e3 / ne2e, "get_state_ms": t_get * 1e3 / ne2e,
                        "transfer_form": "direct (kernels access page-locked host memory)" if direct else "staged",
                        "transfer_split": split, "staged_form_once": staged},
                "gpu_launches": launches, "clocks": clk, "serving": serving, "uniform_step_mode": uniform,
                "per_box_form": per_box}
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
    ap.add_argument("--serving-requests", type=int, default=64,
                    help="requests of the served-vs-plain ensemble embedded in the default line (0: skip)")
    args = ap.parse_args()
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
