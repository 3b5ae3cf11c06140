"""Small, self-contained cases for kernel profiling (ncu) and quick timing.

    python -m paper_2503_09629_gb300.profile_case z4c [n] [steps] [fd_order]
    python -m paper_2503_09629_gb300.profile_case wave [n] [steps] [fd_order]
    python -m paper_2503_09629_gb300.profile_case wavekernel [n]

z4c: Brill-Lindquist head-on, 3 nested levels of n^3 (default 64: about
1.3 GB of device state, more than L2); wave: the 2-level standing wave.
Prints the wall time per coarse step.  wavekernel: the scalar-wave stage
kernel alone on one periodic n^3 level (default 256), CUDA-event time per
launch and its rates against the FP64-issue and HBM bounds.
"""
import json
import os
import sys
import time

import paper_2503_09629_gb300 as sc
from paper_2503_09629_gb300 import workloads as W


# FP64 instructions per cell of one stage-input update of the 4th-order wave
# stage kernel (two 6-neighbour sums of 5 adds, 3 for the Laplacian, 2
# updates; all issued as DFMAs) and its algorithmic bytes: reads u, Pi, y_n
# (u, Pi), writes k (2) and the next stage input (2).
WAVE_INSTR_PER_CELL = 15
WAVE_BYTES_PER_CELL = 8 * 8


def wave_kernel(n: int) -> dict:
    h = W.Hierarchy(system=W.WAVE, boxes=[[W.cube(0, n)]], ncells0=(n, n, n), origin=(0.0, 0.0, 0.0), h0=1.0 / n,
                    id_kind=W.ID_STANDING_WAVE, id_params=[1.0, 1.0, 1.0, 1.0], name=f"wave 1-level {n}^3")
    ctx = sc.Context(h)
    ctx.sc_autotune()
    ctx.sc_set_initial_data(h.id_kind, h.id_params)
    ms, _ = ctx.sc_time_stage_kernels(0, 20)
    cells = n ** 3
    issue_peak = 152 * 2.070 * 2  # G DFMA/s
    hbm = 6800.0
    try:
        with open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")) as fh:
            hbm = float(json.load(fh)["hbm_gbs"])
    except Exception:
        pass
    out = {"workload": h.name, "ms_per_launch": ms, "cells": cells,
           "fp64_issue_G_per_s": cells * WAVE_INSTR_PER_CELL / (ms * 1e-3) / 1e9,
           "fp64_issue_frac": cells * WAVE_INSTR_PER_CELL / (ms * 1e-3) / 1e9 / issue_peak,
           "algorithmic_GB_per_s": cells * WAVE_BYTES_PER_CELL / (ms * 1e-3) / 1e9,
           "hbm_frac": cells * WAVE_BYTES_PER_CELL / (ms * 1e-3) / 1e9 / hbm,
           "bound_ms": {"fp64_issue": cells * WAVE_INSTR_PER_CELL / issue_peak / 1e6,
                        "hbm": cells * WAVE_BYTES_PER_CELL / hbm / 1e6}}
    ctx.close()
    return out


def main(argv):
    kind = argv[1] if len(argv) > 1 else "z4c"
    if kind == "wavekernel":
        print(json.dumps(wave_kernel(int(argv[2]) if len(argv) > 2 else 256)))
        return
    n = int(argv[2]) if len(argv) > 2 else 64
    steps = int(argv[3]) if len(argv) > 3 else 2
    h = W.bl_3level(n) if kind == "z4c" else W.standing_wave_2level(n)
    h.fd_order = int(argv[4]) if len(argv) > 4 else 4
    ctx = sc.Context(h)
    ctx.sc_set_initial_data(h.id_kind, h.id_params)
    ctx.sc_advance(1)
    ctx.sc_synchronize()
    t0 = time.perf_counter()
    ctx.sc_advance(steps)
    ctx.sc_synchronize()
    dt = (time.perf_counter() - t0) / max(steps, 1)
    print(f"{h.name}, fd order {h.fd_order}: {dt * 1e3:.3f} ms per coarse step, {ctx.sc_launches_per_step()} launches per step")
    ctx.close()


if __name__ == "__main__":
    main(sys.argv)
