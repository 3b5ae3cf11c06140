"""Moving-box run of the 9-level binary-black-hole layout (two box stacks
following the punctures, regridded every coarse step).

    python -m paper_2503_09629_gb300.study_moving [--steps 32]

Each coarse step: interpolate the shift at the punctures, move them along
dx/dt = -beta (forward Euler over the coarse step), regrid levels 3-8 around
the new positions, advance one coarse step.  Prints one JSON line with the
finest-equivalent zone-updates/s including and excluding the regrid and
tracking time, the regrid share, and the puncture track.
"""
import argparse
import json
import time

import numpy as np

import paper_2503_09629_gb300 as sc
from paper_2503_09629_gb300 import workloads as W


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=32)
    ap.add_argument("--n", type=int, default=32)
    args = ap.parse_args()
    import torch
    h, pos, radii, fm = W.moving_9level(args.n)
    ctx = sc.Context(h)
    ctx.sc_autotune()
    ctx.sc_set_initial_data(h.id_kind, h.id_params)
    dt0 = h.cfl * h.h0
    t_regrid = 0.0
    t_step = 0.0
    fin = 0.0
    track = [pos]
    cells = []
    for _ in range(args.steps):
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
        f, _a = ctx.h.zone_updates_per_coarse_step()
        fin += f
        track.append(pos)
        cells.append(sum(ctx.h.interior_cells(l) for l in range(ctx.h.nlevels)))
    finite = ctx.sc_check_finite()
    out = {"workload": h.name, "coarse_steps": args.steps,
           "zone_updates_per_s_incl_regrid": fin / (t_step + t_regrid),
           "zone_updates_per_s_step_only": fin / t_step,
           "regrid_share": t_regrid / (t_step + t_regrid), "mean_step_ms": t_step / args.steps * 1e3,
           "mean_regrid_ms": t_regrid / args.steps * 1e3, "interior_cells_first_last": [cells[0], cells[-1]],
           "puncture_x_first_last": [track[0][1][0], track[-1][1][0]], "state_finite": bool(finite),
           "final_boxes_per_level": [len(b) for b in ctx.h.boxes]}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
