"""Scalar-wave 3-level study on seeded uneven boxes (64^3, 128^3, 256^3 base).

    python -m paper_2503_09629_gb300.study_wave3level [--steps64 32]

Runs the Gaussian pulse (amplitude 1, width 0.05) plus seeded smooth noise
(1e-3) on three resolutions with identical physical box layouts (the seeded
layout scaled by 2 and 4) to the same final time, and prints one JSON line:
  * self-convergence order on the finest level: log2(|u64 - I u128| /
    |u128 - I u256|), where I maps a level-2 solution to the cell centres of
    the next coarser resolution by 6-point Lagrange interpolation at the
    midpoint in each dimension (6th-order accurate, far below the 4th-order
    error it measures);
  * finest-equivalent zone-updates/s of the batched graph form and of the
    plain per-box form on each resolution (same fields, bitwise).
"""
import argparse
import json

import numpy as np

import paper_2503_09629_gb300 as sc
from paper_2503_09629_gb300 import workloads as W

MID6 = np.array([3.0, -25.0, 150.0, 150.0, -25.0, 3.0]) / 256.0


def finest_region(ctx, h, seed):
    """Level-2 field u as one array over the bounding box of its boxes."""
    boxes = h.boxes[2]
    lo = np.min([b[0] for b in boxes], axis=0)
    hi = np.max([b[1] for b in boxes], axis=0)
    out = np.full(tuple((hi - lo + 1)[::-1]), np.nan)
    for bi, (blo, bhi) in enumerate(boxes):
        a = ctx.sc_get_field(2, bi, 0)
        sl = tuple(slice(blo[d] - lo[d], bhi[d] - lo[d] + 1) for d in (2, 1, 0))
        out[sl] = a
    return out


def to_coarse(u):
    """6-point midpoint interpolation of a fine cell-centred array onto the
    centres of the coarse cells (pairs of fine cells), per dimension."""
    for ax in range(3):
        n = u.shape[ax] // 2
        pieces = []
        for C in range(2, n - 2):
            idx = np.arange(2 * C - 2, 2 * C + 4)
            pieces.append(np.tensordot(np.take(u, idx, axis=ax), MID6, axes=([ax], [0])))
        u = np.stack(pieces, axis=ax)
    return u


def run(n, steps, mode, seed=0, tune=True):
    h = W.gaussian_3level(n, seed)
    ctx = sc.Context(h, exec_mode=mode)
    for l in range(h.nlevels):
        for b in range(len(h.boxes[l])):
            a = W.initial_fields(h, l, b, noise_seed=seed)
            for f in range(2):
                ctx.sc_set_field(l, b, f, a[f])
    tile = None
    if tune and mode == sc.SC_EXEC_GRAPH:
        tile, _ = ctx.sc_autotune()
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ctx.sc_advance(steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    fin, _act = ctx.sc_zone_updates()
    return ctx, h, fin / (ms * 1e-3), ms, tile


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps64", type=int, default=32)
    args = ap.parse_args()
    res = {"workload": "wave 3-level seeded uneven boxes, Gaussian w=0.05 + 1e-3 noise", "runs": []}
    fine = {}
    for n in (64, 128, 256):
        steps = args.steps64 * n // 64
        ctx, h, zu, ms, tile = run(n, steps, sc.SC_EXEC_GRAPH)
        fine[n] = finest_region(ctx, h, 0)
        t = ctx.sc_get_time()
        ctx.close()
        pctx, _h, zu_plain, ms_plain, _ = run(n, steps, sc.SC_EXEC_PER_BOX)
        same = np.array_equal(finest_region(pctx, _h, 0), fine[n])
        pctx.close()
        res["runs"].append({"n": n, "coarse_steps": steps, "t_final": t, "graph_zone_updates_per_s": zu,
                            "graph_ms": ms, "per_box_zone_updates_per_s": zu_plain, "per_box_ms": ms_plain,
                            "tile": tile, "per_box_bitwise_equal": bool(same),
                            "boxes_per_level": [len(b) for b in h.boxes]})
    # to_coarse drops 2 coarse cells at each end, matching [2:-2] of the coarser run
    e1 = np.abs(fine[64][2:-2, 2:-2, 2:-2] - to_coarse(fine[128])).max()
    e2 = np.abs(fine[128][2:-2, 2:-2, 2:-2] - to_coarse(fine[256])).max()
    res["self_convergence"] = {"e_64_128": float(e1), "e_128_256": float(e2), "order": float(np.log2(e1 / e2))}
    print(json.dumps(res))


if __name__ == "__main__":
    main()
