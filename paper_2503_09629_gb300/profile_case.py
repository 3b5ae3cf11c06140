"""Small, self-contained cases for kernel profiling (ncu) and quick timing.

    python -m paper_2503_09629_gb300.profile_case z4c [n] [steps] [fd_order]
    python -m paper_2503_09629_gb300.profile_case wave [n] [steps] [fd_order]

z4c: Brill-Lindquist head-on, 3 nested levels of n^3 (default 64: about
1.3 GB of device state, more than L2); wave: the 2-level standing wave.
Prints the wall time per coarse step.
"""
import sys
import time

import paper_2503_09629_gb300 as sc
from paper_2503_09629_gb300 import workloads as W


def main(argv):
    kind = argv[1] if len(argv) > 1 else "z4c"
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
