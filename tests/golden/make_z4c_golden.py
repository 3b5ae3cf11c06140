"""Write the stored expected values of the full-size Z4c parity tests.

Calls only the CPU oracle (``oracle/``) and the seeded input generators
(``paper_2503_09629_gb300.workloads``); nothing here touches the CUDA path.
Each case evolves one Z4c hierarchy from Brill-Lindquist data (Sec. III.B,
lapse psi^-2) with the paper's subcycling (Sec. II, steps 1-7 per coarse step)
and stores sampled 8^3 blocks of all 22 fields of every level, taken from the
ghosted box arrays, so that the samples cover

  * a corner and a face of every box with its ghost layers: on refined levels
    these are refinement-boundary ghosts filled by the dense output at the end
    of the last substep (Sec. II, steps 3 and 5), on level 0 the evolved
    radiative shell;
  * the centre of every level that has a finer level: cells overwritten by
    restriction (Sec. II, step 7);
  * the punctures on the finest level.

Cases (names used by tests/test_gpu_z4c_fullsize.py):
  bl7_2steps   the 7-level benchmark hierarchy (64^3 base over [-32,32]^3,
               finest h = 1/64), 2 coarse steps: about an hour single-threaded;
  bl3_48_16    3 levels of 48^3 over [-8,8]^3, 16 coarse steps: a few minutes;
  bl3_32_16_unequal  3 levels of 32^3 over [-8,8]^3, masses 0.3 and 0.7 at
               separation 6 (the smallest and most asymmetric Z4c requests of
               the serving ensemble), 16 coarse steps: about two minutes.

Usage: python tests/golden/make_z4c_golden.py [bl7_2steps|bl3_48_16 ...]
Output: tests/golden/z4c_<case>.npz (block origins, fields, the largest
|value| of each field over the interior cells of the whole hierarchy -- the
scale of the max-relative-difference metric --, oracle time and zone-update
counts).
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2503_09629_gb300 import workloads as W  # noqa: E402

B = 8  # sampled block edge


def sample_origins(h: W.Hierarchy, level: int, box: int):
    """Block origins (z, y, x) in the ghosted box array of one box."""
    lo, hi = h.boxes[level][box]
    g = h.ghost
    ext = [hi[d] - lo[d] + 1 + 2 * g for d in range(3)]  # x, y, z
    cz, cy, cx = [(ext[d] - B) // 2 for d in (2, 1, 0)]
    out = [(0, 0, 0),                         # corner incl. ghosts (refinement boundary / radiative shell)
           (0, cy, cx),                       # centre of the low-z face, incl. ghosts
           (ext[2] - B, ext[1] - B, cx)]      # high-y/high-z edge, incl. ghosts
    if level + 1 < h.nlevels:
        out.append((cz, cy, cx))              # centre: restricted from the finer level
    else:
        # finest level: the puncture inside this box (Brill-Lindquist at z = +-1)
        p = h.id_params
        hl = h.h0 / 2 ** level
        for q in range(2):
            pz = p[4 * q + 3]
            k = int(np.floor((pz - h.origin[2]) / hl - 0.5)) - (lo[2] - g)
            if B // 2 <= k <= ext[2] - B // 2:
                out.append((k - B // 2 + 1, cy, cx))
    return out


def load_initial(o: oracle.Oracle, h: W.Hierarchy):
    """Brill-Lindquist data from the shared input generator; level 0 with its
    ghost layers (the evolved shell of the radiative boundary)."""
    g = h.ghost
    for l in range(h.nlevels):
        for b in range(len(h.boxes[l])):
            a = W.initial_fields(h, l, b, ghosted=True)
            for f in range(a.shape[0]):
                if l == 0:
                    o.set_field(l, b, f, a[f], ghosted=True)
                else:
                    o.set_field(l, b, f, a[f][g:-g, g:-g, g:-g])


def case_hierarchy(name: str):
    if name == "bl7_2steps":
        return W.bl_7level(), 2
    if name == "bl3_48_16":
        return W.bl_3level(48), 16
    if name == "bl3_32_16_unequal":
        return W.bl_3level(32, 0.3, 0.7, 6.0), 16
    raise ValueError(name)


def make(name: str) -> str:
    h, nsteps = case_hierarchy(name)
    o = oracle.Oracle(h.system, h.boxes, h.ncells0, h.origin, h.h0, **h.kwargs())
    load_initial(o, h)
    t0 = time.perf_counter()
    o.advance(nsteps)
    wall = time.perf_counter() - t0
    meta, blocks = [], []
    field_max = np.zeros(22)  # max |value| of each field over the interior cells of the whole hierarchy
    for l in range(h.nlevels):
        for b in range(len(h.boxes[l])):
            full = np.stack([o.get_field(l, b, f, ghosted=True) for f in range(22)])
            g = h.ghost
            field_max = np.maximum(field_max, np.abs(full[:, g:-g, g:-g, g:-g]).max(axis=(1, 2, 3)))
            for (z, y, x) in sample_origins(h, l, b):
                meta.append((l, b, z, y, x))
                blocks.append(full[:, z:z + B, y:y + B, x:x + B].copy())
    fin, act = o.zone_updates()
    path = os.path.join(HERE, f"z4c_{name}.npz")
    np.savez_compressed(path, meta=np.array(meta, dtype=np.int32), blocks=np.stack(blocks),
                        steps=np.int32(nsteps), time=np.float64(o.time), zone_updates=np.array([fin, act]),
                        field_max=field_max, oracle_wall_s=np.float64(wall))
    print(f"{name}: {nsteps} coarse steps in {wall:.0f} s, {len(meta)} blocks -> {path}", flush=True)
    return path


if __name__ == "__main__":
    for n in sys.argv[1:] or ["bl3_48_16", "bl3_32_16_unequal", "bl7_2steps"]:
        make(n)
