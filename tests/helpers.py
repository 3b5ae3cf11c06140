"""Shared helpers of the GPU parity tests: run one seeded workload through
the CUDA library and through the CPU oracle from the same input arrays, and
compare with the max-relative-field-difference metric."""
import numpy as np

from paper_2503_09629_gb300 import workloads as W


def init_arrays(h, noise_seed=None):
    """[level][box] -> (F, nz, ny, nx) initial data incl. ghosts."""
    return [[W.initial_fields(h, l, b, ghosted=True, noise_seed=noise_seed) for b in range(len(h.boxes[l]))]
            for l in range(h.nlevels)]


def _interior(a, g=3):
    return a[:, g:-g, g:-g, g:-g]


def load(target, h, arrays, ghosted_level0=None):
    """Set every field of every box; level 0 with ghosts when the outer
    boundary is radiative (its ghost shell is evolved)."""
    if ghosted_level0 is None:
        ghosted_level0 = h.bc == W.BC_RADIATIVE
    setf = target.sc_set_field if hasattr(target, "sc_set_field") else target.set_field
    for l in range(h.nlevels):
        for b in range(len(h.boxes[l])):
            a = arrays[l][b]
            g = ghosted_level0 and l == 0
            for f in range(a.shape[0]):
                setf(l, b, f, a[f] if g else _interior(a, h.ghost)[f], ghosted=g)


def fetch(target, h):
    getf = target.sc_get_field if hasattr(target, "sc_get_field") else target.get_field
    F = h.nfields()
    return [[np.stack([getf(l, b, f) for f in range(F)]) for b in range(len(h.boxes[l]))] for l in range(h.nlevels)]


def max_rel_diff(gpu, ref, floor=1e-14):
    """max over levels, boxes and fields of max|gpu - ref| / max|ref| (per
    field over the whole hierarchy; fields identically zero use floor)."""
    nf = ref[0][0].shape[0]
    worst = 0.0
    for f in range(nf):
        scale = max(max(np.abs(r[f]).max() for lv in ref for r in lv), floor)
        diff = max(np.abs(g[f] - r[f]).max() for lg, lr in zip(gpu, ref) for g, r in zip(lg, lr))
        worst = max(worst, diff / scale)
    return worst


def make_oracle(orc, h, **over):
    kw = h.kwargs()
    kw.update(over)
    return orc.Oracle(h.system, h.boxes, h.ncells0, h.origin, h.h0, **kw)
