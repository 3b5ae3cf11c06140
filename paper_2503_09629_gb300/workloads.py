"""Seeded synthetic workloads: box hierarchies, initial-data parameters, noise.

This module holds geometry and seeded random inputs only -- none of the
method's arithmetic.  Both the CUDA path and the CPU oracle are fed from here.

Workloads (cell-centred grids, refinement factor 2, 3 ghost cells for 4th-order
differences and 4 for 8th order):
  * ``standing_wave_2level(n)``: periodic [0,1)^3, level 0 n^3, one fine box
    over [0.25,0.75]^3; u = sin(2 pi x) sin(2 pi y) sin(2 pi z), Pi = 0.
  * ``gaussian_3level(n, seed)``: periodic [0,1)^3, 3 levels; levels 1 and 2
    are unions of 6-20 uneven seeded boxes (edges 8-24 cells at n = 64, scaled
    with n); Gaussian pulse (amplitude 1, width 0.05, centre) plus smooth
    seeded noise of total amplitude 1e-3 (8 Fourier modes, |k| <= 4).
  * ``bl_7level()``: Z4c, [-32,32]^3, 7 nested levels, level 0 64^3 (h = 1),
    finest h = 1/64; Brill-Lindquist punctures m = 0.5 at z = +-1.
  * ``bl_3level(n, m1, m2, sep)``: small Z4c hierarchy for parity and serving.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

Box = Tuple[Tuple[int, int, int], Tuple[int, int, int]]

WAVE, Z4C = 0, 1
BC_PERIODIC, BC_RADIATIVE = 0, 1
ID_STANDING_WAVE, ID_GAUSSIAN, ID_BRILL_LINDQUIST, ID_MINKOWSKI, ID_SPHERICAL_GAUSSIAN = 0, 1, 2, 3, 4
ID_BRILL_LINDQUIST_AVG_LAPSE = 5


@dataclass
class Hierarchy:
    system: int
    boxes: List[List[Box]]
    ncells0: Tuple[int, int, int]
    origin: Tuple[float, float, float]
    h0: float
    bc: int = BC_PERIODIC
    cfl: float = 0.25
    subcycle: bool = True
    kappa1: float = 0.02
    kappa2: float = 0.0
    eta: float = 2.0
    ko_sigma: float = 0.3
    eta_profile: Optional[Tuple[float, float, float]] = None  # (eta_c, eta_s, eta_o) of Sec. III.A
    fd_order: int = 4  # finite-difference order of the right-hand sides (4 or 8)
    rk_order: int = 4  # Runge-Kutta method: 4 (classic), 3 (Heun's third order), 2 (midpoint)
    id_kind: int = ID_STANDING_WAVE
    id_params: List[float] = field(default_factory=list)
    name: str = ""

    @property
    def nlevels(self) -> int:
        return len(self.boxes)

    def interior_cells(self, level: int) -> int:
        return sum((hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1) for lo, hi in self.boxes[level])

    def zone_updates_per_coarse_step(self) -> Tuple[float, float]:
        """(finest-equivalent, actual) cell updates of one coarse step."""
        L = self.nlevels
        fin = float(2 ** (L - 1) * sum(self.interior_cells(l) for l in range(L)))
        if self.subcycle:
            act = float(sum(2 ** l * self.interior_cells(l) for l in range(L)))
        else:
            act = fin
        return fin, act

    def nfields(self) -> int:
        return 2 if self.system == WAVE else 22

    @property
    def ghost(self) -> int:
        return 4 if self.fd_order == 8 else 3

    def cell_centres(self, level: int, box: int, ghosted: bool = False):
        lo, hi = self.boxes[level][box]
        h = self.h0 / 2 ** level
        g = self.ghost if ghosted else 0
        ax = [self.origin[d] + (np.arange(lo[d] - g, hi[d] + 1 + g) + 0.5) * h for d in range(3)]
        Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        return X, Y, Z

    def kwargs(self) -> dict:
        kw = dict(bc=self.bc, cfl=self.cfl, subcycle=self.subcycle, kappa1=self.kappa1,
                  kappa2=self.kappa2, eta=self.eta, ko_sigma=self.ko_sigma)
        if self.eta_profile is not None:
            kw["eta_profile"] = self.eta_profile
        if self.fd_order != 4:
            kw["fd_order"] = self.fd_order
        if self.rk_order != 4:
            kw["rk_order"] = self.rk_order
        return kw


def cube(lo: int, n: int) -> Box:
    return ((lo, lo, lo), (lo + n - 1, lo + n - 1, lo + n - 1))


def split_uniform(box: Box, parts: Tuple[int, int, int]) -> List[Box]:
    """Split a box into parts[d] pieces per dimension (even-sized, for alignment)."""
    (lo, hi) = box
    cuts = []
    for d in range(3):
        n = hi[d] - lo[d] + 1
        p = parts[d]
        sizes = [2 * ((n // 2) // p + (1 if q < (n // 2) % p else 0)) for q in range(p)]
        edges = [lo[d]]
        for s in sizes:
            edges.append(edges[-1] + s)
        cuts.append(edges)
    out = []
    for k in range(parts[2]):
        for j in range(parts[1]):
            for i in range(parts[0]):
                out.append(((cuts[0][i], cuts[1][j], cuts[2][k]),
                            (cuts[0][i + 1] - 1, cuts[1][j + 1] - 1, cuts[2][k + 1] - 1)))
    return out


def random_split(box: Box, rng: np.random.Generator, min_edge: int, max_edge: int,
                 scale: int = 1) -> List[Box]:
    """Seeded split of a box into a tensor grid of uneven boxes: each dimension
    is cut into 2 or 3 even-sized pieces with edges in [min_edge, max_edge]
    (at the base resolution; every edge is then multiplied by scale).  The
    number of boxes is 8, 12 or 18."""
    (lo, hi) = box
    n = [(hi[d] - lo[d] + 1) // scale for d in range(3)]
    nparts = [(2, 2, 2), (2, 2, 3), (2, 3, 3)][rng.integers(3)]
    nparts = tuple(np.array(nparts)[rng.permutation(3)])
    edges = []
    for d in range(3):
        for _ in range(10000):
            sizes = 2 * rng.integers(min_edge // 2, max_edge // 2 + 1, size=nparts[d] - 1)
            last = n[d] - int(sizes.sum())
            if min_edge <= last <= max_edge and last % 2 == 0:
                sizes = list(sizes) + [last]
                break
        else:
            raise RuntimeError("random_split: no admissible partition")
        e = [lo[d]]
        for sz in sizes:
            e.append(int(e[-1] + int(sz) * scale))
        edges.append(e)
    out = []
    for k in range(nparts[2]):
        for j in range(nparts[1]):
            for i in range(nparts[0]):
                out.append(((edges[0][i], edges[1][j], edges[2][k]),
                            (edges[0][i + 1] - 1, edges[1][j + 1] - 1, edges[2][k + 1] - 1)))
    return out


def standing_wave_2level(n: int = 32, subcycle: bool = True) -> Hierarchy:
    """Periodic [0,1)^3, level 0 n^3, fine box over [0.25,0.75]^3."""
    return Hierarchy(system=WAVE, boxes=[[cube(0, n)], [cube(n // 2, n)]], ncells0=(n, n, n),
                     origin=(0.0, 0.0, 0.0), h0=1.0 / n, subcycle=subcycle,
                     id_kind=ID_STANDING_WAVE, id_params=[1.0, 1.0, 1.0, 1.0],
                     name=f"wave standing 2-level {n}^3 + fine {n}^3")


def gaussian_3level(n: int = 64, seed: int = 0, subcycle: bool = True) -> Hierarchy:
    """Periodic [0,1)^3, 3 levels; level 0 is a 3x3x3 uneven split of n^3."""
    s = n // 64
    assert s >= 1 and n % 64 == 0
    rng = np.random.default_rng(seed)
    l0 = split_uniform(cube(0, n), (3, 3, 3))
    l1 = random_split(cube(40 * s, 48 * s), rng, 8, 24, scale=s)
    l2 = random_split(cube(104 * s, 48 * s), rng, 8, 24, scale=s)
    return Hierarchy(system=WAVE, boxes=[l0, l1, l2], ncells0=(n, n, n), origin=(0.0, 0.0, 0.0),
                     h0=1.0 / n, subcycle=subcycle, id_kind=ID_GAUSSIAN,
                     id_params=[1.0, 0.05, 0.5, 0.5, 0.5], name=f"wave gaussian 3-level {n}^3 seed {seed}")


def noise_modes(seed: int, nmodes: int = 8, kmax: int = 4, total_amplitude: float = 1e-3):
    """Seeded smooth noise: integer wave vectors with |k| <= kmax, phases,
    amplitudes summing to total_amplitude."""
    rng = np.random.default_rng(10_000 + seed)
    ks = []
    while len(ks) < nmodes:
        k = rng.integers(-kmax, kmax + 1, size=3)
        if 0 < np.linalg.norm(k) <= kmax:
            ks.append(k)
    amps = rng.random(nmodes)
    amps *= total_amplitude / amps.sum()
    phases = rng.random(nmodes) * 2 * np.pi
    return np.array(ks), amps, phases


def noise_field(X, Y, Z, seed: int) -> np.ndarray:
    ks, amps, phases = noise_modes(seed)
    out = np.zeros_like(X)
    for k, a, p in zip(ks, amps, phases):
        out += a * np.sin(2 * np.pi * (k[0] * X + k[1] * Y + k[2] * Z) + p)
    return out


def bl_7level(ko_sigma: float = 0.3) -> Hierarchy:
    """Z4c 7-level box-in-box hierarchy over [-32,32]^3 (level 0: 64^3, h = 1)."""
    def rng_cells(a, b, l):
        h = 1.0 / 2 ** l
        return int(round((a + 32) / h)), int(round((b + 32) / h)) - 1

    def box(l, xr, yr, zr):
        xs, ys, zs = rng_cells(*xr, l), rng_cells(*yr, l), rng_cells(*zr, l)
        return ((xs[0], ys[0], zs[0]), (xs[1], ys[1], zs[1]))

    levels = [
        [box(0, (-32, 32), (-32, 32), (-32, 32))],
        [box(1, (-16, 16), (-16, 16), (-16, 16))],
        [box(2, (-8, 8), (-8, 8), (-8, 8))],
        [box(3, (-4, 4), (-4, 4), (-4, 4))],
        [box(4, (-2, 2), (-2, 2), (-3, 3))],
        [box(5, (-1, 1), (-1, 1), (-2, 2))],
        [box(6, (-0.5, 0.5), (-0.5, 0.5), (-1.5, -0.5)), box(6, (-0.5, 0.5), (-0.5, 0.5), (0.5, 1.5))],
    ]
    return Hierarchy(system=Z4C, boxes=levels, ncells0=(64, 64, 64), origin=(-32.0, -32.0, -32.0), h0=1.0,
                     bc=BC_RADIATIVE, kappa1=0.02, kappa2=0.0, eta=2.0, ko_sigma=ko_sigma,
                     id_kind=ID_BRILL_LINDQUIST, id_params=[0.5, 0.0, 0.0, 1.0, 0.5, 0.0, 0.0, -1.0],
                     name="z4c BL 7-level 64^3 over [-32,32]^3, finest h=1/64")


def bl_3level(n: int = 24, m1: float = 0.5, m2: float = 0.5, sep: float = 2.0, L: float = 8.0) -> Hierarchy:
    """Small Z4c hierarchy: [-L,L]^3, level 0 n^3, levels 1/2 cubes of n cells
    centred on the origin (n >= 20 for proper nesting); BL punctures on the z
    axis."""
    assert n % 4 == 0 and n >= 20
    return Hierarchy(system=Z4C, boxes=[[cube(0, n)], [cube(n - n // 2, n)], [cube(2 * n - n // 2, n)]],
                     ncells0=(n, n, n), origin=(-L, -L, -L), h0=2 * L / n, bc=BC_RADIATIVE,
                     id_kind=ID_BRILL_LINDQUIST,
                     id_params=[m1, 0.0, 0.0, sep / 2, m2, 0.0, 0.0, -sep / 2],
                     name=f"z4c BL 3-level {n}^3 over [-{L},{L}]^3")


def initial_fields(h: Hierarchy, level: int, box: int, ghosted: bool = False, noise_seed=None) -> np.ndarray:
    """Initial data of one box as an array (F, nz, ny, nx) at cell centres
    (ghost cells included when ghosted).  Standing wave / Gaussian (plus the
    seeded smooth noise when noise_seed is given) for the wave, Brill-Lindquist
    or flat space for Z4c."""
    X, Y, Z = h.cell_centres(level, box, ghosted)
    p = h.id_params
    if h.system == WAVE:
        if h.id_kind == ID_STANDING_WAVE:
            u = p[0] * np.sin(2 * np.pi * p[1] * X) * np.sin(2 * np.pi * p[2] * Y) * np.sin(2 * np.pi * p[3] * Z)
        elif h.id_kind == ID_GAUSSIAN:
            u = p[0] * np.exp(-((X - p[2]) ** 2 + (Y - p[3]) ** 2 + (Z - p[4]) ** 2) / (2 * p[1] ** 2))
        else:
            raise ValueError("unsupported wave initial data")
        if noise_seed is not None:
            u = u + noise_field(X, Y, Z, noise_seed)
        return np.stack([u, np.zeros_like(u)])
    out = np.zeros((22,) + X.shape)
    psi = np.ones_like(X)
    if h.id_kind in (ID_BRILL_LINDQUIST, ID_BRILL_LINDQUIST_AVG_LAPSE):
        for q in range(2):
            m, cx, cy, cz = p[4 * q:4 * q + 4]
            psi += m / (2 * np.sqrt((X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2))
    out[0] = psi ** -2       # W = gamma^(-1/6) for gamma_ij = psi^4 delta_ij
    out[1] = out[4] = out[6] = 1.0  # conformal metric = delta
    out[18] = psi ** -2      # lapse psi^-2
    if h.id_kind == ID_BRILL_LINDQUIST_AVG_LAPSE:
        s = psi - 1.0
        out[18] = 0.5 * (1.0 + (1.0 - s) / (1.0 + s))  # averaged lapse (Sec. III.B)
    return out


def serving_requests(n: int = 256, seed: int = 0, burst: bool = False, mean_interarrival: float = 0.0):
    """Seeded serving ensemble: (arrival time, hierarchy, coarse steps) triples.

    60% scalar-wave 2-level runs (coarse n^3 with n in 16..64 step 8, fine box
    over the central half, integer wave numbers 1-4, 8-64 coarse steps) and 40%
    Z4c Brill-Lindquist 3-level runs (coarse n^3 with n in 32..48 step 8 over
    [-8,8]^3, masses 0.3-0.7, separation 2-6 on the z axis, 16 coarse steps).
    Arrivals: all at t = 0 (burst) or Poisson with the given mean interarrival."""
    rng = np.random.default_rng(20_000 + seed)
    out = []
    t = 0.0
    for _ in range(n):
        if not burst and mean_interarrival > 0:
            t += rng.exponential(mean_interarrival)
        if rng.random() < 0.6:
            nb = int(rng.choice(np.arange(16, 65, 8)))
            k = [float(v) for v in rng.integers(1, 5, size=3)]
            h = standing_wave_2level(nb)
            h.id_params = [1.0] + k
            h.name = f"wave 2-level {nb}^3 k={k}"
            steps = int(rng.integers(8, 65))
        else:
            nb = int(rng.choice([32, 40, 48]))
            m1, m2 = rng.uniform(0.3, 0.7, size=2)
            sep = float(rng.uniform(2.0, 6.0))
            h = bl_3level(nb, float(m1), float(m2), sep)
            steps = 16
        out.append((0.0 if burst else t, h, steps))
    return out


# ---------------------------------------------------------------------------
# Moving boxes: box stacks that follow the punctures.

def box_around(centre, radius, level, h0, origin):
    """Box of level `level` covering [centre - radius, centre + radius] in
    every dimension, aligned to parent cells (lo even, hi odd)."""
    h = h0 / 2 ** level
    lo, hi = [], []
    for d in range(3):
        a = int(np.floor((centre[d] - radius - origin[d]) / h))
        b = int(np.ceil((centre[d] + radius - origin[d]) / h)) - 1
        a -= a % 2
        b += 1 - b % 2
        lo.append(a)
        hi.append(b)
    return (tuple(lo), tuple(hi))


def _touch(a, b):
    return all(a[0][d] <= b[1][d] + 1 and b[0][d] <= a[1][d] + 1 for d in range(3))


def merged(boxes):
    """Merge boxes that overlap or touch into their bounding boxes."""
    boxes = list(boxes)
    changed = True
    while changed:
        changed = False
        for i in range(len(boxes)):
            for j in range(i + 1, len(boxes)):
                if _touch(boxes[i], boxes[j]):
                    a, b = boxes[i], boxes[j]
                    boxes[i] = (tuple(min(a[0][d], b[0][d]) for d in range(3)),
                                tuple(max(a[1][d], b[1][d]) for d in range(3)))
                    del boxes[j]
                    changed = True
                    break
            if changed:
                break
    return sorted(boxes)


def moving_layout(h: Hierarchy, positions, radii, first_moving: int):
    """Boxes of every level: the fixed levels of h below first_moving, and for
    each level l >= first_moving one box of radius radii[l] around every
    puncture (merged where they touch)."""
    out = [list(b) for b in h.boxes[:first_moving]]
    for l in range(first_moving, h.nlevels):
        out.append(merged(box_around(p, radii[l], l, h.h0, h.origin) for p in positions))
    return out


def moving_bl(n: int = 32, L: float = 16.0, sep: float = 3.0, m: float = 0.5):
    """Small moving-box Z4c case: level 0 n^3 over [-L,L]^3, level 1 the
    central half, levels 2 and 3 box stacks of radius 2.5 and 1.0 (in units
    of the coordinates) around two Brill-Lindquist punctures on the x axis.
    Returns (hierarchy, positions, radii, first_moving)."""
    q = n // 2
    positions = [(-sep / 2, 0.0, 0.0), (sep / 2, 0.0, 0.0)]
    radii = [None, None, 2.5, 1.0]
    base = Hierarchy(system=Z4C, boxes=[[cube(0, n)], [cube(q, n)]], ncells0=(n, n, n), origin=(-L, -L, -L),
                     h0=2 * L / n, bc=BC_RADIATIVE, id_kind=ID_BRILL_LINDQUIST,
                     id_params=[m, positions[0][0], 0.0, 0.0, m, positions[1][0], 0.0, 0.0],
                     name=f"z4c BL moving boxes {n}^3, 4 levels")
    base.boxes = moving_layout(Hierarchy(**{**base.__dict__, "boxes": base.boxes + [[], []]}), positions, radii, 2)
    return base, positions, radii, 2


def track_punctures(target, positions, dt, shift_fields=(19, 20, 21)):
    """Move the punctures one coarse step along dx/dt = -beta(x) (forward
    Euler with the shift interpolated at the start of the step); target is
    anything with interpolate(points, field)."""
    pts = np.asarray(positions, dtype=np.float64)
    beta = np.stack([target.interpolate(pts, f) for f in shift_fields], axis=1)
    return [tuple(p) for p in pts - dt * beta]


def moving_9level(n: int = 32, sep: float = 6.0, m: float = 0.5):
    """9-level moving-box Brill-Lindquist workload at a size one GPU runs in
    about a second per coarse step: Z4c Brill-Lindquist m = 0.5 at x = +-3,
    9 levels over [-128,128]^3 (level 0 n^3), levels 0-2 fixed nested cubes,
    levels 3-8 box stacks around the punctures with radii 12, 6, 3, 1.5,
    0.75, 0.375 (about 24 cells across at every level; stacks merge where
    they touch).  The Gamma-driver damping uses the eta(r) profile of
    Sec. III.A (eta_c = 2, eta_s = 40, eta_o = 0.25): with the constant
    eta = 2, eta * dt = 4 on level 0 (dt = 2) lies outside RK4's stability
    interval and the coarse levels blow up after about 15 coarse steps, the
    time-step limit dt_max ~ 1/eta that the paper discusses.  The full-size layout (base 128^3, finest radius 1.5 at h = 1/128,
    about 1.7e8 cells and 3e10 cell updates per coarse step) needs about ten
    minutes per coarse step at this path's rate.
    Returns (hierarchy, positions, radii, first_moving)."""
    L = 128.0
    h0 = 2 * L / n
    positions = [(-sep / 2, 0.0, 0.0), (sep / 2, 0.0, 0.0)]
    radii = [None, None, None, 12.0, 6.0, 3.0, 1.5, 0.75, 0.375]
    fixed = [[cube(0, n)], [cube(n // 2, n)], [cube(3 * n // 2, n)]]
    base = Hierarchy(system=Z4C, boxes=fixed + [[] for _ in range(6)], ncells0=(n, n, n), origin=(-L, -L, -L),
                     h0=h0, bc=BC_RADIATIVE, id_kind=ID_BRILL_LINDQUIST,
                     id_params=[m, positions[0][0], 0.0, 0.0, m, positions[1][0], 0.0, 0.0],
                     eta_profile=(2.0, 40.0, 0.25),
                     name=f"z4c BL moving boxes 9-level {n}^3 over [-128,128]^3, eta(r)")
    base.boxes = moving_layout(base, positions, radii, 3)
    return base, positions, radii, 3
