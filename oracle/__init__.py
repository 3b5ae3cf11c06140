"""ctypes wrapper around the single-threaded FP64 CPU oracle (``oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.  It
shares no code with the CUDA library.

The oracle follows arXiv:2503.09629 Sec. II: RK4 (Eqs. rk1-rk5) on every level,
dense output (Eqs. denseoutput1/2) and the Taylor stage formulas (Eqs. Y1-Y4)
for the refinement-boundary ghost zones, the seven-step subcycling recursion,
tensor-product quintic prolongation and restriction; Sec. III for the Z4c
right-hand side, the puncture gauge and Kreiss-Oliger dissipation; Sec. IV.A
for the scalar wave.  Every part is pinned by the CPU tests (closed forms,
polynomial exactness, exact solutions, convergence orders); the radiative
outer boundary is pinned against its stated reading (outgoing spherical
waves satisfy it exactly), since the paper does not print its formula.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")

WAVE, Z4C = 0, 1
BC_PERIODIC, BC_RADIATIVE, BC_CALLBACK = 0, 1, 2
ID_STANDING_WAVE, ID_GAUSSIAN, ID_BRILL_LINDQUIST, ID_MINKOWSKI, ID_SPHERICAL_GAUSSIAN = 0, 1, 2, 3, 4
ID_BRILL_LINDQUIST_AVG_LAPSE = 5
V_Y, V_YOLD, V_STAGE, V_K1 = 0, 1, 2, 3
GHOST = 3

BC_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                         ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double))


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2, no FMA contraction)."""
    src = os.path.join(HERE, "oracle.cpp")
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(src):
        tmp = LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, src])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB_PATH)
        D = ctypes.c_double
        P = ctypes.c_void_p
        I = ctypes.c_int
        DP = ctypes.POINTER(ctypes.c_double)
        IP = ctypes.POINTER(ctypes.c_int)
        L.orc_create.argtypes = [I, I, IP, IP, IP, DP, D, I, D, I, DP, ctypes.POINTER(P)]
        L.orc_create_ex.argtypes = [I, I, IP, IP, IP, DP, D, I, D, I, DP, I, I, ctypes.POINTER(P)]
        L.orc_destroy.argtypes = [P]
        L.orc_nfields.argtypes = [P]
        L.orc_set_bc_callback.argtypes = [P, BC_FN, P]
        L.orc_set_eta_profile.argtypes = [P, D, D, D]
        L.orc_set_initial_data.argtypes = [P, I, DP, I]
        for name in ("orc_set_field", "orc_get_field", "orc_set_field_ghosted", "orc_get_field_ghosted"):
            getattr(L, name).argtypes = [P, I, I, I, DP]
        L.orc_advance.argtypes = [P, I]
        L.orc_time.argtypes = [P]
        L.orc_time.restype = D
        L.orc_zone_updates.argtypes = [P, DP, DP]
        L.orc_dense_b.argtypes = [D, I, DP]
        L.orc_amr_value.argtypes = [D, DP, D, D, I]
        L.orc_amr_value.restype = D
        L.orc_dense_b_rk.argtypes = [I, D, I, DP]
        L.orc_amr_value_rk.argtypes = [I, D, DP, D, D, I]
        L.orc_amr_value_rk.restype = D
        L.orc_rhs_box.argtypes = [P, I, I, DP, DP]
        L.orc_constraints.argtypes = [P, I, I, DP]
        L.orc_debug_set_vector.argtypes = [P, I, I, I, I, DP]
        L.orc_debug_get_vector.argtypes = [P, I, I, I, I, DP]
        L.orc_debug_prolong.argtypes = [P, I]
        L.orc_debug_fill_amr.argtypes = [P, I, I, D, I]
        L.orc_debug_restrict.argtypes = [P, I]
        L.orc_debug_fill_ghosts.argtypes = [P]
        L.orc_flop_counts.argtypes = [DP]
        L.orc_regrid.argtypes = [P, IP, IP]
        L.orc_interpolate.argtypes = [P, I, DP, I, DP]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def dense_b(theta: float, m: int = 0, rk: int = 4) -> np.ndarray:
    """m-th theta-derivative of the dense-output weights b_1..b_4 of the
    rk-stage method (unused stages have weight 0)."""
    b = np.zeros(4)
    if rk == 4:
        lib().orc_dense_b(theta, m, _dp(b))
    else:
        lib().orc_dense_b_rk(rk, theta, m, _dp(b))
    return b


def amr_value(y: float, k, H: float, theta0: float, which: int, rk: int = 4) -> float:
    kk = np.zeros(4)
    kk[:len(k)] = np.asarray(k, dtype=np.float64)
    k = kk
    if rk == 4:
        return lib().orc_amr_value(y, _dp(k), H, theta0, which)
    return lib().orc_amr_value_rk(rk, y, _dp(k), H, theta0, which)


def flop_counts() -> dict:
    c = np.zeros(4)
    lib().orc_flop_counts(_dp(c))
    return {"add": c[0], "mul": c[1], "div": c[2], "total": c[3]}


class Oracle:
    """One box hierarchy evolved by the oracle.

    boxes: list over levels of lists of ((lo_x, lo_y, lo_z), (hi_x, hi_y, hi_z)),
    inclusive cell indices in the level's own index space.
    """

    def __init__(self, system, boxes, ncells0, origin, h0, bc=BC_PERIODIC, cfl=0.25,
                 subcycle=True, kappa1=0.02, kappa2=0.0, eta=2.0, ko_sigma=0.3, eta_profile=None, fd_order=4,
                 rk_order=4):
        L = lib()
        self.system = system
        self.boxes = [[(tuple(lo), tuple(hi)) for lo, hi in lvl] for lvl in boxes]
        nb = (ctypes.c_int * len(boxes))(*[len(b) for b in boxes])
        flat = []
        for lvl in boxes:
            for lo, hi in lvl:
                flat += list(lo) + list(hi)
        fb = (ctypes.c_int * len(flat))(*flat)
        nc = (ctypes.c_int * 3)(*ncells0)
        org = (ctypes.c_double * 3)(*origin)
        prm = (ctypes.c_double * 4)(kappa1, kappa2, eta, ko_sigma)
        h = ctypes.c_void_p()
        rc = L.orc_create_ex(system, len(boxes), nb, fb, nc, org, h0, bc, cfl, 1 if subcycle else 0, prm,
                             int(fd_order), int(rk_order), ctypes.byref(h))
        if rc != 0:
            raise ValueError(f"oracle create failed ({rc})")
        self.h = h
        self.ghost = 4 if fd_order == 8 else 3
        self.F = L.orc_nfields(h)
        self._cb = None
        if eta_profile is not None:
            if L.orc_set_eta_profile(h, *[float(v) for v in eta_profile]) != 0:
                raise ValueError("bad eta profile")

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def shape(self, level, box, ghosted=False):
        lo, hi = self.boxes[level][box]
        n = [hi[d] - lo[d] + 1 + (2 * self.ghost if ghosted else 0) for d in range(3)]
        return (n[2], n[1], n[0])

    def set_bc_callback(self, fn):
        """fn(which, t_n, dt, xyz[npts,3]) -> values[F, npts]."""
        F = self.F

        def cb(user, which, t_n, dt, npts, xyz, out):
            x = np.ctypeslib.as_array(xyz, shape=(npts * 3,)).reshape(npts, 3).copy()
            vals = np.asarray(fn(which, t_n, dt, x), dtype=np.float64).reshape(F, npts)
            o = np.ctypeslib.as_array(out, shape=(F * npts,))
            o[:] = vals.ravel()

        self._cb = BC_FN(cb)
        lib().orc_set_bc_callback(self.h, self._cb, None)

    def set_initial_data(self, kind, params):
        p = np.ascontiguousarray(params, dtype=np.float64)
        rc = lib().orc_set_initial_data(self.h, kind, _dp(p), len(p))
        if rc != 0:
            raise ValueError("initial data failed")

    def set_field(self, level, box, field, arr, ghosted=False):
        a = np.ascontiguousarray(arr, dtype=np.float64)
        assert a.shape == self.shape(level, box, ghosted)
        fn = lib().orc_set_field_ghosted if ghosted else lib().orc_set_field
        if fn(self.h, level, box, field, _dp(a)) != 0:
            raise IndexError("set_field")

    def get_field(self, level, box, field, ghosted=False):
        a = np.zeros(self.shape(level, box, ghosted))
        fn = lib().orc_get_field_ghosted if ghosted else lib().orc_get_field
        if fn(self.h, level, box, field, _dp(a)) != 0:
            raise IndexError("get_field")
        return a

    def set_vector(self, level, box, vec, field, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64)
        assert a.shape == self.shape(level, box, True)
        if lib().orc_debug_set_vector(self.h, level, box, vec, field, _dp(a)) != 0:
            raise IndexError("set_vector")

    def get_vector(self, level, box, vec, field):
        a = np.zeros(self.shape(level, box, True))
        if lib().orc_debug_get_vector(self.h, level, box, vec, field, _dp(a)) != 0:
            raise IndexError("get_vector")
        return a

    def advance(self, n):
        if lib().orc_advance(self.h, n) != 0:
            raise RuntimeError("advance")

    @property
    def time(self):
        return lib().orc_time(self.h)

    def zone_updates(self):
        a, b = ctypes.c_double(), ctypes.c_double()
        lib().orc_zone_updates(self.h, ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value

    def rhs_box(self, level, box, state_ghosted):
        s = np.ascontiguousarray(state_ghosted, dtype=np.float64)
        assert s.shape == (self.F,) + self.shape(level, box, True)
        out = np.zeros_like(s)
        if lib().orc_rhs_box(self.h, level, box, _dp(s), _dp(out)) != 0:
            raise IndexError("rhs_box")
        return out

    def constraints(self, level, box):
        out = np.zeros((7,) + self.shape(level, box))
        if lib().orc_constraints(self.h, level, box, _dp(out)) != 0:
            raise ValueError("constraints")
        return out

    def prolong(self, level):
        assert lib().orc_debug_prolong(self.h, level) == 0

    def fill_amr(self, level, vec, theta0, which):
        assert lib().orc_debug_fill_amr(self.h, level, vec, theta0, which) == 0

    def restrict(self, level):
        assert lib().orc_debug_restrict(self.h, level) == 0

    def fill_ghosts(self):
        assert lib().orc_debug_fill_ghosts(self.h) == 0

    def regrid(self, boxes):
        """New boxes for every level (level 0 unchanged)."""
        nb = (ctypes.c_int * len(boxes))(*[len(b) for b in boxes])
        flat = [v for lvl in boxes for lo, hi in lvl for v in list(lo) + list(hi)]
        fb = (ctypes.c_int * len(flat))(*flat)
        rc = lib().orc_regrid(self.h, nb, fb)
        if rc != 0:
            raise ValueError(f"regrid failed ({rc})")
        self.boxes = [[(tuple(lo), tuple(hi)) for lo, hi in lvl] for lvl in boxes]

    def interpolate(self, points, field):
        p = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
        out = np.zeros(len(p))
        if lib().orc_interpolate(self.h, len(p), _dp(p), field, _dp(out)) != 0:
            raise ValueError("interpolate failed")
        return out

    def cell_centres(self, level, box, h0, origin, ghosted=False):
        """Cell-centre coordinates (z, y, x order arrays) of a box."""
        lo, hi = self.boxes[level][box]
        h = h0 / 2 ** level
        g = self.ghost if ghosted else 0
        ax = [origin[d] + (np.arange(lo[d] - g, hi[d] + 1 + g) + 0.5) * h for d in range(3)]
        Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        return X, Y, Z
