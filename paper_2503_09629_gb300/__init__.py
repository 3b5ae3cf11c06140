"""GB300-native RK4 subcycling in time with dense-output ghost filling.

Python binding of ``libsubcyc.so`` (C ABI declared in ``include/subcyc.h``):
argument marshalling only.  Every step of the evolution runs in the library's
CUDA kernels; there is no CPU fallback -- if the library cannot be loaded, or
no CUDA device is present, every call raises.  PyTorch supplies device memory
(through its caching allocator) and the CUDA stream.

Method: arXiv:2503.09629 Sec. II (RK4 with dense output, Taylor stage
reconstruction at refinement-boundary ghosts, subcycling recursion,
restriction), Sec. III (Z4c with puncture gauge and Kreiss-Oliger
dissipation), Sec. IV.A (scalar wave).
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import workloads  # noqa: F401  (seeded synthetic inputs)

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsubcyc.so")

SC_OK, SC_EINVAL, SC_ENOMEM, SC_ECUDA, SC_ENESTING, SC_ENONFINITE, SC_ETIMEOUT, SC_EBUSY = 0, -1, -2, -3, -4, -5, -6, -7
SC_WAVE, SC_Z4C = 0, 1
SC_BC_PERIODIC, SC_BC_RADIATIVE = 0, 1
SC_EXEC_GRAPH, SC_EXEC_PER_BOX, SC_EXEC_PERSISTENT = 0, 1, 2
SC_XFER_AUTO, SC_XFER_STAGED, SC_XFER_DIRECT = 0, 1, 2
GHOST = 3
NCONSTRAINTS = 7


class SubcycError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class sc_box(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_int * 3), ("hi", ctypes.c_int * 3)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class sc_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", ctypes.c_void_p)]


class sc_desc(ctypes.Structure):
    _fields_ = [
        ("system", ctypes.c_int),
        ("nlevels", ctypes.c_int),
        ("nboxes", ctypes.POINTER(ctypes.c_int)),
        ("boxes", ctypes.POINTER(sc_box)),
        ("ncells0", ctypes.c_int * 3),
        ("origin", ctypes.c_double * 3),
        ("h0", ctypes.c_double),
        ("outer_bc", ctypes.c_int),
        ("cfl", ctypes.c_double),
        ("subcycle", ctypes.c_int),
        ("kappa1", ctypes.c_double),
        ("kappa2", ctypes.c_double),
        ("eta", ctypes.c_double),
        ("ko_sigma", ctypes.c_double),
        ("cuda_stream", ctypes.c_void_p),
        ("allocator", ctypes.POINTER(sc_allocator)),
        ("exec_mode", ctypes.c_int),
        ("autotune", ctypes.c_int),
        ("eta_profile", ctypes.c_int),
        ("eta_c", ctypes.c_double),
        ("eta_s", ctypes.c_double),
        ("eta_o", ctypes.c_double),
        ("fd_order", ctypes.c_int),
        ("rk_order", ctypes.c_int),
        ("finite_check", ctypes.c_int),
    ]


_lib = None


def build(verbose: bool = False) -> str:
    from . import buildlib
    return buildlib.build(verbose=verbose)


def lib():
    """Load libsubcyc.so (building it first if absent); raises if impossible."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        build()
    L = ctypes.CDLL(LIB_PATH)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    DP = ctypes.POINTER(ctypes.c_double)
    L.sc_last_error.restype = ctypes.c_char_p
    L.sc_create.argtypes = [ctypes.POINTER(sc_desc), ctypes.POINTER(P)]
    L.sc_destroy.argtypes = [P]
    L.sc_destroy.restype = None
    L.sc_set_initial_data.argtypes = [P, I, DP, I]
    for name in ("sc_set_field", "sc_set_field_ghosted", "sc_get_field", "sc_get_field_ghosted"):
        getattr(L, name).argtypes = [P, I, I, I, DP]
    for name in ("sc_set_field_device", "sc_get_field_device"):
        getattr(L, name).argtypes = [P, I, I, I, P]
    L.sc_advance.argtypes = [P, I]
    L.sc_synchronize.argtypes = [P]
    L.sc_synchronize_timeout.argtypes = [P, D]
    L.sc_get_constraints.argtypes = [P, I, I, DP]
    L.sc_get_time.argtypes = [P, DP]
    L.sc_zone_updates.argtypes = [P, DP, DP]
    L.sc_launches_per_step.argtypes = [P, ctypes.POINTER(ctypes.c_long)]
    L.sc_footprint.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
    L.sc_footprint_estimate.argtypes = [ctypes.POINTER(sc_desc), ctypes.POINTER(ctypes.c_size_t)]
    L.sc_time_stage_kernels.argtypes = [P, I, I, DP]
    L.sc_run_op_class_pass.argtypes = [P, I]
    L.sc_autotune.argtypes = [P, ctypes.POINTER(ctypes.c_int), DP]
    L.sc_get_tuning.argtypes = [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_int)]
    L.sc_set_tuning.argtypes = [P, ctypes.POINTER(ctypes.c_int), I, I]
    L.sc_time_ghost_kernels.argtypes = [P, I, I, DP, ctypes.POINTER(ctypes.c_long)]
    L.sc_debug_get_vector.argtypes = [P, I, I, I, I, I, DP]
    L.sc_regrid.argtypes = [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(sc_box)]
    L.sc_check_finite.argtypes = [P]
    L.sc_interpolate.argtypes = [P, I, DP, I, DP]
    L.sc_state_bytes.argtypes = [P, I, ctypes.POINTER(ctypes.c_size_t)]
    L.sc_set_state.argtypes = [P, P, I]
    L.sc_get_state.argtypes = [P, P, I]
    L.sc_set_transfer_mode.argtypes = [P, I]
    L.sc_transfer_stats.argtypes = [P, DP, DP, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_int)]
    L.sc_z4c_constraints_noalloc.argtypes = [P, P, ctypes.POINTER(ctypes.c_int), D, P]
    L.sc_measure_fp64_peak.argtypes = [P, DP, DP, ctypes.POINTER(ctypes.c_int), DP]
    IP = ctypes.POINTER(ctypes.c_int)
    U64 = ctypes.c_ulonglong
    L.sc_server_create.argtypes = [ctypes.c_size_t, I, I, ctypes.POINTER(P)]
    L.sc_server_submit.argtypes = [P, ctypes.POINTER(sc_desc), I, DP, I, I, ctypes.POINTER(U64)]
    L.sc_server_tick.argtypes = [P, IP, IP, IP]
    L.sc_server_poll.argtypes = [P, U64, IP, DP]
    L.sc_server_wait.argtypes = [P, U64, D, DP]
    L.sc_server_inject_alloc_failure.argtypes = [P, ctypes.c_long]
    L.sc_server_set_merge.argtypes = [P, I]
    L.sc_server_read.argtypes = [P, U64, I, I, I, DP]
    L.sc_server_release.argtypes = [P, U64]
    L.sc_server_stats.argtypes = [P, DP, DP, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_size_t)]
    L.sc_server_destroy.argtypes = [P]
    _lib = L
    return L


def _check(rc: int):
    if rc != SC_OK:
        raise SubcycError(rc, lib().sc_last_error().decode(errors="replace"))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _torch_allocator():
    """sc_allocator backed by PyTorch's CUDA caching allocator."""
    import torch

    dev = torch.cuda.current_device()

    def _alloc(nbytes, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev)
        except Exception:  # out of memory -> NULL, the library reports SC_ENOMEM
            return None

    def _free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)

    a = sc_allocator(ALLOC_FN(_alloc), FREE_FN(_free), None)
    return a


def make_desc(h, stream: Optional[int] = None, allocator=None, exec_mode: int = SC_EXEC_GRAPH,
              finite_check: bool = False):
    """sc_desc for a workloads.Hierarchy; returns (desc, keepalive)."""
    nb = (ctypes.c_int * h.nlevels)(*[len(b) for b in h.boxes])
    flat = [bx for lvl in h.boxes for bx in lvl]
    boxes = (sc_box * len(flat))()
    for i, (lo, hi) in enumerate(flat):
        boxes[i].lo[:] = list(lo)
        boxes[i].hi[:] = list(hi)
    d = sc_desc()
    d.system = h.system
    d.nlevels = h.nlevels
    d.nboxes = nb
    d.boxes = boxes
    d.ncells0[:] = list(h.ncells0)
    d.origin[:] = list(h.origin)
    d.h0 = h.h0
    d.outer_bc = h.bc
    d.cfl = h.cfl
    d.subcycle = 1 if h.subcycle else 0
    d.kappa1, d.kappa2, d.eta, d.ko_sigma = h.kappa1, h.kappa2, h.eta, h.ko_sigma
    d.cuda_stream = stream
    d.exec_mode = exec_mode
    d.fd_order = int(getattr(h, "fd_order", 4))
    d.rk_order = int(getattr(h, "rk_order", 4))
    d.finite_check = 1 if finite_check else 0
    prof = getattr(h, "eta_profile", None)
    if prof is not None:
        d.eta_profile = 1
        d.eta_c, d.eta_s, d.eta_o = (float(v) for v in prof)
    keep = [nb, boxes]
    if allocator is not None:
        d.allocator = ctypes.pointer(allocator)
        keep.append(allocator)
    return d, keep


def sc_z4c_constraints_noalloc(dev_state: int, dev_out: int, n: Sequence[int], h: float,
                               stream: Optional[int] = None) -> None:
    """Z4c constraints of one box in caller-owned device memory, with no
    device allocation (for callers that cannot allocate: an embedding
    application that owns all device memory, a fixed memory pool, or a loop
    that must not trigger the implicit synchronisation of cudaMalloc/cudaFree).
    dev_state: 22 ghosted fields of (n+6)^3-shaped boxes, contiguous; dev_out:
    7 * prod(n) doubles.  At most 32,768 cells including ghosts.  Calls share
    one static scratch array: do not overlap them on the GPU."""
    nn = (ctypes.c_int * 3)(*[int(v) for v in n])
    _check(lib().sc_z4c_constraints_noalloc(ctypes.c_void_p(dev_state), ctypes.c_void_p(dev_out), nn, float(h),
                                            ctypes.c_void_p(stream) if stream else None))


def sc_measure_fp64_peak(stream: Optional[int] = None) -> dict:
    """Measured FP64 issue rates of the current GPU (G instr/s) with its SM
    count and maximum SM clock."""
    a, b, mhz = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    n = ctypes.c_int()
    _check(lib().sc_measure_fp64_peak(ctypes.c_void_p(stream) if stream else None, ctypes.byref(a), ctypes.byref(b),
                                      ctypes.byref(n), ctypes.byref(mhz)))
    return {"dfma_g_per_s": a.value, "dadd_g_per_s": b.value, "sms": n.value, "sm_clock_mhz": mhz.value}


def sc_footprint_estimate(h) -> int:
    d, _keep = make_desc(h)
    n = ctypes.c_size_t()
    _check(lib().sc_footprint_estimate(ctypes.byref(d), ctypes.byref(n)))
    return n.value


class Context:
    """One box hierarchy resident on the GPU (wraps an ``sc_ctx*``).

    Method names follow the C ABI (``sc_<name>``).  ``use_torch`` routes
    device allocation through PyTorch's caching allocator and orders all work
    on PyTorch's current CUDA stream.
    """

    def __init__(self, h, use_torch: bool = True, stream: Optional[int] = None, exec_mode: int = SC_EXEC_GRAPH,
                 finite_check: bool = True, allocator=None):
        L = lib()
        self.h = h
        self._alloc = None
        if use_torch:
            import torch
            if not torch.cuda.is_available():
                raise SubcycError(SC_ECUDA, "no CUDA device available")
            if stream is None:
                stream = torch.cuda.current_stream().cuda_stream
            self._alloc = _torch_allocator()
        if allocator is not None:
            self._alloc = allocator
        d, self._keep = make_desc(h, stream, self._alloc, exec_mode, finite_check)
        ctx = ctypes.c_void_p()
        _check(L.sc_create(ctypes.byref(d), ctypes.byref(ctx)))
        self.ctx = ctx
        self.F = h.nfields()

    def close(self):
        if getattr(self, "ctx", None):
            lib().sc_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def ghost(self) -> int:
        """Ghost layers per box: 3 (4th-order differences) or 4 (8th order)."""
        return 4 if int(getattr(self.h, "fd_order", 4)) == 8 else 3

    def shape(self, level: int, box: int, ghosted: bool = False) -> Tuple[int, int, int]:
        lo, hi = self.h.boxes[level][box]
        g = 2 * self.ghost if ghosted else 0
        return (hi[2] - lo[2] + 1 + g, hi[1] - lo[1] + 1 + g, hi[0] - lo[0] + 1 + g)

    def sc_set_initial_data(self, kind: int, params: Sequence[float]):
        p = np.ascontiguousarray(params, dtype=np.float64)
        _check(lib().sc_set_initial_data(self.ctx, kind, _dp(p) if len(p) else None, len(p)))

    def sc_set_field(self, level, box, field, arr, ghosted=False):
        a = np.ascontiguousarray(arr, dtype=np.float64)
        if a.shape != self.shape(level, box, ghosted):
            raise ValueError(f"shape {a.shape} != {self.shape(level, box, ghosted)}")
        fn = lib().sc_set_field_ghosted if ghosted else lib().sc_set_field
        _check(fn(self.ctx, level, box, field, _dp(a)))

    def sc_get_field(self, level, box, field, ghosted=False) -> np.ndarray:
        a = np.empty(self.shape(level, box, ghosted))
        fn = lib().sc_get_field_ghosted if ghosted else lib().sc_get_field
        _check(fn(self.ctx, level, box, field, _dp(a)))
        return a

    def sc_set_field_device(self, level, box, field, dev_ptr: int):
        _check(lib().sc_set_field_device(self.ctx, level, box, field, ctypes.c_void_p(dev_ptr)))

    def sc_get_field_device(self, level, box, field, dev_ptr: int):
        _check(lib().sc_get_field_device(self.ctx, level, box, field, ctypes.c_void_p(dev_ptr)))

    def sc_state_bytes(self, ghosted_level0: bool = False) -> int:
        n = ctypes.c_size_t(0)
        _check(lib().sc_state_bytes(self.ctx, 1 if ghosted_level0 else 0, ctypes.byref(n)))
        return n.value

    def sc_set_state(self, host_ptr, ghosted_level0: bool = False):
        """Whole state from a packed host buffer: a numpy float64 array or a
        raw address (e.g. of a page-locked torch tensor)."""
        if isinstance(host_ptr, np.ndarray):
            assert host_ptr.dtype == np.float64 and host_ptr.flags.c_contiguous
            assert host_ptr.nbytes == self.sc_state_bytes(ghosted_level0)
            host_ptr = host_ptr.ctypes.data
        _check(lib().sc_set_state(self.ctx, ctypes.c_void_p(host_ptr), 1 if ghosted_level0 else 0))

    def sc_get_state(self, host_ptr=None, ghosted_level0: bool = False):
        """Whole state into a packed host buffer (allocated when None)."""
        out = None
        if host_ptr is None:
            out = np.empty(self.sc_state_bytes(ghosted_level0) // 8)
            host_ptr = out.ctypes.data
        elif isinstance(host_ptr, np.ndarray):
            assert host_ptr.dtype == np.float64 and host_ptr.flags.c_contiguous
            assert host_ptr.nbytes == self.sc_state_bytes(ghosted_level0)
            out, host_ptr = host_ptr, host_ptr.ctypes.data
        _check(lib().sc_get_state(self.ctx, ctypes.c_void_p(host_ptr), 1 if ghosted_level0 else 0))
        return out

    def sc_set_transfer_mode(self, mode: int):
        """SC_XFER_AUTO (direct for page-locked host memory), SC_XFER_STAGED or SC_XFER_DIRECT."""
        _check(lib().sc_set_transfer_mode(self.ctx, int(mode)))

    def sc_transfer_stats(self) -> dict:
        """Split timing of the last sc_set_state / sc_get_state (CUDA events)."""
        c, k = ctypes.c_double(), ctypes.c_double()
        n, d = ctypes.c_size_t(), ctypes.c_int()
        _check(lib().sc_transfer_stats(self.ctx, ctypes.byref(c), ctypes.byref(k), ctypes.byref(n), ctypes.byref(d)))
        return {"copy_ms": c.value, "kernel_ms": k.value, "bytes": n.value, "direct": bool(d.value)}

    def sc_advance(self, n: int):
        _check(lib().sc_advance(self.ctx, n))

    def sc_synchronize(self):
        """Wait for the context's stream; raises SubcycError with SC_ENONFINITE
        when the per-step finiteness check found a non-finite value."""
        _check(lib().sc_synchronize(self.ctx))

    def sc_synchronize_timeout(self, timeout_s: float):
        """As sc_synchronize with a bounded wait (SC_ETIMEOUT when it runs out)."""
        _check(lib().sc_synchronize_timeout(self.ctx, float(timeout_s)))

    def sc_get_constraints(self, level, box) -> np.ndarray:
        a = np.empty((NCONSTRAINTS,) + self.shape(level, box))
        _check(lib().sc_get_constraints(self.ctx, level, box, _dp(a)))
        return a

    def sc_get_time(self) -> float:
        t = ctypes.c_double()
        _check(lib().sc_get_time(self.ctx, ctypes.byref(t)))
        return t.value

    def sc_zone_updates(self) -> Tuple[float, float]:
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(lib().sc_zone_updates(self.ctx, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def sc_launches_per_step(self) -> int:
        n = ctypes.c_long()
        _check(lib().sc_launches_per_step(self.ctx, ctypes.byref(n)))
        return n.value

    def sc_footprint(self) -> int:
        n = ctypes.c_size_t()
        _check(lib().sc_footprint(self.ctx, ctypes.byref(n)))
        return n.value

    def sc_autotune(self) -> Tuple[Tuple[int, int, int], float]:
        t = (ctypes.c_int * 3)()
        ms = ctypes.c_double()
        _check(lib().sc_autotune(self.ctx, t, ctypes.byref(ms)))
        return (t[0], t[1], t[2]), ms.value

    def sc_get_tuning(self) -> dict:
        """Tile shape, Z4c derivative form (0 two kernels, 1 one kernel) and stage blocks per SM in effect."""
        t = (ctypes.c_int * 3)()
        f, b = ctypes.c_int(), ctypes.c_int()
        _check(lib().sc_get_tuning(self.ctx, t, ctypes.byref(f), ctypes.byref(b)))
        return {"tile": (t[0], t[1], t[2]), "deriv_form": f.value, "stage_blocks_per_sm": b.value}

    def sc_set_tuning(self, tile, deriv_form: int = 0, stage_blocks_per_sm: int = 3):
        t = (ctypes.c_int * 3)(*[int(v) for v in tile])
        _check(lib().sc_set_tuning(self.ctx, t, int(deriv_form), int(stage_blocks_per_sm)))

    def sc_check_finite(self) -> bool:
        """True if the evolved state is finite everywhere (device scan)."""
        rc = lib().sc_check_finite(self.ctx)
        if rc == SC_ENONFINITE:
            return False
        _check(rc)
        return True

    def sc_regrid(self, boxes):
        """New boxes for every level (level 0 unchanged); updates self.h."""
        nb = (ctypes.c_int * len(boxes))(*[len(b) for b in boxes])
        flat = [bx for lvl in boxes for bx in lvl]
        arr = (sc_box * len(flat))()
        for i, (lo, hi) in enumerate(flat):
            arr[i].lo[:] = list(lo)
            arr[i].hi[:] = list(hi)
        _check(lib().sc_regrid(self.ctx, nb, arr))
        import copy
        h = copy.copy(self.h)
        h.boxes = [[(tuple(lo), tuple(hi)) for lo, hi in lvl] for lvl in boxes]
        self.h = h

    def sc_interpolate(self, points, field: int) -> np.ndarray:
        p = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
        out = np.empty(len(p))
        _check(lib().sc_interpolate(self.ctx, len(p), _dp(p), field, _dp(out)))
        return out

    # the same names as the oracle's, so one driver can move either
    def regrid(self, boxes):
        self.sc_regrid(boxes)

    def interpolate(self, points, field):
        return self.sc_interpolate(points, field)

    def advance(self, n):
        self.sc_advance(n)

    def sc_debug_get_vector(self, level: int, box: int, vec: int, field: int, ghosted: bool = False) -> np.ndarray:
        a = np.empty(self.shape(level, box, ghosted))
        _check(lib().sc_debug_get_vector(self.ctx, level, box, vec, field, 1 if ghosted else 0, _dp(a)))
        return a

    def sc_time_ghost_kernels(self, level: int, nrep: int = 5):
        ms = np.zeros(2)
        cnt = (ctypes.c_long * 4)()
        _check(lib().sc_time_ghost_kernels(self.ctx, level, nrep, _dp(ms), cnt))
        return float(ms[0]), float(ms[1]), (cnt[0], cnt[1], cnt[2], cnt[3])

    def sc_time_stage_kernels(self, level: int, nrep: int = 5) -> Tuple[float, float]:
        ms = np.zeros(2)
        _check(lib().sc_time_stage_kernels(self.ctx, level, nrep, _dp(ms)))
        return float(ms[0]), float(ms[1])

    def sc_run_op_class_pass(self, level: int) -> None:
        _check(lib().sc_run_op_class_pass(self.ctx, level))

    # convenience
    def set_initial_data_from(self, h=None):
        h = h or self.h
        self.sc_set_initial_data(h.id_kind, h.id_params)

    def get_all(self, ghosted=False) -> List[List[np.ndarray]]:
        """[level][box] -> array (F, nz, ny, nx)."""
        return [[np.stack([self.sc_get_field(l, b, f, ghosted) for f in range(self.F)])
                 for b in range(len(self.h.boxes[l]))] for l in range(self.h.nlevels)]


class Server:
    """Continuous-batching server of independent evolutions (wraps ``sc_server*``).

    Requests are admitted in arrival order as slots and device memory free up,
    each on its own stream; every ``sc_server_tick`` launches the next coarse
    step of every active request.  Results are bitwise independent of the mix.
    """

    def __init__(self, hbm_budget_bytes: int, max_active: int = 16, depth: int = 2):
        srv = ctypes.c_void_p()
        _check(lib().sc_server_create(int(hbm_budget_bytes), int(max_active), int(depth), ctypes.byref(srv)))
        self.srv = srv
        self.hier = {}

    def close(self):
        if getattr(self, "srv", None):
            lib().sc_server_destroy(self.srv)
            self.srv = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sc_server_submit(self, h, n_coarse_steps: int, exec_mode: int = SC_EXEC_GRAPH) -> int:
        d, keep = make_desc(h, exec_mode=exec_mode)
        p = np.ascontiguousarray(h.id_params, dtype=np.float64)
        t = ctypes.c_ulonglong()
        _check(lib().sc_server_submit(self.srv, ctypes.byref(d), h.id_kind, _dp(p) if len(p) else None, len(p),
                                      int(n_coarse_steps), ctypes.byref(t)))
        self.hier[t.value] = h
        return t.value

    def sc_server_tick(self) -> Tuple[int, int, int]:
        a, q, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().sc_server_tick(self.srv, ctypes.byref(a), ctypes.byref(q), ctypes.byref(n)))
        return a.value, q.value, n.value

    def sc_server_poll(self, ticket: int) -> Tuple[bool, float]:
        d, lat = ctypes.c_int(), ctypes.c_double()
        _check(lib().sc_server_poll(self.srv, ticket, ctypes.byref(d), ctypes.byref(lat)))
        return bool(d.value), lat.value

    def sc_server_wait(self, ticket: int, timeout_s: float) -> float:
        """Tick until the request is done (its latency) or raise SC_ETIMEOUT."""
        lat = ctypes.c_double()
        _check(lib().sc_server_wait(self.srv, ticket, float(timeout_s), ctypes.byref(lat)))
        return lat.value

    def sc_server_set_merge(self, on: bool):
        """Merge scalar-wave requests into one persistent launch per tick (default off)."""
        _check(lib().sc_server_set_merge(self.srv, 1 if on else 0))

    def sc_server_inject_alloc_failure(self, k: int):
        _check(lib().sc_server_inject_alloc_failure(self.srv, int(k)))

    def sc_server_read(self, ticket: int, level: int, box: int, field: int) -> np.ndarray:
        h = self.hier[ticket]
        lo, hi = h.boxes[level][box]
        a = np.empty((hi[2] - lo[2] + 1, hi[1] - lo[1] + 1, hi[0] - lo[0] + 1))
        _check(lib().sc_server_read(self.srv, ticket, level, box, field, _dp(a)))
        return a

    def sc_server_release(self, ticket: int):
        _check(lib().sc_server_release(self.srv, ticket))
        self.hier.pop(ticket, None)

    def sc_server_stats(self) -> dict:
        f, a = ctypes.c_double(), ctypes.c_double()
        n, b = ctypes.c_long(), ctypes.c_size_t()
        _check(lib().sc_server_stats(self.srv, ctypes.byref(f), ctypes.byref(a), ctypes.byref(n), ctypes.byref(b)))
        return {"zu_finest": f.value, "zu_actual": a.value, "launches": n.value, "bytes_in_use": b.value}

    def run_until_done(self, tickets, timeout_s: float = 600.0, on_done=None):
        """Tick until every ticket has finished; on_done(ticket) is called once
        per finished request (a client reads and releases it there, so its
        memory returns to the budget).  Raises if nothing can progress (queued
        requests blocked by finished requests that were never released) or if
        timeout_s passes."""
        import time
        t0 = time.perf_counter()
        pending = set(tickets)
        while pending:
            active, queued, launched = self.sc_server_tick()
            for t in list(pending):
                if self.sc_server_poll(t)[0]:
                    pending.discard(t)
                    if on_done is not None:
                        on_done(t)
            if pending and active == 0 and queued > 0 and launched == 0:
                self.sc_server_tick()
                active, queued, launched = self.sc_server_tick()
                if active == 0 and launched == 0:
                    raise SubcycError(SC_EBUSY, "server stalled: queued requests wait for memory held by "
                                                "finished requests that were not released")
            if time.perf_counter() - t0 > timeout_s:
                raise SubcycError(SC_ETIMEOUT, f"requests not finished after {timeout_s} s")
