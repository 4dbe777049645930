"""Python binding of libsphst, the GB300 pair-sweep library for the
Riemann-based multiphase SPH scheme with surface stress and the
zero-surface-energy penalty (arXiv 2503.16082).

Argument marshalling only: every step of the method runs in the CUDA
library.  Names follow the C ABI in include/sphst.h without the ``sphst_``
prefix.  There is no CPU fallback: if the library cannot be built or loaded,
importing a function that needs it raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional, Sequence

import numpy as np

from . import build as _build

OK = 0
ERR_INVALID_ARG, ERR_STATE, ERR_UNSUPPORTED, ERR_OOM, ERR_CUDA = -1, -2, -3, -4, -5
ERR_NONFINITE, ERR_TIMEOUT, ERR_OVER_BUDGET, ERR_DOMAIN = -6, -7, -8, -9
ERR_COINCIDENT, ERR_STALLED, ERR_CAPACITY, ERR_NEIGHBORS = -10, -11, -12, -13
NBR_LIST, NBR_CELLS = 0, 1
FLUID, WALL = 0, 1
LIMITER_DENSITY, LIMITER_NONE, LIMITER_ZERO, LIMITER_PRINTED = 0, 1, 2, 3
GRAD_COMMON, GRAD_PRINTED = 0, 1
PENALTY_NN, PENALTY_EE, PENALTY_SCALAR = 0, 1, 2
PENALTY_SCOPE_BOTH, PENALTY_SCOPE_CROSS_ONLY = 0, 1
WALL_MIRROR, WALL_NO_SUCTION = 0, 1
STRESS_PRINTED, STRESS_OWN = 0, 1
SURFACE_CORR_PRINTED, SURFACE_CORR_OWN_FLUID = 0, 1
# one engine with neighbour lists holds at most 2^26 particles (a list entry
# is j << 6 | cell code in 32 bits; sphst_batch_step rejects more)
MAX_LIST_ENGINE_PARTICLES = 1 << 26
VSTAR_CORRECTED, VSTAR_PRINTED = 0, 1
LOOP_GRAPH, LOOP_HOST = 0, 1
FIELD_POS, FIELD_VEL, FIELD_RHO, FIELD_PRESSURE, FIELD_PHASE, FIELD_GRADC, FIELD_ACC_VISC = range(7)
VECTOR_FIELDS = (FIELD_POS, FIELD_VEL, FIELD_GRADC, FIELD_ACC_VISC)


class CaseParams(C.Structure):
    _fields_ = [("dim", C.c_int32), ("precision", C.c_int32), ("dx", C.c_double),
                ("h_factor", C.c_double), ("c0", C.c_double), ("gamma", C.c_double),
                ("xi", C.c_double), ("tvf_alpha", C.c_double), ("limiter", C.c_int32),
                ("grad_mode", C.c_int32), ("penalty_form", C.c_int32), ("loop_mode", C.c_int32),
                ("grid_pad", C.c_int32), ("block", C.c_int32), ("max_substeps", C.c_int64),
                ("cfl_ad", C.c_double), ("cfl_ac", C.c_double),
                ("nbr_mode", C.c_int32), ("max_neighbors", C.c_int32),
                ("periodic", C.c_int32), ("vstar_form", C.c_int32),
                ("period_lo", C.c_double * 3), ("period_hi", C.c_double * 3),
                ("lanes", C.c_int32), ("penalty_scope", C.c_int32), ("wall_form", C.c_int32),
                ("work_lists", C.c_int32), ("stress_weights", C.c_int32), ("surface_corr", C.c_int32)]


class PhaseProps(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad_", C.c_int32), ("rho0", C.c_double),
                ("eta", C.c_double), ("wall_vel", C.c_double * 3)]


class StepInfo(C.Structure):
    _fields_ = [("n_adv", C.c_int64), ("n_sub", C.c_int64), ("t", C.c_double),
                ("last_dt_ad", C.c_double), ("last_dt_ac", C.c_double),
                ("status", C.c_int32), ("pad_", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad_"}


class Diagnostics(C.Structure):
    _fields_ = [("momentum", C.c_double * 3), ("kinetic", C.c_double), ("count", C.c_int64 * 2),
                ("first", C.c_double * 3), ("second", C.c_double * 6), ("p_in", C.c_double),
                ("p_out", C.c_double), ("n_in", C.c_int64), ("n_out", C.c_int64),
                ("n_nonfinite", C.c_int64)]

    def as_dict(self):
        out = {}
        for f, _ in self._fields_:
            v = getattr(self, f)
            out[f] = list(v) if hasattr(v, "__len__") else v
        return out


class SphstError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sphst error {code}: {msg}")
        self.code = code


EXPORTS = {
    "sphst_default_params": (None, [C.POINTER(CaseParams)]),
    "sphst_create_case": (C.c_int, [C.POINTER(CaseParams), C.POINTER(C.c_void_p)]),
    "sphst_add_phase_particles": (C.c_int, [C.c_void_p, C.POINTER(PhaseProps), C.c_int64,
                                            C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.POINTER(C.c_int32)]),
    "sphst_step": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(StepInfo)]),
    "sphst_read_fields": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64]),
    "sphst_case_info": (C.c_int, [C.c_void_p, C.POINTER(StepInfo)]),
    "sphst_num_particles": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "sphst_destroy": (C.c_int, [C.c_void_p]),
    "sphst_last_error": (C.c_char_p, []),
    "sphst_debug_grid": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    "sphst_debug_keys": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]),
    "sphst_debug_neighbor_counts": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "sphst_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sphst_profile_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "sphst_cell_order_noalloc": (C.c_int, [C.c_int32, C.c_int64, C.c_void_p, C.c_void_p, C.c_double,
                                           C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sphst_batch_create": (C.c_int, [C.c_int32, C.POINTER(C.c_void_p)]),
    "sphst_batch_add": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sphst_batch_remove": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sphst_batch_step": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(StepInfo)]),
    "sphst_batch_size": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "sphst_batch_destroy": (C.c_int, [C.c_void_p]),
    "sphst_footprint_bytes": (C.c_int, [C.POINTER(CaseParams), C.c_int64, C.POINTER(C.c_int64)]),
    "sphst_diagnose": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.POINTER(Diagnostics)]),
    "sphst_fma_peak": (C.c_int, [C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "sphst_device_info": (C.c_int, [C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                     C.POINTER(C.c_int32)]),
    "sphst_struct_sizes": (C.c_int, [C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
}

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load():
    """Load libsphst (building it with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            lib = C.CDLL(path)
            for name, (res, args) in EXPORTS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            sizes = [C.c_int64() for _ in range(3)]
            lib.sphst_struct_sizes(*[C.byref(v) for v in sizes])
            want = [C.sizeof(CaseParams), C.sizeof(PhaseProps), C.sizeof(StepInfo)]
            if [v.value for v in sizes] != want:
                raise RuntimeError(f"libsphst structure sizes {[v.value for v in sizes]} differ from the "
                                   f"binding's {want}: rebuild the library")
            _lib = lib
    return _lib


def last_error() -> str:
    return load().sphst_last_error().decode()


def _check(rc: int, what: str):
    if rc != OK:
        raise SphstError(rc, f"{what}: {last_error()}")
    return rc


def default_params(**kw) -> CaseParams:
    p = CaseParams()
    load().sphst_default_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def create_case(params: CaseParams) -> C.c_void_p:
    h = C.c_void_p()
    _check(load().sphst_create_case(C.byref(params), C.byref(h)), "create_case")
    return h


def add_phase_particles(case, kind: int, pos: np.ndarray, rho0: float = 0.0, eta: float = 0.0,
                        vel: Optional[np.ndarray] = None, rho: Optional[np.ndarray] = None,
                        wall_vel: Sequence[float] = (0.0, 0.0, 0.0)) -> int:
    props = PhaseProps()
    props.kind, props.rho0, props.eta = kind, rho0, eta
    for a in range(3):
        props.wall_vel[a] = float(wall_vel[a]) if a < len(wall_vel) else 0.0
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    vel = None if vel is None else np.ascontiguousarray(vel, dtype=np.float64)
    rho = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
    pid = C.c_int32(-1)
    _check(load().sphst_add_phase_particles(
        case, C.byref(props), len(pos), pos.ctypes.data,
        None if vel is None else vel.ctypes.data, None if rho is None else rho.ctypes.data,
        C.byref(pid)), "add_phase_particles")
    return pid.value


def step(case, n_adv: int, check: bool = True) -> dict:
    info = StepInfo()
    rc = load().sphst_step(case, n_adv, C.byref(info))
    if check:
        _check(rc, "step")
    d = info.as_dict()
    d["rc"] = rc
    return d


def case_info(case) -> dict:
    info = StepInfo()
    _check(load().sphst_case_info(case, C.byref(info)), "case_info")
    return info.as_dict()


def num_particles(case):
    a, b = C.c_int64(), C.c_int64()
    _check(load().sphst_num_particles(case, C.byref(a), C.byref(b)), "num_particles")
    return a.value, b.value


def read_fields(case, field: int, dim: int, out: Optional[np.ndarray] = None) -> np.ndarray:
    """FP64 field in insertion order, (n, dim) for vectors.  `out`, if given,
    is a C-contiguous float64 array of at least n * width elements that
    receives it (for example a view of pinned host memory, which the
    device-to-host copy reads faster than pageable memory)."""
    n, _ = num_particles(case)
    w = dim if field in VECTOR_FIELDS else 1
    if out is None:
        buf = np.empty(n * w, dtype=np.float64)
    else:
        if out.dtype != np.float64 or not out.flags["C_CONTIGUOUS"] or out.size < n * w:
            raise ValueError("out must be a C-contiguous float64 array of at least n * width elements")
        buf = out.reshape(-1)[: n * w]
    _check(load().sphst_read_fields(case, field, buf.ctypes.data, buf.size), "read_fields")
    return buf.reshape(n, w) if w > 1 else buf


def destroy(case) -> None:
    _check(load().sphst_destroy(case), "destroy")


def debug_grid(case):
    origin = np.zeros(3)
    cs = C.c_double()
    ncell = np.zeros(3, dtype=np.int32)
    _check(load().sphst_debug_grid(case, origin.ctypes.data, C.byref(cs), ncell.ctypes.data), "debug_grid")
    return origin, cs.value, ncell


def debug_keys(case):
    n, _ = num_particles(case)
    keys = np.zeros(max(n, 1), dtype=np.uint64)
    ids = np.zeros(max(n, 1), dtype=np.int64)
    _check(load().sphst_debug_keys(case, keys.ctypes.data, ids.ctypes.data, n), "debug_keys")
    return keys[:n], ids[:n]


def debug_neighbor_counts(case):
    n, _ = num_particles(case)
    cnt = np.zeros(max(n, 1), dtype=np.int32)
    _check(load().sphst_debug_neighbor_counts(case, cnt.ctypes.data, n), "debug_neighbor_counts")
    return cnt[:n]


def diagnose(case, center=(0.0, 0.0, 0.0), r_in: float = 0.0, r_out: float = float("inf")) -> dict:
    """FP64 device reductions of a case (sphst_diagnose): momentum, kinetic
    energy, phase counts, phase-0 first and second moments, Laplace sampling
    sums around `center`, non-finite count."""
    c = np.zeros(3, dtype=np.float64)
    c[:len(center)] = center
    out = Diagnostics()
    _check(load().sphst_diagnose(case, c.ctypes.data, float(r_in), float(r_out), C.byref(out)), "diagnose")
    return out.as_dict()


def fma_peak(precision: int = 32) -> dict:
    """Measured FMA throughput of the GPU (sphst_fma_peak)."""
    tf, ms = C.c_double(0.0), C.c_double(0.0)
    _check(load().sphst_fma_peak(precision, C.byref(tf), C.byref(ms)), "fma_peak")
    return {"tflops": tf.value, "kernel_ms": ms.value}


def device_info() -> dict:
    """SM count, peak SM clock and compute capability of the current GPU
    (sphst_device_info)."""
    v = [C.c_int32(0) for _ in range(4)]
    _check(load().sphst_device_info(*[C.byref(x) for x in v]), "device_info")
    return {"sm_count": v[0].value, "max_sm_clock_khz": v[1].value, "cc": (v[2].value, v[3].value)}


PROFILE_GROUPS = ("rebuild", "setup", "criterion", "sweep_A", "sweep_B", "sweep_C", "sweep_S")


def set_stream(case, cuda_stream: int) -> None:
    _check(load().sphst_set_stream(case, C.c_void_p(cuda_stream)), "set_stream")


def profile_step(case) -> dict:
    """One advection step with per-kernel-group CUDA-event timing:
    {group: (milliseconds, launches)}."""
    ms = np.zeros(len(PROFILE_GROUPS))
    nl = np.zeros(len(PROFILE_GROUPS), dtype=np.int64)
    _check(load().sphst_profile_step(case, ms.ctypes.data, nl.ctypes.data), "profile_step")
    return {g: (float(ms[k]), int(nl[k])) for k, g in enumerate(PROFILE_GROUPS)}


def cell_order_noalloc(dim: int, n: int, pos_dev_ptr: int, origin, cell_size: float, ncell,
                       keys_dev_ptr: int, order_dev_ptr: int, cuda_stream: int = 0) -> None:
    """Canonical cell order of n particles already on the device, computed
    without any device allocation (all buffers are the caller's; the
    library's fixed scratch array holds the intermediates).  Arguments are
    raw device pointers, e.g. ``tensor.data_ptr()``; origin and ncell have
    `dim` or 3 entries (a 2D grid is padded to 3)."""
    def three(v, dtype, pad):
        v = np.asarray(v, dtype=dtype).reshape(-1)
        if len(v) not in (dim, 3):
            raise ValueError(f"origin and ncell need {dim} or 3 entries, got {len(v)}")
        return np.ascontiguousarray(np.concatenate([v, np.full(3 - len(v), pad, dtype=dtype)]))
    origin = three(origin, np.float64, 0.0)
    ncell = three(ncell, np.int32, 1)
    _check(load().sphst_cell_order_noalloc(dim, n, C.c_void_p(pos_dev_ptr), origin.ctypes.data,
                                           cell_size, ncell.ctypes.data, C.c_void_p(keys_dev_ptr),
                                           C.c_void_p(order_dev_ptr), C.c_void_p(cuda_stream)),
           "cell_order_noalloc")


def batch_create(precision: int = 32):
    h = C.c_void_p()
    _check(load().sphst_batch_create(precision, C.byref(h)), "batch_create")
    return h


def batch_add(batch, case) -> None:
    _check(load().sphst_batch_add(batch, case), "batch_add")


def batch_remove(batch, case) -> None:
    _check(load().sphst_batch_remove(batch, case), "batch_remove")


def batch_step(batch, n_adv: int) -> dict:
    info = StepInfo()
    _check(load().sphst_batch_step(batch, n_adv, C.byref(info)), "batch_step")
    return info.as_dict()


def batch_size(batch) -> int:
    n = C.c_int64()
    _check(load().sphst_batch_size(batch, C.byref(n)), "batch_size")
    return n.value


def batch_destroy(batch) -> None:
    _check(load().sphst_batch_destroy(batch), "batch_destroy")


def footprint_bytes(params: CaseParams, n: int) -> int:
    out = C.c_int64()
    _check(load().sphst_footprint_bytes(C.byref(params), n, C.byref(out)), "footprint_bytes")
    return out.value


# --------------------------------------------------------------------------
# convenience: a whole problem statement from a seeded case description
# --------------------------------------------------------------------------
def params_from_spec(spec, precision: int = 32, **params) -> CaseParams:
    """The case parameters of a ``sphcases.Case``-like object (fields dim,
    dx, h_factor, c0, gamma, xi, optional periodic and cfl_ac), with
    ``params`` overriding fields of the result."""
    p = default_params(dim=spec.dim, precision=precision, dx=spec.dx, h_factor=spec.h_factor,
                       c0=spec.c0, gamma=spec.gamma, xi=spec.xi,
                       cfl_ac=getattr(spec, "cfl_ac", 0.6))
    if getattr(spec, "periodic", 0):
        p.periodic = spec.periodic
        for a in range(spec.dim):
            p.period_lo[a], p.period_hi[a] = spec.lo[a], spec.hi[a]
    for k, v in params.items():
        setattr(p, k, v)
    return p


def case_from_spec(spec, precision: int = 32, **params):
    """Create and fill a case from a ``sphcases.Case``-like object (the
    fields of ``params_from_spec`` and phases with kind/pos/rho0/eta/vel/
    rho/wall_vel).  Returns the handle."""
    h = create_case(params_from_spec(spec, precision, **params))
    try:
        for ph in spec.phases:
            if ph.kind == "fluid":
                add_phase_particles(h, FLUID, ph.pos, rho0=ph.rho0, eta=ph.eta, vel=ph.vel, rho=ph.rho)
            else:
                add_phase_particles(h, WALL, ph.pos, wall_vel=ph.wall_vel)
    except Exception:
        destroy(h)
        raise
    return h
