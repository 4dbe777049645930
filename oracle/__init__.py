"""FP64 CPU oracle of the Riemann multiphase SPH scheme (arXiv 2503.16082).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it; the product path never does.  The
arithmetic lives in ``sph_oracle.c`` (plain C, FP64, OpenMP over particles);
this module only builds it with gcc and marshals numpy arrays through ctypes.

``SPH_ORACLE_LIB`` may name a separately built library of the same source;
the pin-strength test uses it to load copies with planted mistakes.

Pins (see the header of ``sph_oracle.c``): every term of Eq. 33 for a
single pair, the cross-phase line by an isolated pair of different fluids and
the same-phase line by three pairs that reduce by hand (``ora_surface_pair``,
the routine the force loop calls); the integrator and the wall's mirror
pressure and volume by acoustic modes, v* = v_w at a wall by the water hammer,
the wall's dissipative term by a fluid particle beside one wall particle.  No
single term is unpinned; the scheme as a whole over many substeps is checked
through its integral observables (Laplace jump, oscillation periods).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsph_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [("dim", C.c_int32), ("limiter", C.c_int32), ("grad_mode", C.c_int32),
                ("nbr_mode", C.c_int32), ("n_threads", C.c_int32), ("penalty_form", C.c_int32),
                ("dx", C.c_double), ("h", C.c_double), ("c0", C.c_double),
                ("gamma", C.c_double), ("xi", C.c_double),
                ("rho0", C.c_double * 2), ("eta", C.c_double * 2),
                ("nhat_eps", C.c_double), ("max_substeps", C.c_int64),
                ("tvf_alpha", C.c_double), ("cfl_ad", C.c_double), ("cfl_ac", C.c_double),
                ("periodic", C.c_int32), ("pad2_", C.c_int32),
                ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3),
                ("vstar_form", C.c_int32), ("penalty_scope", C.c_int32), ("wall_form", C.c_int32),
                ("stress_weights", C.c_int32), ("surface_corr", C.c_int32), ("pad4_", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("n_adv", C.c_int64), ("n_sub", C.c_int64), ("t", C.c_double),
                ("last_dt_ad", C.c_double), ("last_dt_ac", C.c_double),
                ("status", C.c_int32), ("pad_", C.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # SPH_ORACLE_LIB: a separately built library of the same source
            # (the pin-strength test loads deliberately broken copies)
            path = os.environ.get("SPH_ORACLE_LIB") or build()
            lib = C.CDLL(path)
            P = C.POINTER
            d, i32, i64 = C.c_double, C.c_int32, C.c_int64
            dp, ip, lp = P(C.c_double), P(C.c_int32), P(C.c_int64)
            lib.ora_kernel_W.restype = d
            lib.ora_kernel_W.argtypes = [i32, d, d]
            lib.ora_kernel_dW.restype = d
            lib.ora_kernel_dW.argtypes = [i32, d, d]
            lib.ora_xi.restype = d
            lib.ora_xi.argtypes = [P(Params)]
            lib.ora_neighbors.restype = i64
            lib.ora_neighbors.argtypes = [P(Params), i64, dp, ip, ip, i64]
            lib.ora_grid.restype = None
            lib.ora_grid.argtypes = [P(Params), i64, dp, i32, dp, dp, ip]
            lib.ora_cell_keys.restype = i64
            lib.ora_cell_keys.argtypes = [P(Params), i64, dp, dp, d, ip,
                                          P(C.c_uint64), ip, lp]
            lib.ora_riemann_pair.restype = None
            lib.ora_riemann_pair.argtypes = [P(Params), d, d, dp, d, d, dp, dp, dp]
            lib.ora_surface_pair_apply.restype = None
            lib.ora_surface_pair_apply.argtypes = [P(Params), i32, i32, dp, dp, dp, d, dp, dp]
            lib.ora_surface_pair.restype = None
            lib.ora_surface_pair.argtypes = [P(Params), i32, i32, dp, dp, dp, d, dp]
            lib.ora_dt_advection.restype = d
            lib.ora_dt_advection.argtypes = [P(Params), dp, ip]
            lib.ora_dt_acoustic.restype = d
            lib.ora_dt_acoustic.argtypes = [P(Params), dp, ip]
            lib.ora_correction_matrices.restype = C.c_int
            lib.ora_correction_matrices.argtypes = [P(Params), i64, dp, dp, dp, ip, dp, dp]
            lib.ora_forces.restype = C.c_int
            lib.ora_forces.argtypes = [P(Params), i64, dp, dp, dp, ip, dp, dp, dp, dp, dp, dp]
            lib.ora_run.restype = C.c_int
            lib.ora_run.argtypes = [P(Params), i64, dp, dp, dp, ip, i64, P(Info), dp, dp]
            lib.ora_max_threads.restype = i32
            lib.ora_max_threads.argtypes = []
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def make_params(dim: int, dx: float, h: float, c0: float, gamma: float,
                rho0=(1.0, 1.0), eta=(1.0, 1.0), xi: float = -1.0,
                limiter: int = 0, grad_mode: int = 0, nbr_mode: Optional[int] = None,
                n: int = 0, n_threads: int = 0, nhat_eps: float = 1e-4,
                max_substeps: int = 0, tvf_alpha: float = 0.2,
                penalty_form: int = 0, cfl_ad: float = 0.1, cfl_ac: float = 0.6,
                periodic: int = 0, box_lo=(0.0, 0.0, 0.0), box_hi=(0.0, 0.0, 0.0),
                vstar_form: int = 0, penalty_scope: int = 0, wall_form: int = 0,
                stress_weights: int = 0, surface_corr: int = 0) -> Params:
    """Build a parameter block.  nbr_mode None: brute force below 4096
    particles, uniform grid above."""
    p = Params()
    p.dim, p.limiter, p.grad_mode = dim, limiter, grad_mode
    p.nbr_mode = (0 if n <= 4096 else 1) if nbr_mode is None else nbr_mode
    p.n_threads = n_threads
    p.dx, p.h, p.c0, p.gamma, p.xi = dx, h, c0, gamma, xi
    p.rho0[0], p.rho0[1] = rho0
    p.eta[0], p.eta[1] = eta
    p.nhat_eps = nhat_eps
    p.max_substeps = max_substeps
    p.tvf_alpha = tvf_alpha
    p.penalty_form = penalty_form
    p.cfl_ad, p.cfl_ac = cfl_ad, cfl_ac
    p.periodic = periodic
    p.vstar_form = vstar_form
    p.penalty_scope = penalty_scope
    p.wall_form = wall_form
    p.stress_weights = stress_weights
    p.surface_corr = surface_corr
    for a in range(3):
        p.box_lo[a], p.box_hi[a] = box_lo[a], box_hi[a]
    return p


def params_for_case(case, **kw) -> Params:
    """Parameters of a ``sphcases.Case`` (h = h_factor * dx)."""
    rho0, eta = case.fluid_props()
    kw.setdefault("xi", case.xi)
    kw.setdefault("cfl_ac", getattr(case, "cfl_ac", 0.6))
    if getattr(case, "periodic", 0):
        kw.setdefault("periodic", case.periodic)
        kw.setdefault("box_lo", tuple(case.lo) + (0.0,) * (3 - len(case.lo)))
        kw.setdefault("box_hi", tuple(case.hi) + (0.0,) * (3 - len(case.hi)))
    return make_params(case.dim, case.dx, case.h_factor * case.dx, case.c0,
                       case.gamma, rho0=tuple(rho0), eta=tuple(eta), n=case.n, **kw)


def kernel_W(dim: int, h: float, r: float) -> float:
    return _load().ora_kernel_W(dim, h, r)


def kernel_dW(dim: int, h: float, r: float) -> float:
    return _load().ora_kernel_dW(dim, h, r)


def xi(params: Params) -> float:
    return _load().ora_xi(C.byref(params))


def neighbors(params: Params, pos: np.ndarray):
    """CSR neighbour lists (counts, idx) of positions (n, 3)."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n = len(pos)
    counts = np.zeros(max(n, 1), dtype=np.int32)
    tot = lib.ora_neighbors(C.byref(params), n, _dp(pos), _ip(counts), None, 0)
    if tot < 0:
        raise ValueError("coincident particles")
    idx = np.zeros(max(tot, 1), dtype=np.int32)
    lib.ora_neighbors(C.byref(params), n, _dp(pos), _ip(counts), _ip(idx), tot)
    return counts[:n], idx[:tot]


def grid(params: Params, pos: np.ndarray, pad: int = 2):
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    origin = np.zeros(3)
    cs = C.c_double(0.0)
    ncell = np.zeros(3, dtype=np.int32)
    lib.ora_grid(C.byref(params), len(pos), _dp(pos), pad, _dp(origin), C.byref(cs), _ip(ncell))
    return origin, cs.value, ncell


def cell_keys(params: Params, pos: np.ndarray, origin, cs: float, ncell):
    """Morton keys, cell coordinates and canonical order (key, insertion id)."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n = len(pos)
    origin = np.ascontiguousarray(origin, dtype=np.float64)
    ncell = np.ascontiguousarray(ncell, dtype=np.int32)
    keys = np.zeros(max(n, 1), dtype=np.uint64)
    cells = np.zeros((max(n, 1), 3), dtype=np.int32)
    order = np.zeros(max(n, 1), dtype=np.int64)
    out = lib.ora_cell_keys(C.byref(params), n, _dp(pos), _dp(origin), cs, _ip(ncell),
                            keys.ctypes.data_as(C.POINTER(C.c_uint64)), _ip(cells),
                            order.ctypes.data_as(C.POINTER(C.c_int64)))
    return keys[:n], cells[:n], order[:n], int(out)


def riemann_pair(params: Params, rho_i, p_i, v_i, rho_j, p_j, v_j, e):
    """(P*, U*, beta, pbar, v*) of one pair along unit vector e."""
    lib = _load()
    v_i = np.zeros(3) + np.pad(np.asarray(v_i, float), (0, 3 - len(v_i)))
    v_j = np.zeros(3) + np.pad(np.asarray(v_j, float), (0, 3 - len(v_j)))
    e = np.zeros(3) + np.pad(np.asarray(e, float), (0, 3 - len(e)))
    out = np.zeros(7)
    lib.ora_riemann_pair(C.byref(params), rho_i, p_i, _dp(v_i), rho_j, p_j, _dp(v_j),
                         _dp(e), _dp(out))
    return out[0], out[1], out[2], out[3], out[4:7].copy()


def surface_pair(params: Params, k_i: int, k_j: int, gradC_i, gradC_j, e, r: float) -> np.ndarray:
    """S_ij e_ij of Eq. 33 for one pair of fluid particles (phases k_i, k_j
    in {0, 1}) with colour gradients gradC_i, gradC_j, unit vector e_ij and
    distance r; the pair adds it times W'(r) V_j / rho_i to a^s_i."""
    lib = _load()
    three = lambda v: np.ascontiguousarray(np.pad(np.asarray(v, float), (0, 3 - len(v))))
    gi, gj, ee = three(gradC_i), three(gradC_j), three(e)
    out = np.zeros(3)
    lib.ora_surface_pair(C.byref(params), int(k_i), int(k_j), _dp(gi), _dp(gj), _dp(ee), float(r), _dp(out))
    return out[:params.dim].copy()


def surface_pair_apply(params: Params, k_i: int, k_j: int, gradC_i, gradC_j, e, r: float, v) -> np.ndarray:
    """The pair matrix S_ij of Eq. 33 (as in ``surface_pair``) applied to the
    vector v instead of e_ij."""
    lib = _load()
    three = lambda x: np.ascontiguousarray(np.pad(np.asarray(x, float), (0, 3 - len(x))))
    gi, gj, ee, vv = three(gradC_i), three(gradC_j), three(e), three(v)
    out = np.zeros(3)
    lib.ora_surface_pair_apply(C.byref(params), int(k_i), int(k_j), _dp(gi), _dp(gj), _dp(ee), float(r), _dp(vv),
                               _dp(out))
    return out[:params.dim].copy()


def dt_advection(params: Params, vmax, present=(1, 1)) -> float:
    v = np.asarray(vmax, dtype=np.float64)
    pr = np.asarray(present, dtype=np.int32)
    return _load().ora_dt_advection(C.byref(params), _dp(v), _ip(pr))


def dt_acoustic(params: Params, vmax, present=(1, 1)) -> float:
    v = np.asarray(vmax, dtype=np.float64)
    pr = np.asarray(present, dtype=np.int32)
    return _load().ora_dt_acoustic(C.byref(params), _dp(v), _ip(pr))


def forces(params: Params, pos, vel, rho, kind):
    """All right-hand sides at one state: dict of gradC, a_p, a_s, a_v, drho
    and the transport-velocity shift dr."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    vel = np.ascontiguousarray(vel, dtype=np.float64)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    kind = np.ascontiguousarray(kind, dtype=np.int32)
    n = len(pos)
    out = {k: np.zeros((n, 3)) for k in ("gradC", "a_p", "a_s", "a_v", "dr")}
    out["drho"] = np.zeros(n)
    st = lib.ora_forces(C.byref(params), n, _dp(pos), _dp(vel), _dp(rho), _ip(kind),
                        _dp(out["gradC"]), _dp(out["a_p"]), _dp(out["a_s"]),
                        _dp(out["a_v"]), _dp(out["drho"]), _dp(out["dr"]))
    if st != 0:
        raise ValueError(f"oracle status {st}")
    return out


def correction_matrices(params: Params, pos, vel, rho, kind):
    """Eq. 15's correction matrix of every particle, over all neighbours and
    over the neighbours of the particle's own fluid: two (n, 3, 3) arrays."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    vel = np.ascontiguousarray(vel, dtype=np.float64)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    kind = np.ascontiguousarray(kind, dtype=np.int32)
    n = len(pos)
    B = np.zeros((n, 9))
    Bk = np.zeros((n, 9))
    st = lib.ora_correction_matrices(C.byref(params), n, _dp(pos), _dp(vel), _dp(rho), _ip(kind), _dp(B), _dp(Bk))
    if st != 0:
        raise ValueError(f"oracle status {st}")
    return B.reshape(n, 3, 3), Bk.reshape(n, 3, 3)


def run(params: Params, pos, vel, rho, kind, n_adv: int):
    """Advance n_adv advection steps; returns (pos, vel, rho, info dict, gradC, a_v)."""
    lib = _load()
    pos = np.array(pos, dtype=np.float64, order="C", copy=True)
    vel = np.array(vel, dtype=np.float64, order="C", copy=True)
    rho = np.array(rho, dtype=np.float64, order="C", copy=True)
    kind = np.ascontiguousarray(kind, dtype=np.int32)
    n = len(pos)
    info = Info()
    gC = np.zeros((n, 3))
    av = np.zeros((n, 3))
    lib.ora_run(C.byref(params), n, _dp(pos), _dp(vel), _dp(rho), _ip(kind), n_adv,
                C.byref(info), _dp(gC), _dp(av))
    d = {f: getattr(info, f) for f, _ in Info._fields_ if f != "pad_"}
    return pos, vel, rho, d, gC, av


def run_case(case, n_adv: int, **kw):
    """Run a ``sphcases.Case`` for n_adv advection steps on the oracle."""
    pos, vel, rho, kind = case.flat()
    P = params_for_case(case, **kw)
    return run(P, pos, vel, rho, kind, n_adv)


def max_threads() -> int:
    return int(_load().ora_max_threads())
