"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bars (see the readings and tolerances documented with the library):
  * cell keys, canonical order and neighbour counts: bit-exact;
  * FP64 fields after one advection step (tens of acoustic substeps):
    max |gpu - oracle| <= 1e-12 * max |oracle| per field;
  * FP32 fields after one acoustic substep: <= 1e-5 * max |oracle|;
    after a whole advection step: <= 2e-4 (rounding of FP32 amplified
    through the substeps, see the derivation in the design notes).
Fields compared: displacement x - x0, velocity, density deviation rho - rho0,
colour gradient and viscous acceleration, fluid particles only.
"""
import numpy as np
import pytest

import oracle
import sphcases

pytestmark = pytest.mark.gpu

S = pytest.importorskip("paper_2503_16082_gb300")


def gpu_case(case, precision, **kw):
    return S.case_from_spec(case, precision=precision, **kw)


def run_both(case, precision, n_adv, ora_kw=None, **kw):
    h = gpu_case(case, precision, **kw)
    try:
        info = S.step(h, n_adv)
        g = {
            "pos": S.read_fields(h, S.FIELD_POS, case.dim),
            "vel": S.read_fields(h, S.FIELD_VEL, case.dim),
            "rho": S.read_fields(h, S.FIELD_RHO, case.dim),
            "gradC": S.read_fields(h, S.FIELD_GRADC, case.dim),
            "acc_visc": S.read_fields(h, S.FIELD_ACC_VISC, case.dim),
        }
    finally:
        S.destroy(h)
    pos, vel, rho, kind = case.flat()
    P = oracle.params_for_case(case, **(ora_kw or {}))
    p1, v1, r1, oinfo, gC, av = oracle.run(P, pos, vel, rho, kind, n_adv)
    d = case.dim
    o = {"pos": p1[:, :d], "vel": v1[:, :d], "rho": r1, "gradC": gC[:, :d], "acc_visc": av[:, :d]}
    return g, o, info, oinfo, pos[:, :d], kind


def rel_err(g, o, pos0, kind, key, case):
    fl = kind < 2
    a, b = g[key][fl], o[key][fl]
    if key == "pos":
        a, b = a - pos0[fl], b - pos0[fl]
    if key == "rho":
        rho0 = np.asarray(case.fluid_props()[0])[kind[fl]]
        a, b = a - rho0, b - rho0
    scale = np.abs(b).max()
    return np.abs(a - b).max() / scale if scale > 0 else np.abs(a - b).max()


def small(dim, **kw):
    args = dict(n_side=24 if dim == 2 else 10, R_frac=0.3, seed=11, jitter=0.15, vel_amp=0.05)
    args.update(kw)
    return sphcases.small_droplet(dim, **args)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("precision", [32, 64])
def test_keys_order_and_counts_bit_exact(dim, precision):
    case = small(dim)
    h = gpu_case(case, precision)
    try:
        S.step(h, 1)
        origin, cs, ncell = S.debug_grid(h)
        keys, ids = S.debug_keys(h)
        counts = S.debug_neighbor_counts(h)
    finally:
        S.destroy(h)
    pos, vel, rho, kind = case.flat()
    P = oracle.params_for_case(case)
    o_origin, o_cs, o_ncell = oracle.grid(P, pos, pad=2)
    assert cs == o_cs
    assert np.array_equal(origin, o_origin) and np.array_equal(ncell, o_ncell)
    okeys, cells, order, outside = oracle.cell_keys(P, pos, o_origin, o_cs, o_ncell)
    assert outside == 0
    assert np.array_equal(ids, order)                 # canonical order
    assert np.array_equal(keys, okeys[order])         # Morton key of every slot
    ocounts, _ = oracle.neighbors(P, pos)
    assert np.array_equal(counts, ocounts)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("nbr", ["list", "cells"])
def test_fp64_one_advection_step(dim, nbr):
    case = small(dim)
    g, o, info, oinfo, pos0, kind = run_both(case, 64, 1, nbr_mode=S.NBR_LIST if nbr == "list" else S.NBR_CELLS)
    assert info["n_sub"] == oinfo["n_sub"] > 5
    for key in ("pos", "vel", "rho", "gradC", "acc_visc"):
        assert rel_err(g, o, pos0, kind, key, case) <= 1e-12, key


@pytest.mark.parametrize("dim", [2, 3])
def test_fp64_three_advection_steps_and_keys_after_motion(dim):
    case = small(dim)
    g, o, info, oinfo, pos0, kind = run_both(case, 64, 3)
    assert info["n_sub"] == oinfo["n_sub"]
    assert info["t"] == pytest.approx(oinfo["t"], rel=1e-14)
    for key in ("pos", "vel", "rho", "gradC", "acc_visc"):
        assert rel_err(g, o, pos0, kind, key, case) <= 1e-11, key


def one_substep_case(dim):
    # viscous enough that the advection step is shorter than the acoustic
    # step, so one advection step is exactly one acoustic substep (Eq. 16-18)
    return small(dim, mu_l=50.0, mu_g=0.5)


@pytest.mark.parametrize("dim", [2, 3])
def test_fp32_one_substep(dim):
    case = one_substep_case(dim)
    g, o, info, oinfo, pos0, kind = run_both(case, 32, 1)
    assert info["n_sub"] == oinfo["n_sub"] == 1
    for key in ("pos", "vel", "rho", "gradC", "acc_visc"):
        assert rel_err(g, o, pos0, kind, key, case) <= 1e-5, key


@pytest.mark.parametrize("dim", [2, 3])
def test_fp32_one_advection_step(dim):
    case = small(dim)
    g, o, info, oinfo, pos0, kind = run_both(case, 32, 1)
    assert info["n_sub"] == oinfo["n_sub"]
    for key in ("pos", "vel", "rho", "gradC", "acc_visc"):
        assert rel_err(g, o, pos0, kind, key, case) <= 2e-4, key


@pytest.mark.parametrize("opts,ora", [
    (dict(limiter=1), dict(limiter=1)),
    (dict(limiter=2), dict(limiter=2)),
    (dict(grad_mode=1), dict(grad_mode=1)),
    (dict(penalty_form=1), dict(penalty_form=1)),
    (dict(tvf_alpha=0.0), dict(tvf_alpha=0.0)),
    (dict(xi=0.0), dict(xi=0.0)),
    (dict(limiter=3), dict(limiter=3)),
    (dict(penalty_form=2), dict(penalty_form=2)),
    (dict(penalty_scope=1), dict(penalty_scope=1)),
    (dict(wall_form=1), dict(wall_form=1)),
    (dict(stress_weights=1), dict(stress_weights=1)),
    (dict(surface_corr=1), dict(surface_corr=1)),
    (dict(surface_corr=1, nbr_mode=1), dict(surface_corr=1)),
])
def test_fp64_readings_flags(opts, ora):
    case = small(2)
    g, o, info, oinfo, pos0, kind = run_both(case, 64, 1, ora_kw=ora, **opts)
    assert info["n_sub"] == oinfo["n_sub"]
    for key in ("pos", "vel", "rho", "gradC"):
        assert rel_err(g, o, pos0, kind, key, case) <= 1e-12, key


def test_no_suction_wall_reading_changes_near_wall_particles():
    # the droplet's jittered lattice puts near-wall particles in tension
    # during the step: the no-suction reading must change their kicks (and
    # the oracle agrees with each reading, above)
    case = small(2)
    out = {}
    for form in (0, 1):
        h = gpu_case(case, 64, wall_form=form)
        S.step(h, 1)
        out[form] = S.read_fields(h, S.FIELD_VEL, 2)
        S.destroy(h)
    assert not np.array_equal(out[0], out[1])


def test_fp64_printed_vstar_one_substep():
    # the printed v* of Eq. 8 is anti-diffusive and diverges within an
    # advection step; compared over one acoustic substep of a state with
    # density (pressure) differences, where it departs from the default
    case = sphcases.free_blob(dim=2, n_side=20, seed=5, vel_amp=0.05, rho_ratio=10.0, rho_jitter=1e-3)
    pos, vel, rho, kind = case.flat()
    out = {}
    for form in (0, 1):
        h = gpu_case(case, 64, vstar_form=form, max_substeps=1)
        S.step(h, 1, check=False)
        out[form] = S.read_fields(h, S.FIELD_RHO, 2)
        S.destroy(h)
    P = oracle.params_for_case(case, vstar_form=1, max_substeps=1)
    _, _, orho, oinfo, _, _ = oracle.run(P, pos, vel, rho, kind, 1)
    assert oinfo["n_sub"] == 1
    fl = kind < 2
    rho0 = np.asarray(case.fluid_props()[0])[kind[fl]]
    a, b = out[1][fl] - rho0, orho[fl] - rho0
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    assert np.abs(out[0][fl] - out[1][fl]).max() > 1e-9 * np.abs(b).max()


@pytest.mark.parametrize("precision", [32, 64])
def test_graph_and_host_loop_identical(precision):
    case = small(3)
    out = []
    for mode in (S.LOOP_GRAPH, S.LOOP_HOST):
        h = gpu_case(case, precision, loop_mode=mode)
        S.step(h, 2)
        out.append((S.read_fields(h, S.FIELD_POS, 3), S.read_fields(h, S.FIELD_VEL, 3),
                    S.read_fields(h, S.FIELD_RHO, 3), S.case_info(h)))
        S.destroy(h)
    for a, b in zip(out[0][:3], out[1][:3]):
        assert np.array_equal(a, b)
    assert out[0][3]["n_sub"] == out[1][3]["n_sub"]


def test_profile_step_matches_graph_step():
    case = small(2)
    h1, h2 = gpu_case(case, 32), gpu_case(case, 32)
    S.step(h1, 1)
    prof = S.profile_step(h2)
    assert prof["sweep_B"][1] == S.case_info(h1)["n_sub"]
    assert all(ms >= 0 for ms, _ in prof.values())
    assert np.array_equal(S.read_fields(h1, S.FIELD_VEL, 2), S.read_fields(h2, S.FIELD_VEL, 2))
    S.destroy(h1)
    S.destroy(h2)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("precision", [32, 64])
def test_list_and_cell_walk_agree(dim, precision):
    # the list holds the same neighbours with the same pair geometry, but
    # other-phase neighbours first, and the surface sum runs in its own
    # kernel over the interface band: the two sources agree to the rounding
    # of a reordered sum
    case = small(dim)
    out = []
    for mode in (S.NBR_LIST, S.NBR_CELLS):
        h = gpu_case(case, precision, nbr_mode=mode)
        info = S.step(h, 2)
        out.append(([S.read_fields(h, f, dim) for f in (S.FIELD_POS, S.FIELD_VEL, S.FIELD_RHO, S.FIELD_GRADC)],
                    info["n_sub"]))
        S.destroy(h)
    assert out[0][1] == out[1][1]
    pos0 = case.flat()[0][:, :dim]
    tol = 1e-12 if precision == 64 else 1e-4
    for k, (a, b) in enumerate(zip(out[0][0], out[1][0])):
        if k == 0:
            a, b = a - pos0, b - pos0
        if k == 2:
            a, b = a - np.round(a), b - np.round(a)
        scale = np.abs(b).max()
        assert np.abs(a - b).max() <= tol * scale, k


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("lanes", [2, 4, 8])
def test_lanes_per_particle_fp64_against_oracle(dim, lanes):
    # L lanes split each particle's list (sweeps A, B, C): same pairs, sums
    # in another order, so the oracle bar of one advection step holds
    case = small(dim)
    g, o, info, oinfo, pos0, kind = run_both(case, 64, 1, lanes=lanes)
    assert info["n_sub"] == oinfo["n_sub"] > 5
    for key in ("pos", "vel", "rho", "gradC", "acc_visc"):
        assert rel_err(g, o, pos0, kind, key, case) <= 1e-12, key


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("lanes", [2, 4, 8])
def test_lanes_per_particle_fp32_one_substep(dim, lanes):
    case = one_substep_case(dim)
    g, o, info, oinfo, pos0, kind = run_both(case, 32, 1, lanes=lanes)
    assert info["n_sub"] == oinfo["n_sub"] == 1
    for key in ("pos", "vel", "rho", "gradC", "acc_visc"):
        assert rel_err(g, o, pos0, kind, key, case) <= 1e-5, key


@pytest.mark.parametrize("lanes", [2, 4, 8])
def test_lanes_per_particle_repeat_bitwise(lanes):
    # the group sums run in a fixed order: two runs are identical, and a
    # tile's last, partly filled block (ragged tail) is covered
    case = small(3, n_side=11)
    out = []
    for _ in range(2):
        h = gpu_case(case, 32, lanes=lanes, block=64)
        S.step(h, 2)
        out.append([S.read_fields(h, f, 3) for f in (S.FIELD_POS, S.FIELD_VEL, S.FIELD_RHO, S.FIELD_GRADC)])
        S.destroy(h)
    assert case.n % 64 != 0
    for a, b in zip(*out):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("lanes", [2, 4, 8])
def test_lanes_change_the_summation_order(lanes):
    # with L lanes a particle's list is split and the parts added in another
    # order, so FP32 results differ from one lane's in the last bits: the
    # L-lane kernels ran
    case = small(3, n_side=11)
    res = {}
    for L in (1, lanes):
        h = gpu_case(case, 32, lanes=L, block=64)
        S.step(h, 1)
        res[L] = S.read_fields(h, S.FIELD_VEL, 3)
        S.destroy(h)
    assert not np.array_equal(res[1], res[lanes])


def test_profiled_launch_counts():
    # one advection step of a two-phase list case: every per-substep kernel
    # (criterion, A, S, B, C) runs once per substep
    case = small(3)
    h = gpu_case(case, 32)
    prof = S.profile_step(h)
    n_sub = S.case_info(h)["n_sub"]
    S.destroy(h)
    for g in ("criterion", "sweep_A", "sweep_S", "sweep_B", "sweep_C"):
        assert prof[g][1] == n_sub, g
    # keys, 3 scans, scatter, cell sort, gather, copy-back, fluid ranks (flag,
    # 3 scans, scatter), list, band
    assert prof["rebuild"][1] == 15


@pytest.mark.parametrize("dim", [2, 3])
def test_surface_band_covers_every_surface_pair(dim):
    # a drop whose interface band holds a small share of the particles: the
    # band-restricted surface kernel must give the same velocities as the
    # cell walk, which evaluates the surface terms of every pair
    case = sphcases.small_droplet(dim, 24 if dim == 2 else 14, R_frac=0.25, shape="mode2", amp=0.15)
    out = []
    for mode in (S.NBR_LIST, S.NBR_CELLS):
        h = gpu_case(case, 64, nbr_mode=mode, max_substeps=1)
        S.step(h, 1, check=False)
        out.append(S.read_fields(h, S.FIELD_VEL, dim))
        S.destroy(h)
    scale = np.abs(out[1]).max()
    assert scale > 0
    assert np.abs(out[0] - out[1]).max() <= 1e-12 * scale


def test_neighbor_overflow_is_reported():
    case = small(3)
    h = gpu_case(case, 32, max_neighbors=8)
    info = S.step(h, 1, check=False)
    assert info["rc"] == S.ERR_NEIGHBORS
    S.destroy(h)


@pytest.mark.parametrize("block", [64, 160, 256])
def test_block_size_changes_no_bit(block):
    # one lane per particle: no particle's sums depend on the tile size, so
    # the timed line's 256-thread blocks (and any other size) give the
    # default 128's fields bit for bit, in the one-case mode (3D, FP32)
    case = small(3, n_side=14)
    out = {}
    for b in (128, block):
        h = gpu_case(case, 32, block=b)
        S.step(h, 2)
        out[b] = [S.read_fields(h, f, 3) for f in (S.FIELD_POS, S.FIELD_VEL, S.FIELD_RHO, S.FIELD_GRADC)], \
            S.case_info(h)
        S.destroy(h)
    (fa, ia), (fb, ib) = out[128], out[block]
    assert ia["n_sub"] == ib["n_sub"] and ia["t"] == ib["t"]
    for a, b in zip(fa, fb):
        assert np.array_equal(a, b)
