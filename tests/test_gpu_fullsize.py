"""Parity at the full size of the benchmarked workload (the 3D oscillating
drop, 1,191,016 particles, in the launch configuration bench.py times):

* cell grid, Morton keys, canonical order and neighbour counts of all
  particles: bit-exact against the oracle;
* one acoustic substep of the whole case (max_substeps = 1): every fluid
  particle's velocity, density deviation, colour gradient and viscous
  acceleration against the oracle's, within 1e-12 (FP64) / 1e-5 (FP32) of
  each field's maximum (densities: plus the rounding of rho ~ 1000 itself);
* the same substep particle by particle: |g_i - o_i| <= tol |o_i| + kappa
  max|o| for every fluid particle, and positions against the oracle's.

The per-particle floor kappa: at rest, a particle's acceleration is a sum
of ~80 pair terms, each as large as p_i |W'| V_j, that cancel to a small
residual in the bulk.  Each term carries the rounding of its arithmetic and
of the stored positions (FP32 offsets from the cell origin: ~4e-9 absolute,
1.5e-7 of h), so a sum has an absolute error of about sqrt(80) x 10 ops x
eps relative to the largest terms -- 5e-6 of the field's maximum in FP32
(eps = 6e-8), 1e-13 in FP64 (eps = 1.1e-16).  Below that floor a particle's
relative error measures the cancellation, not the kernel; above it (the
particles carrying the field) the relative bar 1e-5 / 1e-12 applies.
"""
import numpy as np
import pytest

import oracle
import sphcases

pytestmark = pytest.mark.gpu

S = pytest.importorskip("paper_2503_16082_gb300")


@pytest.fixture(scope="module")
def big():
    case = sphcases.oscillating_3d()
    pos, vel, rho, kind = case.flat()
    P1 = oracle.params_for_case(case, max_substeps=1)
    _, ov, orho, oinfo, ogc, oav = oracle.run(P1, pos, vel, rho, kind, 1)
    return case, (pos, vel, rho, kind), (ov, orho, ogc, oav, oinfo)


def test_fullsize_keys_order_counts(big):
    case, (pos, vel, rho, kind), _ = big
    h = S.case_from_spec(case, precision=32, max_substeps=1)
    S.step(h, 1, check=False)
    origin, cs, ncell = S.debug_grid(h)
    keys, ids = S.debug_keys(h)
    counts = S.debug_neighbor_counts(h)
    S.destroy(h)
    P = oracle.params_for_case(case)
    o_origin, o_cs, o_ncell = oracle.grid(P, pos, pad=2)
    assert cs == o_cs and np.array_equal(origin, o_origin) and np.array_equal(ncell, o_ncell)
    okeys, _, order, outside = oracle.cell_keys(P, pos, o_origin, o_cs, o_ncell)
    assert outside == 0
    assert np.array_equal(ids, order)
    assert np.array_equal(keys, okeys[order])
    ocounts, _ = oracle.neighbors(P, pos)
    assert np.array_equal(counts, ocounts)


@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 1e-5)])
def test_fullsize_one_substep(big, precision, tol):
    case, (pos, vel, rho, kind), (ov, orho, ogc, oav, oinfo) = big
    h = S.case_from_spec(case, precision=precision, max_substeps=1)
    info = S.step(h, 1, check=False)
    assert info["n_sub"] == oinfo["n_sub"] == 1
    g = {"vel": S.read_fields(h, S.FIELD_VEL, 3), "rho": S.read_fields(h, S.FIELD_RHO, 3),
         "gradC": S.read_fields(h, S.FIELD_GRADC, 3), "acc_visc": S.read_fields(h, S.FIELD_ACC_VISC, 3)}
    S.destroy(h)
    fl = kind < 2
    rho0 = np.asarray(case.fluid_props()[0])[kind[fl]]
    ref = {"vel": ov[fl], "rho": orho[fl] - rho0, "gradC": ogc[fl], "acc_visc": oav[fl]}
    got = {"vel": g["vel"][fl], "rho": g["rho"][fl] - rho0, "gradC": g["gradC"][fl], "acc_visc": g["acc_visc"][fl]}
    for k in ref:
        scale = np.abs(ref[k]).max()
        err = np.abs(got[k] - ref[k]).max()
        if scale == 0.0:                  # e.g. viscous acceleration of a fluid at rest
            assert err == 0.0, k
            continue
        # densities are read back as rho0 + drho, so both sides carry the
        # representation error of rho ~ 1000 (ulp 1.1e-13 in FP64)
        slack = 4 * np.spacing(1000.0) if k == "rho" else 0.0
        assert err <= tol * scale + slack, (k, err / scale)


# (tol, kappa) of the per-particle bar |g_i - o_i| <= tol |o_i| + kappa max|o|
PER_PARTICLE = {64: (1e-12, 1e-13), 32: (1e-5, 5e-6)}


@pytest.mark.parametrize("precision", [64, 32])
def test_fullsize_one_substep_per_particle(big, precision):
    case, (pos, vel, rho, kind), (ov, orho, ogc, oav, oinfo) = big
    P1 = oracle.params_for_case(case, max_substeps=1)
    opos, _, _, _, _, _ = oracle.run(P1, pos, vel, rho, kind, 1)
    h = S.case_from_spec(case, precision=precision, max_substeps=1)
    S.step(h, 1, check=False)
    g = {"vel": S.read_fields(h, S.FIELD_VEL, 3), "rho": S.read_fields(h, S.FIELD_RHO, 3),
         "gradC": S.read_fields(h, S.FIELD_GRADC, 3), "pos": S.read_fields(h, S.FIELD_POS, 3)}
    S.destroy(h)
    fl = kind < 2
    rho0 = np.asarray(case.fluid_props()[0])[kind[fl]]
    tol, kappa = PER_PARTICLE[precision]
    ref = {"vel": ov[fl], "rho": orho[fl] - rho0, "gradC": ogc[fl]}
    got = {"vel": g["vel"][fl], "rho": g["rho"][fl] - rho0, "gradC": g["gradC"][fl]}
    for k in ref:
        o = np.linalg.norm(ref[k].reshape(len(ref[k]), -1), axis=1)
        err = np.linalg.norm((got[k] - ref[k]).reshape(len(o), -1), axis=1)
        slack = 4 * np.spacing(1000.0) if k == "rho" else 0.0
        bar = tol * o + kappa * o.max() + slack
        bad = err > bar
        assert not bad.any(), (k, int(bad.sum()), float((err / np.maximum(o, 1e-300))[bad].max()))
        # the particles that carry the field (above the floor) meet the
        # relative bar on their own
        carry = o > (kappa / tol) * o.max()
        assert np.all(err[carry] <= 2 * tol * o[carry] + slack), k
    # positions: the oracle's x + dt v against the GPU's, to the storage
    # resolution of a position (FP64: a few ulp of |x|; FP32: a few ulp of
    # an offset inside a 2h-wide cell, about 4e-9 here) plus the relative
    # bar on the displacement
    disp = np.linalg.norm(opos[fl] - pos[fl], axis=1)
    dx = np.linalg.norm(g["pos"][fl] - opos[fl], axis=1)
    res = 4 * np.spacing(np.abs(opos[fl]).max()) if precision == 64 else 4 * np.spacing(np.float32(2.6 * case.dx))
    assert np.all(dx <= tol * disp + res), (float(dx.max()), float(res))
