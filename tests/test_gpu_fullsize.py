"""Parity at the full size of the benchmarked workload (the 3D oscillating
drop, 1,191,016 particles, in the launch configuration bench.py times):

* cell grid, Morton keys, canonical order and neighbour counts of all
  particles: bit-exact against the oracle;
* one acoustic substep of the whole case (max_substeps = 1): every fluid
  particle's velocity, density deviation, colour gradient and viscous
  acceleration against the oracle's, within 1e-12 (FP64) / 1e-5 (FP32) of
  each field's maximum (densities: plus the rounding of rho ~ 1000 itself).
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
