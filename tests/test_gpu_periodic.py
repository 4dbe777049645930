"""Periodic boundaries on the GPU against the oracle: cell grid, keys,
canonical order and neighbour counts bit-exact; one FP64 advection step of a
drop across the wrap within 1e-12 (list and cell walk, 2D periodic in x and
y, 3D periodic in x); a uniformly translating periodic lattice stays uniform
and re-enters through the opposite side."""
import numpy as np
import pytest

import oracle
import sphcases

pytestmark = pytest.mark.gpu

S = pytest.importorskip("paper_2503_16082_gb300")

CASES = [(2, 3), (3, 1)]


def blob(dim, per):
    return sphcases.periodic_blob(dim, 20 if dim == 2 else 10, periodic=per, seed=9)


def wrapped(d, per, dim):
    d = d.copy()
    for a in range(dim):
        if (per >> a) & 1:
            d[:, a] -= np.round(d[:, a])          # period 1: minimum image
    return d


@pytest.mark.parametrize("dim,per", CASES)
def test_periodic_keys_order_counts_bit_exact(dim, per):
    case = blob(dim, per)
    h = S.case_from_spec(case, precision=64, max_substeps=1)
    S.step(h, 1, check=False)
    origin, cs, ncell = S.debug_grid(h)
    keys, ids = S.debug_keys(h)
    counts = S.debug_neighbor_counts(h)
    S.destroy(h)
    pos, vel, rho, kind = case.flat()
    P = oracle.params_for_case(case)
    o_origin, o_cs, o_ncell = oracle.grid(P, pos, pad=2)
    assert cs == o_cs and np.array_equal(origin, o_origin) and np.array_equal(ncell, o_ncell)
    okeys, _, order, outside = oracle.cell_keys(P, pos, o_origin, o_cs, o_ncell)
    assert outside == 0
    assert np.array_equal(ids, order) and np.array_equal(keys, okeys[order])
    ocounts, _ = oracle.neighbors(P, pos)
    assert np.array_equal(counts, ocounts)


@pytest.mark.parametrize("dim,per", CASES)
@pytest.mark.parametrize("nbr", ["list", "cells"])
def test_periodic_fp64_one_advection_step(dim, per, nbr):
    case = blob(dim, per)
    mode = S.NBR_LIST if nbr == "list" else S.NBR_CELLS
    h = S.case_from_spec(case, precision=64, nbr_mode=mode)
    info = S.step(h, 1)
    g = {f: S.read_fields(h, k, dim) for f, k in (("pos", S.FIELD_POS), ("vel", S.FIELD_VEL),
                                                  ("rho", S.FIELD_RHO), ("gradC", S.FIELD_GRADC))}
    S.destroy(h)
    pos, vel, rho, kind = case.flat()
    P = oracle.params_for_case(case)
    p1, v1, r1, oinfo, gC, _ = oracle.run(P, pos, vel, rho, kind, 1)
    assert info["n_sub"] == oinfo["n_sub"] > 3
    fl = kind < 2
    dg = wrapped(g["pos"][fl] - pos[fl, :dim], per, dim)
    do = wrapped(p1[fl, :dim] - pos[fl, :dim], per, dim)
    assert np.abs(dg - do).max() <= 1e-12 * np.abs(do).max()
    for key, o in (("vel", v1[:, :dim]), ("rho", r1), ("gradC", gC[:, :dim])):
        a, b = g[key][fl], o[fl]
        if key == "rho":
            rho0 = np.asarray(case.fluid_props()[0])[kind[fl]]
            a, b = a - rho0, b - rho0
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), key
    # positions stay inside the period on the periodic axes
    for a in range(dim):
        if (per >> a) & 1:
            assert (g["pos"][:, a] >= 0.0).all() and (g["pos"][:, a] < 1.0).all()


def test_translating_periodic_lattice_stays_uniform():
    n, U = 16, 0.3
    dx = 1.0 / n
    p = sphcases.lattice([0.0, 0.0], [1.0, 1.0], dx)
    case = sphcases.Case(name="translating lattice", dim=2, lo=[0.0, 0.0], hi=[1.0, 1.0], dx=dx, gamma=1.0,
                         phases=[sphcases.Phase("fluid", p, rho0=1.0, eta=0.001,
                                                vel=np.tile([U, 0.0], (len(p), 1)))],
                         periodic=3)
    h = S.case_from_spec(case, precision=64)
    info = S.step(h, 6)
    pos = S.read_fields(h, S.FIELD_POS, 2)
    vel = S.read_fields(h, S.FIELD_VEL, 2)
    rho = S.read_fields(h, S.FIELD_RHO, 2)
    S.destroy(h)
    assert np.abs(vel[:, 0] - U).max() < 1e-12 and np.abs(vel[:, 1]).max() < 1e-12
    assert np.abs(rho - 1.0).max() < 1e-12
    expect = np.mod(p[:, 0] + U * info["t"], 1.0)
    d = np.abs(pos[:, 0] - expect)
    assert np.minimum(d, 1.0 - d).max() < 1e-12
    assert U * info["t"] > 0.5 * dx
