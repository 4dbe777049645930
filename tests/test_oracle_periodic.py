"""Periodic boundaries in the oracle (the shear drop of Section 5.2 is
periodic in x): brute-force minimum-image neighbours equal the wrapped grid
search; a periodic lattice is translation invariant; a pair across the wrap
has its minimum-image distance; total momentum of a wall-free periodic drop
is conserved; a uniformly translating periodic lattice stays a uniform
lattice and re-enters through the opposite side; the key grid of a periodic
axis tiles the period exactly."""
import math

import numpy as np
import pytest

import oracle
import sphcases


def csr_sets(P, pos):
    cnt, idx = oracle.neighbors(P, pos)
    row = np.concatenate([[0], np.cumsum(cnt)])
    return [set(idx[row[i]:row[i + 1]].tolist()) for i in range(len(pos))]


@pytest.mark.parametrize("dim,per", [(2, 3), (2, 1), (3, 1), (3, 7)])
def test_bruteforce_equals_wrapped_grid(dim, per):
    case = sphcases.periodic_blob(dim, 16 if dim == 2 else 9, periodic=per, seed=4)
    pos, vel, rho, kind = case.flat()
    a = csr_sets(oracle.params_for_case(case, nbr_mode=0), pos)
    b = csr_sets(oracle.params_for_case(case, nbr_mode=1), pos)
    assert a == b
    # pairs across the wrap exist
    L = 1.0
    assert any(abs(pos[i, 0] - pos[j, 0]) > 0.5 * L for i in range(len(pos)) for j in a[i])


@pytest.mark.parametrize("dim,expected", [(2, 20), (3, 80)])
def test_periodic_lattice_is_translation_invariant(dim, expected):
    n = 12 if dim == 2 else 8
    dx = 1.0 / n
    pos = np.zeros((n ** dim, 3))
    pos[:, :dim] = sphcases.lattice([0.0] * dim, [1.0] * dim, dx)
    P = oracle.make_params(dim, dx, 1.3 * dx, 10.0, 1.0, periodic=(1 << dim) - 1,
                           box_lo=(0, 0, 0), box_hi=(1, 1, 1), nbr_mode=1)
    cnt, _ = oracle.neighbors(P, pos)
    assert (cnt == expected).all()


def test_pair_across_the_wrap_has_its_minimum_image_distance():
    pos = np.array([[0.01, 0.5, 0.0], [0.99, 0.5, 0.0]])
    P = oracle.make_params(2, 0.02, 0.013, 10.0, 1.0, periodic=1, box_lo=(0, 0, 0), box_hi=(1, 1, 0),
                           nbr_mode=0)
    cnt, idx = oracle.neighbors(P, pos)
    assert list(cnt) == [1, 1]
    P.periodic = 0
    cnt, _ = oracle.neighbors(P, pos)
    assert list(cnt) == [0, 0]


def test_wall_free_periodic_drop_conserves_momentum():
    case = sphcases.periodic_blob(2, 20, seed=7, vel_amp=0.05, rho_ratio=10.0)
    pos, vel, rho, kind = case.flat()
    P = oracle.params_for_case(case)
    m = np.asarray(case.fluid_props()[0])[kind] * case.dx ** 2
    p0 = (m[:, None] * vel).sum(0)
    pos1, vel1, rho1, info, _, _ = oracle.run(P, pos, vel, rho, kind, 3)
    assert info["status"] == 0
    p1 = (m[:, None] * vel1).sum(0)
    assert np.abs(p1 - p0).max() <= 1e-12 * (m[:, None] * np.abs(vel1)).sum()
    assert (pos1[:, :2] >= 0.0).all() and (pos1[:, :2] < 1.0).all()


def test_translating_periodic_lattice_stays_uniform():
    n, U = 16, 0.3
    dx = 1.0 / n
    p = sphcases.lattice([0.0, 0.0], [1.0, 1.0], dx)
    pos = np.zeros((len(p), 3))
    pos[:, :2] = p
    vel = np.zeros_like(pos)
    vel[:, 0] = U
    rho = np.ones(len(p))
    kind = np.zeros(len(p), dtype=np.int32)
    P = oracle.make_params(2, dx, 1.3 * dx, 10.0, 1.0, rho0=(1.0, 1.0), eta=(0.001, 0.001), periodic=3,
                           box_lo=(0, 0, 0), box_hi=(1, 1, 0), n=len(p))
    pos1, vel1, rho1, info, _, _ = oracle.run(P, pos, vel, rho, kind, 6)
    assert info["status"] == 0
    assert np.abs(vel1[:, 0] - U).max() < 1e-12 and np.abs(vel1[:, 1]).max() < 1e-12
    assert np.abs(rho1 - 1.0).max() < 1e-12
    shift = U * info["t"]
    expect = np.mod(p[:, 0] + shift, 1.0)
    d = np.abs(pos1[:, 0] - expect)
    assert np.minimum(d, 1.0 - d).max() < 1e-12
    assert (pos1[:, 0] >= 0.0).all() and (pos1[:, 0] < 1.0).all()
    assert shift > 0.5 * dx               # the last column crossed x = 1


def test_periodic_key_grid_tiles_the_period():
    case = sphcases.periodic_blob(2, 24, periodic=1, seed=2)
    pos, *_ = case.flat()
    P = oracle.params_for_case(case)
    origin, cs, ncell = oracle.grid(P, pos, pad=2)
    h = case.h_factor * case.dx
    n_expected = math.floor(1.0 / (2 * h * (1 + 2 ** -16)))
    assert ncell[0] == n_expected and origin[0] == 0.0
    assert abs(cs * ncell[0] - 1.0) < 1e-12 and cs >= 2 * h * (1 + 2 ** -16)
    pos2 = pos.copy()
    pos2[0, 0] = 1.0 - 2.0 ** -53        # last double below the period's end
    pos2[1, 0] = -1e-3                   # just below the start: wraps to the end
    pos2[2, 0] = 1.0                     # the end itself is the start
    keys, cells, order, outside = oracle.cell_keys(P, pos2, origin, cs, ncell)
    assert outside == 0
    assert cells[0][0] == ncell[0] - 1 and cells[1][0] == ncell[0] - 1 and cells[2][0] == 0
