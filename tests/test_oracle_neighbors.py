"""Oracle neighbour search: the uniform-grid search equals an O(N^2) brute
force, lattice counts equal an independent enumeration, and the canonical
cell-key order is a valid sort by (Morton code, insertion index)."""
import itertools

import numpy as np
import pytest

import oracle


def jittered(dim, m, seed, jitter=0.3):
    rng = np.random.default_rng(seed)
    dx = 1.0 / m
    g = np.stack(np.meshgrid(*[(np.arange(m) + 0.5) * dx] * dim, indexing="ij"), -1).reshape(-1, dim)
    g = g + rng.uniform(-jitter, jitter, g.shape) * dx
    pos = np.zeros((len(g), 3))
    pos[:, :dim] = g
    return pos, dx


@pytest.mark.parametrize("dim,m", [(2, 30), (3, 11)])
def test_grid_equals_brute_force(dim, m):
    pos, dx = jittered(dim, m, seed=dim)
    P0 = oracle.make_params(dim, dx, 1.3 * dx, 10.0, 1.0, nbr_mode=0)
    P1 = oracle.make_params(dim, dx, 1.3 * dx, 10.0, 1.0, nbr_mode=1)
    c0, i0 = oracle.neighbors(P0, pos)
    c1, i1 = oracle.neighbors(P1, pos)
    assert np.array_equal(c0, c1)
    assert np.array_equal(i0, i1)
    # explicit O(N^2) check in numpy, independent of the C code
    d = np.linalg.norm(pos[:, None, :] - pos[None, :, :], axis=2)
    np.fill_diagonal(d, np.inf)
    assert np.array_equal((d < 2 * 1.3 * dx).sum(1), c0)


@pytest.mark.parametrize("dim,expect", [(2, None), (3, None)])
def test_lattice_interior_count(dim, expect):
    # count integer points k != 0 with |k| < 2.6 by enumeration
    rng = range(-3, 4)
    want = sum(1 for k in itertools.product(rng, repeat=dim)
               if 0 < sum(t * t for t in k) < 2.6 ** 2)
    assert want == (20 if dim == 2 else 80)
    m = 9
    pos, dx = jittered(dim, m, seed=0, jitter=0.0)
    P = oracle.make_params(dim, dx, 1.3 * dx, 10.0, 1.0, nbr_mode=1)
    counts, _ = oracle.neighbors(P, pos)
    centre = np.argmin(np.linalg.norm(pos[:, :dim] - 0.5, axis=1))
    assert counts[centre] == want


def test_coincident_particles_detected():
    pos = np.zeros((3, 3))
    pos[1, 0] = 0.01
    P = oracle.make_params(2, 0.01, 0.013, 10.0, 1.0, nbr_mode=0)
    with pytest.raises(ValueError):
        oracle.neighbors(P, pos)


@pytest.mark.parametrize("dim", [2, 3])
def test_cell_keys_canonical_order(dim):
    pos, dx = jittered(dim, 12 if dim == 2 else 7, seed=5)
    P = oracle.make_params(dim, dx, 1.3 * dx, 10.0, 1.0)
    origin, cs, ncell = oracle.grid(P, pos, pad=2)
    keys, cells, order, outside = oracle.cell_keys(P, pos, origin, cs, ncell)
    assert outside == 0
    assert cs > 2 * 1.3 * dx
    # cells: floor division, recomputed in numpy
    ref = np.floor((pos[:, :dim] - origin[:dim]) / cs).astype(int)
    assert np.array_equal(cells[:, :dim], ref)
    # Morton interleave recomputed bit by bit
    for i in range(0, len(pos), 7):
        code = 0
        for b in range(10):
            for a in range(dim):
                code |= ((int(cells[i, a]) >> b) & 1) << (b * dim + a)
        assert int(keys[i]) == code
    # order sorts by (key, index)
    want = sorted(range(len(pos)), key=lambda i: (int(keys[i]), i))
    assert list(order) == want
