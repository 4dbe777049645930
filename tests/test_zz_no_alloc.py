"""GPU check of sphst_cell_order_noalloc, the cell-order call for callers
that may not allocate device memory (a framework whose pool owns all device
memory, a real-time caller that must not allocate after start-up).  The
test allocates the input and output buffers itself, as such a caller would,
and compares two calls in a row with the oracle's canonical order and with
the order that the library's own rebuild produced for the same particles
(integers: exact match).  Every call that is expected to be rejected still
gets real device buffers large enough for its n, so that a regression of a
limit check gives a wrong result or an error code, never an access outside
a buffer."""
import numpy as np
import pytest

import oracle
import sphcases

pytestmark = pytest.mark.gpu

S = pytest.importorskip("paper_2503_16082_gb300")
torch = pytest.importorskip("torch")


def _run(dim, pos, origin, cs, ncell, dev, fill=-1):
    n = len(pos)
    pos_d = torch.tensor(np.asarray(pos, dtype=np.float64).reshape(n, 3), device=dev)
    keys_d = torch.full((max(n, 1),), fill, dtype=torch.int64, device=dev)
    order_d = torch.full((max(n, 1),), fill, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    err = None
    try:
        S.cell_order_noalloc(dim, n, pos_d.data_ptr(), origin, cs, ncell,
                             keys_d.data_ptr(), order_d.data_ptr(), stream)
    except S.SphstError as e:
        err = e
    return keys_d.cpu().numpy()[:n].view(np.uint64), order_d.cpu().numpy()[:n], err


@pytest.mark.parametrize("dim", [2, 3])
def test_cell_order_noalloc_matches_oracle_and_rebuild(dim):
    case = sphcases.small_droplet(dim, 24 if dim == 2 else 12, R_frac=0.3, seed=3,
                                  jitter=0.2, vel_amp=0.0)
    h = S.case_from_spec(case, precision=64)
    try:
        S.step(h, 1)
        keys_ref, ids_ref = S.debug_keys(h)
        origin, cs, ncell = S.debug_grid(h)
    finally:
        S.destroy(h)
    pos = case.flat()[0]
    okeys, _, oorder, outside = oracle.cell_keys(oracle.params_for_case(case), pos, origin, cs, ncell)
    assert outside == 0
    dev = torch.device("cuda", 0)
    for _ in range(2):
        keys, order, err = _run(dim, pos, origin, cs, ncell, dev)
        assert err is None
        assert np.array_equal(order, oorder)
        assert np.array_equal(keys, okeys[oorder])
        assert np.array_equal(order, ids_ref)
        assert np.array_equal(keys, keys_ref)


def test_cell_order_noalloc_clamps_and_reports_outside():
    """One particle beyond the grid's upper x end: DOMAIN, and the order is
    that of the particle moved into the nearest cell."""
    rng = np.random.default_rng(11)
    n, ncell, cs = 500, np.array([6, 5, 4], dtype=np.int32), 0.25
    origin = np.array([0.0, 0.0, 0.0])
    pos = rng.uniform(0.0, 1.0, size=(n, 3)) * (ncell * cs)
    pos[17, 0] = ncell[0] * cs + 0.3                      # outside along x
    inside = pos.copy()
    inside[17, 0] = (ncell[0] - 0.5) * cs                  # the cell it is clamped into
    P = oracle.make_params(3, 0.1, 0.13, 10.0, 1.0)
    okeys, _, oorder, outside = oracle.cell_keys(P, inside, origin, cs, ncell)
    assert outside == 0
    keys, order, err = _run(3, pos, origin, cs, ncell, torch.device("cuda", 0))
    assert err is not None and err.code == S.ERR_DOMAIN
    assert np.array_equal(order, oorder)
    assert np.array_equal(keys, okeys[oorder])


def test_cell_order_noalloc_coarse_grid():
    """A grid of one cell: 200 particles are ordered by index (bounded work);
    300 exceed the per-cell limit and are rejected with the outputs left as
    they were."""
    rng = np.random.default_rng(12)
    dev = torch.device("cuda", 0)
    origin, cs, ncell = np.zeros(3), 1.0, np.array([1, 1, 1], dtype=np.int32)
    pos = rng.uniform(0.0, 1.0, size=(200, 3))
    keys, order, err = _run(3, pos, origin, cs, ncell, dev)
    assert err is None
    assert np.array_equal(order, np.arange(200)) and np.all(keys == 0)
    pos = rng.uniform(0.0, 1.0, size=(300, 3))
    keys, order, err = _run(3, pos, origin, cs, ncell, dev, fill=-7)
    assert err is not None and err.code == S.ERR_INVALID_ARG
    assert np.all(order == -7) and np.all(keys.view(np.int64) == -7)


def test_cell_order_noalloc_rejects_oversize():
    dev = torch.device("cuda", 0)
    n = (1 << 19) + 1
    pos_d = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    keys_d = torch.zeros(n, dtype=torch.int64, device=dev)
    order_d = torch.zeros(n, dtype=torch.int64, device=dev)
    with pytest.raises(S.SphstError) as e:
        S.cell_order_noalloc(3, n, pos_d.data_ptr(), [0, 0, 0], 0.1, [8, 8, 8],
                             keys_d.data_ptr(), order_d.data_ptr())
    assert e.value.code == S.ERR_INVALID_ARG
    for ncell in ([200, 200, 200], [2000, 1, 1], [1 << 30, 1, 1]):
        with pytest.raises(S.SphstError) as e:
            S.cell_order_noalloc(3, 10, pos_d.data_ptr(), [0, 0, 0], 0.1, ncell,
                                 keys_d.data_ptr(), order_d.data_ptr())
        assert e.value.code == S.ERR_INVALID_ARG
    with pytest.raises(S.SphstError) as e:
        S.cell_order_noalloc(2, 10, pos_d.data_ptr(), [0, 0], 0.1, [40000, 2],
                             keys_d.data_ptr(), order_d.data_ptr())
    assert e.value.code == S.ERR_INVALID_ARG
    with pytest.raises(ValueError):
        S.cell_order_noalloc(3, 10, pos_d.data_ptr(), [0, 0], 0.1, [8, 8],
                             keys_d.data_ptr(), order_d.data_ptr())
