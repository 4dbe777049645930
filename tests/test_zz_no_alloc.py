"""GPU check of sphst_cell_order_noalloc, the cell-order call for callers
that may not allocate device memory (a framework whose pool owns all device
memory, a real-time caller that must not allocate after start-up).  The
test allocates the input and output buffers itself, as such a caller would,
and compares two calls in a row with the order and keys that the library's
own rebuild produced for the same particles (integers: exact match)."""
import numpy as np
import pytest

import sphcases

pytestmark = pytest.mark.gpu

S = pytest.importorskip("paper_2503_16082_gb300")
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("dim", [2, 3])
def test_cell_order_noalloc_matches_rebuild(dim):
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
    n = len(pos)
    dev = torch.device("cuda", 0)
    pos_d = torch.tensor(pos, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for _ in range(2):
        keys_d = torch.full((n,), -1, dtype=torch.int64, device=dev)
        order_d = torch.full((n,), -1, dtype=torch.int64, device=dev)
        S.cell_order_noalloc(dim, n, pos_d.data_ptr(), origin, cs, ncell,
                             keys_d.data_ptr(), order_d.data_ptr(), stream)
        keys = keys_d.cpu().numpy().view(np.uint64)
        order = order_d.cpu().numpy()
        assert np.array_equal(order, ids_ref)
        assert np.array_equal(keys, keys_ref)


def test_cell_order_noalloc_rejects_oversize():
    with pytest.raises(S.SphstError) as e:
        S.cell_order_noalloc(3, (1 << 19) + 1, 1, [0, 0, 0], 0.1, [8, 8, 8], 1, 1)
    assert e.value.code == S.ERR_INVALID_ARG
    with pytest.raises(S.SphstError) as e:
        S.cell_order_noalloc(3, 10, 1, [0, 0, 0], 0.1, [200, 200, 200], 1, 1)
    assert e.value.code == S.ERR_INVALID_ARG
