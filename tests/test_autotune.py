"""Autotuner: cache keys, table round trip and choice of the fastest
candidate (host logic, with a fake timer); on the GPU, a tuned case gives the
same fields as the library default (block size does not enter any sum)."""
import json

import numpy as np
import pytest

import sphcases

S = pytest.importorskip("paper_2503_16082_gb300")
from paper_2503_16082_gb300 import autotune  # noqa: E402


def test_bucket_key_groups_similar_sizes():
    assert autotune.bucket_key(3, 32, 1_000_000) == autotune.bucket_key(3, 32, 1_048_575)
    assert autotune.bucket_key(3, 32, 1_000_000) != autotune.bucket_key(3, 32, 1_048_576)
    assert autotune.bucket_key(2, 32, 5000) != autotune.bucket_key(3, 32, 5000)
    assert autotune.bucket_key(2, 64, 5000) != autotune.bucket_key(2, 32, 5000)


def test_picks_fastest_and_caches(tmp_path):
    calls = []

    def fake(spec, precision, block, mode):
        calls.append((block, mode))
        return 1e6 * block if mode == S.NBR_LIST else 1e5 * block

    path = str(tmp_path / "tune.json")
    t = autotune.Tuner(path, measure=fake)
    spec = sphcases.small_droplet(2, 20)
    assert t.best(spec) == {"block": 256, "nbr_mode": S.NBR_LIST}
    n_calls = len(calls)
    assert n_calls == len(autotune.BLOCKS) * 2
    assert t.best(spec) == {"block": 256, "nbr_mode": S.NBR_LIST}      # cached
    assert len(calls) == n_calls
    t2 = autotune.Tuner(path, measure=fake)                              # reloaded from disk
    assert t2.best(spec) == {"block": 256, "nbr_mode": S.NBR_LIST}
    assert len(calls) == n_calls
    table = json.load(open(path))
    assert list(table) == [autotune.bucket_key(2, 32, spec.n)]


@pytest.mark.gpu
def test_tuned_case_equals_default():
    spec = sphcases.small_droplet(3, 12, R_frac=0.3, shape="mode2", amp=0.15)
    t = autotune.Tuner(adv=1, nbr_modes=(S.NBR_LIST,))
    choice = t.best(spec)
    assert choice["block"] in autotune.BLOCKS
    out = []
    for kw in ({}, choice):
        h = S.case_from_spec(spec, **kw)
        S.step(h, 2)
        out.append([S.read_fields(h, f, 3) for f in (S.FIELD_POS, S.FIELD_VEL, S.FIELD_RHO)])
        S.destroy(h)
    for a, b in zip(*out):
        assert np.array_equal(a, b)
