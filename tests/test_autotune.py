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


def test_candidates_cover_blocks_sources_and_lanes():
    t = autotune.Tuner(measure=lambda *a: 1.0)
    cand = list(t.candidates())
    assert len(cand) == len(set(cand))
    # the cell walk runs one lane per particle; a block keeps >= 16 particles
    assert all(L == 1 for b, m, L in cand if m == S.NBR_CELLS)
    assert all(b // L >= 16 for b, m, L in cand)
    assert {(b, L) for b, m, L in cand if m == S.NBR_LIST} == {
        (b, L) for b in autotune.BLOCKS for L in autotune.LANES if b // L >= 16}
    assert {b for b, m, L in cand if m == S.NBR_CELLS} == set(autotune.BLOCKS)


def test_picks_fastest_and_caches(tmp_path):
    calls = []

    def fake(spec, precision, block, mode, lanes):
        calls.append((block, mode, lanes))
        return (1e6 if mode == S.NBR_LIST else 1e5) * block * (3 - abs(lanes - 2))

    path = str(tmp_path / "tune.json")
    t = autotune.Tuner(path, measure=fake)
    spec = sphcases.small_droplet(2, 20)
    want = {"block": 256, "nbr_mode": S.NBR_LIST, "lanes": 2}
    assert t.best(spec) == want
    n_calls = len(calls)
    assert n_calls == len(list(t.candidates()))
    assert t.best(spec) == want                                          # cached
    assert len(calls) == n_calls
    t2 = autotune.Tuner(path, measure=fake)                              # reloaded from disk
    assert t2.best(spec) == want
    assert len(calls) == n_calls
    table = json.load(open(path))
    assert list(table) == [autotune.bucket_key(2, 32, spec.n)]


def test_old_table_without_lanes_reads_as_one_lane(tmp_path):
    path = str(tmp_path / "tune.json")
    spec = sphcases.small_droplet(2, 20)
    json.dump({autotune.bucket_key(2, 32, spec.n): {"block": 64, "nbr_mode": S.NBR_LIST}}, open(path, "w"))

    def never(*a):
        raise AssertionError("a cached entry must not be re-measured")

    t = autotune.Tuner(path, measure=never)
    assert t.best(spec) == {"block": 64, "nbr_mode": S.NBR_LIST, "lanes": 1}


@pytest.mark.gpu
def test_tuned_case_equals_default():
    # the block size enters no sum: the tuned launch gives the same fields,
    # bit for bit, as the default block with the same lanes per particle
    spec = sphcases.small_droplet(3, 12, R_frac=0.3, shape="mode2", amp=0.15)
    t = autotune.Tuner(adv=1, nbr_modes=(S.NBR_LIST,))
    choice = t.best(spec)
    assert choice["block"] in autotune.BLOCKS and choice["lanes"] in autotune.LANES
    out = []
    for kw in ({"lanes": choice["lanes"]}, choice):
        h = S.case_from_spec(spec, **kw)
        S.step(h, 2)
        out.append([S.read_fields(h, f, 3) for f in (S.FIELD_POS, S.FIELD_VEL, S.FIELD_RHO)])
        S.destroy(h)
    for a, b in zip(*out):
        assert np.array_equal(a, b)
