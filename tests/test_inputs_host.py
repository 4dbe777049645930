"""The seeded synthetic inputs of the batched and served workloads follow
their stated recipe: 2D and 3D cases one to one, particle counts
log-uniform in the stated range, R ~ U[0.2, 0.5], surface tension
log-uniform in [0.1, 10], square / mode-2 / mode-3 shapes with an amplitude
in [0, 0.2] (none for squares), a box of side 4R; the served stream draws
the same way with counts in [5e3, 2e6] and Poisson arrivals at 50 per
second.  The draws repeat for a seed."""
import math

import numpy as np

import sphcases


def test_batch_recipe():
    specs = sphcases.batch_cases(512)
    assert len(specs) == 512 and [s.index for s in specs] == list(range(512))
    dims = np.array([s.dim for s in specs])
    assert set(dims) == {2, 3} and abs((dims == 3).mean() - 0.5) < 0.07
    n = np.array([s.n_target for s in specs], dtype=float)
    assert n.min() >= 2e3 and n.max() <= 2e5
    # log-uniform: the mean of log n sits mid-range, and each decade is drawn
    assert abs(np.log(n).mean() - 0.5 * (math.log(2e3) + math.log(2e5))) < 0.25
    assert ((n < 2e4).mean() > 0.35) and ((n > 2e4).mean() > 0.35)
    R = np.array([s.R for s in specs])
    assert R.min() >= 0.2 and R.max() <= 0.5 and abs(R.mean() - 0.35) < 0.02
    sig = np.array([s.sigma for s in specs])
    assert sig.min() >= 0.1 and sig.max() <= 10.0 and abs(np.log(sig).mean()) < 0.3
    shapes = [s.shape for s in specs]
    for sh in ("square", "mode2", "mode3"):
        assert abs(shapes.count(sh) / 512 - 1 / 3) < 0.07
    amps = np.array([s.amp for s in specs])
    sq = np.array([sh == "square" for sh in shapes])
    assert np.all(amps[sq] == 0.0) and amps[~sq].min() >= 0.0 and amps[~sq].max() <= 0.2


def test_batch_draws_repeat_for_the_seed():
    a, b = sphcases.batch_cases(64), sphcases.batch_cases(64)
    assert [(s.dim, s.n_target, s.R, s.sigma, s.shape, s.amp) for s in a] == \
           [(s.dim, s.n_target, s.R, s.sigma, s.shape, s.amp) for s in b]
    c = sphcases.batch_cases(64, seed=sphcases.BATCH_SEED + 1)
    assert [s.n_target for s in c] != [s.n_target for s in a]


def test_built_cases_have_the_box_and_about_the_target_count():
    specs = [s for s in sphcases.batch_cases(512) if s.n_target < 6000][:6]
    assert {s.dim for s in specs} == {2, 3}
    for s in specs:
        case = s.build()
        assert case.dim == s.dim and math.isclose(case.hi[0] - case.lo[0], 4 * s.R)
        m = max(8, int(round(s.n_target ** (1.0 / s.dim))))
        assert case.n_fluid == m ** s.dim            # the box is filled by the lattice
        assert math.isclose(case.gamma, s.sigma) and case.n > case.n_fluid   # walls outside
        rho0, _ = case.fluid_props()
        assert rho0[0] / rho0[1] == 1000.0


def test_served_stream_recipe():
    specs = sphcases.served_stream(2000)
    n = np.array([s.n_target for s in specs], dtype=float)
    assert n.min() >= 5e3 and n.max() <= 2e6
    t = np.array([s.arrival for s in specs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0) and abs(gaps.mean() - 1 / 50) < 0.002
    dims = np.array([s.dim for s in specs])
    assert abs((dims == 3).mean() - 0.5) < 0.05
