"""Values the paper prints, stored under tests/golden/ with their citation,
against the oracle and the input builders: the penalty coefficient xi for
density ratios 1..1000 (Section 4.2), the particle counts of the 2D
oscillating drop and the shear drop (Sections 5.1, 5.2), and the Reynolds
and Weber numbers of the impact (Section 5.4, Eq. 38)."""
import os

import pytest

import oracle
import sphcases

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [line.split() for line in f if line.strip() and not line.startswith("#")]


@pytest.mark.parametrize("ratio,xi", [(float(a), float(b)) for a, b in rows("xi_density_ratio.txt")])
def test_xi_of_density_ratio(ratio, xi):
    P = oracle.make_params(2, 0.1, 0.13, 10.0, 1.0, rho0=(ratio, 1.0))
    assert oracle.xi(P) == pytest.approx(xi, abs=1e-12)
    P = oracle.make_params(2, 0.1, 0.13, 10.0, 1.0, rho0=(1.0, ratio))    # either fluid heavier
    assert oracle.xi(P) == pytest.approx(xi, abs=1e-12)


@pytest.mark.parametrize("workload,res,count", [(w, int(r), int(c)) for w, r, c in rows("particle_counts.txt")])
def test_printed_particle_counts(workload, res, count):
    if workload == "oscillating_2d":
        case = sphcases.oscillating_2d(R_over_dp=res)
    else:
        case = sphcases.shear_drop_2d(R_over_dp=res)
    assert case.n_fluid == count


@pytest.mark.parametrize("u0,re,we", [tuple(float(x) for x in r) for r in rows("impact_re_we.txt")])
def test_impact_reynolds_and_weber(u0, re, we):
    case = sphcases.impact_sweep_case(u0, 10)
    rho0, eta = case.fluid_props()
    d = 2.0 * case.meta["R"]
    assert rho0[0] * u0 * d / eta[0] == pytest.approx(re, rel=1e-12)
    assert rho0[0] * u0 ** 2 * d / case.gamma == pytest.approx(we, rel=1e-12)
    assert case.meta["Re"] == pytest.approx(re) and case.meta["We"] == pytest.approx(we)
