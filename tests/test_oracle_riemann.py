"""Pins of the oracle's pair Riemann solver (Section 3.1, Eqs. 8-12)."""
import numpy as np
import pytest

import oracle

C0 = 10.0


def P(limiter=0, dim=3):
    return oracle.make_params(dim, 0.02, 0.026, C0, 1.0, rho0=(1000.0, 1.0), limiter=limiter)


def test_equal_states_reproduce_the_state():
    e = np.array([0.6, 0.8, 0.0])
    v = np.array([0.3, -0.2, 0.1])
    Ps, Us, beta, pbar, vs = oracle.riemann_pair(P(), 1000.5, 50.0, v, 1000.5, 50.0, v, e)
    assert Ps == pytest.approx(50.0, abs=1e-12)
    assert Us == pytest.approx(-v @ e, abs=1e-14)
    assert beta == 0.0
    assert np.allclose(vs, v, atol=1e-14)


def test_equal_normal_velocity_gives_pair_average():
    e = np.array([1.0, 0.0, 0.0])
    vi = np.array([0.2, 0.5, 0.0])
    vj = np.array([0.2, -0.4, 0.3])
    Ps, Us, beta, pbar, vs = oracle.riemann_pair(P(), 1000.0, 3.0, vi, 1.0, -0.2, vj, e)
    assert beta == 0.0
    assert Ps == pytest.approx(pbar)
    assert pbar == pytest.approx((1000.0 * -0.2 + 1.0 * 3.0) / 1001.0)


@pytest.mark.parametrize("limiter", [0, 1, 2])
def test_swap_symmetry(limiter):
    rng = np.random.default_rng(1)
    for _ in range(50):
        e = rng.normal(size=3); e /= np.linalg.norm(e)
        vi, vj = rng.normal(size=3), rng.normal(size=3)
        ri, rj = rng.uniform(0.5, 1000), rng.uniform(0.5, 1000)
        pi, pj = rng.normal(), rng.normal()
        a = oracle.riemann_pair(P(limiter), ri, pi, vi, rj, pj, vj, e)
        b = oracle.riemann_pair(P(limiter), rj, pj, vj, ri, pi, vi, -e)
        assert a[0] == pytest.approx(b[0], rel=1e-13, abs=1e-13)      # P* symmetric
        assert a[1] == pytest.approx(-b[1], rel=1e-13, abs=1e-13)     # U* odd in e
        assert np.allclose(a[4], b[4], rtol=1e-12, atol=1e-13)         # v* frame independent


def test_limiter_range_and_closed_form():
    e = np.array([1.0, 0.0, 0.0])
    for dU in np.linspace(-5, 5, 41):
        vi = np.array([-dU, 0, 0])      # U_L = dU, U_R = 0
        _, _, beta, _, _ = oracle.riemann_pair(P(), 1000.0, 0.0, vi, 1.0, 0.0, np.zeros(3), e)
        assert 0.0 <= beta <= 1.0
        # dimensionless reading with one sound speed: beta = min(3 max(dU/c0, 0), 1)
        assert beta == pytest.approx(min(3 * max(dU / C0, 0.0), 1.0), abs=1e-15)


def test_acoustic_characteristics_hold_without_limiter():
    # With beta = 1 the star state is the linear acoustic Riemann solution:
    # it lies on the left and right characteristics p + Z U = const, p - Z U = const.
    rng = np.random.default_rng(2)
    for _ in range(50):
        e = rng.normal(size=3); e /= np.linalg.norm(e)
        vi, vj = rng.normal(size=3), rng.normal(size=3)
        ri, rj = rng.uniform(0.5, 1000), rng.uniform(0.5, 1000)
        pi, pj = 10 * rng.normal(), 10 * rng.normal()
        Ps, Us, beta, _, _ = oracle.riemann_pair(P(1), ri, pi, vi, rj, pj, vj, e)
        UL, UR = -vi @ e, -vj @ e
        zl, zr = ri * C0, rj * C0
        assert beta == 1.0
        assert Ps + zl * Us == pytest.approx(pi + zl * UL, rel=1e-12, abs=1e-10)
        assert Ps - zr * Us == pytest.approx(pj - zr * UR, rel=1e-12, abs=1e-10)


def test_pressure_jump_drives_flow_towards_low_pressure():
    e = np.array([0.0, 0.0, 1.0])          # points from j to i
    Ps, Us, _, _, vs = oracle.riemann_pair(P(), 1000.0, 5.0, np.zeros(3), 1000.0, 1.0, np.zeros(3), e)
    assert Us > 0
    assert vs @ e < 0                       # interface moves towards j (low pressure)


def test_galilean_shift_of_star_velocity():
    rng = np.random.default_rng(3)
    e = np.array([0.0, 1.0, 0.0])
    vi, vj, u0 = rng.normal(size=3), rng.normal(size=3), rng.normal(size=3)
    a = oracle.riemann_pair(P(), 900.0, 2.0, vi, 2.0, -1.0, vj, e)
    b = oracle.riemann_pair(P(), 900.0, 2.0, vi + u0, 2.0, -1.0, vj + u0, e)
    assert a[0] == pytest.approx(b[0], rel=1e-12)
    assert np.allclose(a[4] + u0, b[4], atol=1e-12)


def test_xi_formula():
    # Section 4.2: xi = 1.3 n + 0.6 for a density ratio 10^n
    assert oracle.xi(oracle.make_params(2, 1, 1, 1, 1, rho0=(1000.0, 1.0))) == pytest.approx(4.5)
    assert oracle.xi(oracle.make_params(2, 1, 1, 1, 1, rho0=(1.0, 1000.0))) == pytest.approx(4.5)
    assert oracle.xi(oracle.make_params(2, 1, 1, 1, 1, rho0=(1.0, 1.0))) == pytest.approx(0.6)
    assert oracle.xi(oracle.make_params(2, 1, 1, 1, 1, rho0=(1.0, 1.0), xi=2.0)) == 2.0
