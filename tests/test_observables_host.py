"""Host-side observables against closed forms: the measures the validation
runs report (Laplace jump, deformation, anisotropy, periods, interface
disorder) evaluated on synthetic particle sets whose answer is known."""
import math

import numpy as np
import pytest

ob = pytest.importorskip("paper_2503_16082_gb300.observables")


def lattice(n, dx=1.0, dim=2):
    ax = (np.arange(n) + 0.5) * dx
    g = np.meshgrid(*([ax] * dim), indexing="ij")
    return np.stack([a.ravel() for a in g], axis=1)


def test_effective_radius_closed_form():
    assert ob.effective_radius(314, 0.1, 2) == pytest.approx(math.sqrt(3.14 / math.pi))
    assert ob.effective_radius(4189, 0.1, 3) == pytest.approx((3 * 4.189 / (4 * math.pi)) ** (1 / 3))


def test_laplace_jump_of_a_step_pressure():
    # disc of radius 10 dx on a lattice, p = 2 inside, 0.5 outside: dp = 1.5
    pos = lattice(60)
    r = np.linalg.norm(pos - 30.0, axis=1)
    phase = (r >= 10.0).astype(int)
    p = np.where(phase == 0, 2.0, 0.5)
    dp, R = ob.laplace_jump(pos, p, phase, 1.0, 1.3)
    assert dp == pytest.approx(1.5)
    assert R == pytest.approx(10.0, rel=0.02)


def test_deformation_of_a_filled_ellipse():
    # a filled ellipse with semi-axes a, b has covariance diag(a^2/4, b^2/4)
    # and D = (a - b)/(a + b), whatever its orientation
    pos = lattice(400, dx=0.05)
    a, b, th = 6.0, 4.0, 0.3
    c, s = math.cos(th), math.sin(th)
    d = pos - 10.0
    u, v = c * d[:, 0] + s * d[:, 1], -s * d[:, 0] + c * d[:, 1]
    q = d[(u / a) ** 2 + (v / b) ** 2 < 1.0]
    D = ob.deformation(np.cov(q.T, bias=True))
    assert D == pytest.approx((a - b) / (a + b), rel=2e-3)
    assert ob.taylor_deformation(0.1) == pytest.approx(0.1 * 35 / 32)


def test_anisotropy_sign_and_zero():
    pos = lattice(40)
    disc = np.linalg.norm(pos - 20.0, axis=1) < 15.0
    assert abs(ob.anisotropy(pos, np.where(disc, 0, 1))) < 1e-9
    stretched = pos * np.array([1.2, 1.0])
    assert ob.anisotropy(stretched, np.where(disc, 0, 1)) > 0.0


def test_periods_of_sinusoids():
    t = np.linspace(0.0, 10.0, 4001)
    s = 0.3 + np.sin(2 * math.pi * t / 1.7)
    assert ob.period_from_signal(t, s) == pytest.approx(1.7, rel=1e-3)
    damped = 0.1 + np.exp(-0.2 * t) * np.cos(2 * math.pi * t / 2.3 + 0.4)
    assert ob.fit_period(t, damped, 2.0) == pytest.approx(2.3, rel=1e-6)
    # Eq. 35 and Lamb's n = 2 value
    assert ob.period_2d_drop(0.2, 1.0, 1.0) == pytest.approx(2 * math.pi * math.sqrt(0.008 / 6))
    assert ob.period_lamb_3d(0.5, 1000.0, 1.0, 1.0) == pytest.approx(2 * math.pi / math.sqrt(24 / (0.125 * 3002)))


def test_interface_disorder_measure():
    # a flat interface has no stray particle; each particle moved into the
    # other fluid adds one
    pos = lattice(30)
    phase = (pos[:, 0] > 15.0).astype(int)
    assert ob.stray_fraction(pos, phase, 1.3) == 0.0
    moved = phase.copy()
    far = np.where((pos[:, 0] < 5.0) & (np.abs(pos[:, 1] - 10.5) < 0.1))[0][:2]
    moved[far] = 1
    assert ob.stray_fraction(pos, moved, 1.3) == pytest.approx(2 / len(pos))
    # a checkerboard (every neighbour at distance 1 across) is all stray
    checker = ((np.floor(pos[:, 0]) + np.floor(pos[:, 1])) % 2).astype(int)
    assert ob.stray_fraction(pos, checker, 0.55) == pytest.approx(1.0)
    # walls (phase 2) take no part
    assert ob.stray_fraction(pos, np.where(pos[:, 1] < 3.0, 2, phase), 1.3) == 0.0
