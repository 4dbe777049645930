"""A fluid particle beside a single wall particle, reduced by hand (Eqs. 7-13
with the wall reading: the wall's state is the mirror image of the fluid
particle's, rho_R = rho_i, p_R = p_i, U_R = 2 U_w - U_L; v* = v_w in the
continuity equation; eta_i and v_i - v_w in the viscous term).  With the
wall at r along +x, e_ij = (-1, 0), U_L = u (the fluid's velocity towards
the wall), U_w = a (the wall's), so

    dU  = U_L - U_R = 2 (u - a)
    beta = min(3 max(dU / c0, 0), 1)                      (Eq. 11, reading R6)
    P*  = p_i + beta rho_i c0 dU / 2                       (Eq. 9, Z_L = Z_R)
    a_p = -(2 / rho_i) P* W' e_ij V_w
    a_v = (2 / rho_i) eta_i (v_i - v_w) / r W' V_w         (Eq. 13)
    drho/dt = 2 rho_i (v_i - v_w) . e_ij W' V_w            (Eq. 6, v* = v_w)

The dissipative part of P* is the one piece of the wall reading that no
wave test fixes (it is second order in the amplitude): this pair fixes its
mirrored velocity and its limiter exactly, in the three regimes of Eq. 11
(approach with beta < 1, fast approach with beta = 1, separation)."""
import math

import numpy as np
import pytest

import oracle

WALL = 2


def wendland_dW(h, r):
    a = 7.0 / (4.0 * math.pi * h * h)
    q = r / h
    return -5.0 * a * q * (1.0 - q / 2.0) ** 3 / h


def closed_form(u, w, a, b, rho_i, rho0, eta, c0, dx, h, r):
    dW = wendland_dW(h, r)
    V = dx * dx
    p_i = c0 * c0 * (rho_i - rho0)
    dU = 2.0 * (u - a)
    beta = min(3.0 * max(dU / c0, 0.0), 1.0)
    Ps = p_i + beta * rho_i * c0 * dU / 2.0
    e = np.array([-1.0, 0.0])
    a_p = -(2.0 / rho_i) * Ps * dW * e * V
    vij = np.array([u - a, w - b])
    a_v = (2.0 / rho_i) * eta * vij / r * dW * V
    drho = 2.0 * rho_i * float(vij @ e) * dW * V
    return a_p, a_v, drho, beta


@pytest.mark.parametrize("u,a,rho_eps,beta_want", [(0.5, 0.0, 0.0, 0.3),     # approach
                                                   (0.7, 0.2, 0.01, 0.3),    # moving wall, compressed fluid
                                                   (3.0, 0.0, 0.0, 1.0),     # fast approach: clipped
                                                   (-0.4, 0.1, -0.02, 0.0)])  # separation
def test_fluid_particle_beside_a_wall_particle(u, a, rho_eps, beta_want):
    dx, c0, rho0, eta = 0.1, 10.0, 1.0, 0.3
    h = 1.3 * dx
    r = 0.9 * dx
    w, b = 0.25, -0.15                                   # tangential velocities
    pos = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    vel = np.array([[u, w, 0.0], [a, b, 0.0]])
    rho_i = rho0 * (1.0 + rho_eps)
    rho = np.array([rho_i, rho0])
    kind = np.array([0, WALL], dtype=np.int32)
    P = oracle.make_params(2, dx, h, c0, 1.0, rho0=(rho0, rho0), eta=(eta, eta), n=2, tvf_alpha=0.0)
    out = oracle.forces(P, pos, vel, rho, kind)
    a_p, a_v, drho, beta = closed_form(u, w, a, b, rho_i, rho0, eta, c0, dx, h, r)
    assert beta == pytest.approx(beta_want, rel=1e-12)
    assert out["a_p"][0, :2] == pytest.approx(a_p, rel=1e-13, abs=1e-13 * np.abs(a_p).max() + 1e-300)
    assert out["a_v"][0, :2] == pytest.approx(a_v, rel=1e-13, abs=1e-13 * np.abs(a_v).max())
    assert out["drho"][0] == pytest.approx(drho, rel=1e-13)
    # the wall particle itself takes no force and keeps its density
    assert np.all(out["a_p"][1] == 0.0) and np.all(out["a_v"][1] == 0.0) and out["drho"][1] == 0.0
    assert np.all(out["gradC"] == 0.0) and np.all(out["a_s"] == 0.0)


def test_dissipation_vanishes_for_a_particle_moving_with_the_wall():
    # same normal velocity as the wall: dU = 0, P* = p_i, no density change
    dx, c0 = 0.1, 10.0
    h = 1.3 * dx
    pos = np.array([[0.0, 0.0, 0.0], [0.8 * dx, 0.0, 0.0]])
    vel = np.array([[0.4, 0.0, 0.0], [0.4, 0.0, 0.0]])
    P = oracle.make_params(2, dx, h, c0, 1.0, rho0=(1.0, 1.0), eta=(0.1, 0.1), n=2, tvf_alpha=0.0)
    out = oracle.forces(P, pos, vel, np.array([1.0, 1.0]), np.array([0, WALL], dtype=np.int32))
    assert np.all(out["a_p"][0] == 0.0) and np.all(out["a_v"][0] == 0.0) and out["drho"][0] == 0.0


@pytest.mark.parametrize("u,rho_eps", [(0.0, -0.02), (0.05, -0.02), (-0.3, -0.01)])
def test_no_suction_wall_reading(u, rho_eps):
    """The same pair in tension (p_i < 0) with slow approach or separation:
    the mirror reading's P* = p_i + beta rho_i c0 dU / 2 is negative, so the
    wall pulls the particle towards itself (a_p along +x, the wall's side);
    the no-suction reading (wall_form 1) floors P* at zero, and the pressure
    force vanishes.  Viscous force and density change are unchanged."""
    dx, c0, rho0, eta = 0.1, 10.0, 1.0, 0.3
    h = 1.3 * dx
    r = 0.9 * dx
    pos = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    vel = np.array([[u, 0.1, 0.0], [0.0, 0.0, 0.0]])
    rho_i = rho0 * (1.0 + rho_eps)
    rho = np.array([rho_i, rho0])
    kind = np.array([0, WALL], dtype=np.int32)
    a_p, a_v, drho, beta = closed_form(u, 0.1, 0.0, 0.0, rho_i, rho0, eta, c0, dx, h, r)
    out = {}
    for form in (0, 1):
        P = oracle.make_params(2, dx, h, c0, 1.0, rho0=(rho0, rho0), eta=(eta, eta), n=2, tvf_alpha=0.0,
                               wall_form=form)
        out[form] = oracle.forces(P, pos, vel, rho, kind)
    assert a_p[0] > 0.0                                   # mirror: towards the wall at +x
    assert out[0]["a_p"][0, :2] == pytest.approx(a_p, rel=1e-13)
    assert np.all(out[1]["a_p"][0] == 0.0)
    for form in (0, 1):
        assert out[form]["a_v"][0, :2] == pytest.approx(a_v, rel=1e-13)
        assert out[form]["drho"][0] == pytest.approx(drho, rel=1e-13)


@pytest.mark.parametrize("u,a,rho_eps", [(0.5, 0.0, 0.0), (0.7, 0.2, 0.01), (3.0, 0.0, 0.0)])
def test_no_suction_wall_reading_keeps_pushing_pairs(u, a, rho_eps):
    # with P* > 0 (compression or approach) both wall readings give the
    # closed form of the mirror state
    dx, c0, rho0, eta = 0.1, 10.0, 1.0, 0.3
    h = 1.3 * dx
    r = 0.9 * dx
    pos = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    vel = np.array([[u, 0.25, 0.0], [a, -0.15, 0.0]])
    rho_i = rho0 * (1.0 + rho_eps)
    P = oracle.make_params(2, dx, h, c0, 1.0, rho0=(rho0, rho0), eta=(eta, eta), n=2, tvf_alpha=0.0, wall_form=1)
    out = oracle.forces(P, pos, vel, np.array([rho_i, rho0]), np.array([0, WALL], dtype=np.int32))
    a_p, _, _, _ = closed_form(u, 0.25, a, -0.15, rho_i, rho0, eta, c0, dx, h, r)
    assert a_p[0] < 0.0
    assert out["a_p"][0, :2] == pytest.approx(a_p, rel=1e-13, abs=1e-300)
