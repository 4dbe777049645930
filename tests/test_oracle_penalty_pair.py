"""The surface stress and penalty of Eqs. 24-33 reduced by hand for an
isolated pair of particles of different fluids, at rest (no pressure, no
viscous force).  Each particle's colour gradient comes from the other one
alone, so both normals lie along the pair axis: the stresses Pi vanish on
that axis, N-bar = e e^T, grad C-bar = (1/2)(grad C_i - grad C_j) has length
|W'| V (phi_i + phi_j = 1), and C-hat e = (1 - |W'| V r) e for both tensor
readings of Eq. 30.  What is left is the penalty term of the cross-phase
line of Eq. 33:

    a_i = -(4 phi_i phi_j xi gamma / (rho_i r)) (1 - |W'| V r) W' V e_ij,

a repulsion along the axis, and m_i a_i + m_j a_j = 0.  A transposed
projector, a wrong sign in grad C-bar or in C-hat, or the phi weights
swapped all change it."""
import math

import numpy as np
import pytest

import oracle


def wendland_dW(h, r):
    a = 7.0 / (4.0 * math.pi * h * h)
    q = r / h
    return -5.0 * a * q * (1.0 - q / 2.0) ** 3 / h


@pytest.mark.parametrize("penalty_form", [0, 1])
@pytest.mark.parametrize("r_over_dx", [0.8, 1.0, 1.7])
def test_isolated_cross_phase_pair(penalty_form, r_over_dx):
    dx, rho_a, rho_b, gamma = 0.1, 10.0, 1.0, 1.0
    h = 1.3 * dx
    r = r_over_dx * dx
    pos = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    kind = np.array([0, 1], dtype=np.int32)
    rho = np.array([rho_a, rho_b])
    P = oracle.make_params(2, dx, h, 10.0, gamma, rho0=(rho_a, rho_b), eta=(0.1, 0.01), n=2,
                           penalty_form=penalty_form, tvf_alpha=0.0)
    out = oracle.forces(P, pos, np.zeros((2, 3)), rho, kind)
    assert np.abs(out["a_p"]).max() == 0.0 and np.abs(out["a_v"]).max() == 0.0
    xi = 1.3 * math.log10(rho_a / rho_b) + 0.6
    phi_i, phi_j = rho_a / (rho_a + rho_b), rho_b / (rho_a + rho_b)
    V = dx * dx                                   # m / rho at rest
    dW = wendland_dW(h, r)
    # grad C_i = 2 phi_i W' e_ij V, e_ij = (-1, 0): along +x
    assert out["gradC"][0, :2] == pytest.approx([2.0 * phi_i * abs(dW) * V, 0.0], rel=1e-13, abs=1e-300)
    assert out["gradC"][1, :2] == pytest.approx([-2.0 * phi_j * abs(dW) * V, 0.0], rel=1e-13, abs=1e-300)
    coef = -4.0 * phi_i * phi_j * xi * gamma / r * (1.0 - abs(dW) * V * r)
    a_i = coef * dW * V / rho_a * np.array([-1.0, 0.0])
    a_j = coef * dW * V / rho_b * np.array([1.0, 0.0])
    assert out["a_s"][0, :2] == pytest.approx(a_i, rel=1e-12, abs=1e-12 * abs(a_i[0]))
    assert out["a_s"][1, :2] == pytest.approx(a_j, rel=1e-12, abs=1e-12 * abs(a_j[0]))
    # momentum: m_i a_i + m_j a_j = 0 (m = rho0 V)
    assert rho_a * out["a_s"][0, 0] + rho_b * out["a_s"][1, 0] == pytest.approx(0.0, abs=1e-12 * rho_a * abs(a_i[0]))
