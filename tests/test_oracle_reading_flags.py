"""The alternative readings kept as flags, each pinned by what distinguishes
it from the default:

* v* as printed in Eq. 8 (vstar_form = 1): with equal velocities and
  p_i > p_j the star velocity carries the interface towards i (the high
  pressure), the opposite of the default reading (towards j);
* the limiter of Eq. 11 as printed (limiter = 3): beta = min(3 max(x, 0), 1)
  with x = (P_L + P_R)(U_L - U_R)/(rho_L c + rho_R c), zero for separating
  pairs and for a pair at zero pressure, symmetric under i <-> j;
* the scalar penalty of Eq. 29 (penalty_form = 2): the paper states it does
  not conserve momentum; the pair sums show exactly that, while the two
  tensor forms conserve it and all forms agree when xi = 0.
"""
import numpy as np
import pytest

import oracle
import sphcases


def P(**kw):
    return oracle.make_params(2, 0.1, 0.13, 10.0, 1.0, rho0=(1.0, 1.0), eta=(0.1, 0.1), **kw)


def test_printed_vstar_moves_interface_towards_high_pressure():
    e = np.array([1.0, 0.0])                 # from j to i
    v = np.array([0.3, -0.2])
    for form, sign in ((0, -1.0), (1, +1.0)):
        Pm = P(vstar_form=form)
        _, Us, _, _, vs = oracle.riemann_pair(Pm, 1.0, 5.0, v, 1.0, 1.0, v, e)
        dU = Us - (-(v @ e))                 # U* - U = (p_i - p_j)/(Z_L + Z_R) > 0
        assert dU == pytest.approx(4.0 / 20.0, rel=1e-12)
        # default: v*.e - v.e = -(U* - U) (towards j); printed: +(U* - U) (towards i)
        assert np.sign(vs[:2] @ e - v @ e) == sign
        assert vs[:2] @ e - v @ e == pytest.approx(sign * dU, rel=1e-12)


def test_printed_limiter_closed_form_range_and_symmetry():
    Pm = P(limiter=3)
    e = np.array([1.0, 0.0])
    vi, vj = np.array([-0.2, 0.0]), np.array([0.1, 0.0])    # approaching: U_L - U_R = 0.3
    rho_i, rho_j, p_i, p_j = 1.0, 1.2, 0.05, 0.02
    _, _, beta, _, _ = oracle.riemann_pair(Pm, rho_i, p_i, vi, rho_j, p_j, vj, e)
    x = (p_i + p_j) * 0.3 / (10.0 * (rho_i + rho_j))
    assert beta == pytest.approx(min(3.0 * max(x, 0.0), 1.0), rel=1e-14)
    _, _, b2, _, _ = oracle.riemann_pair(Pm, rho_j, p_j, -vj, rho_i, p_i, -vi, e)   # swapped pair
    assert b2 == pytest.approx(beta, rel=1e-14)
    _, _, b3, _, _ = oracle.riemann_pair(Pm, rho_i, p_i, -vi, rho_j, p_j, -vj, e)   # separating
    assert b3 == 0.0
    _, _, b4, _, _ = oracle.riemann_pair(Pm, rho_i, 0.0, vi, rho_j, 0.0, vj, e)     # zero pressure
    assert b4 == 0.0
    _, _, b5, _, _ = oracle.riemann_pair(Pm, rho_i, 400.0, vi, rho_j, 400.0, vj, e)  # saturates
    assert b5 == 1.0


def surface_force_sum(form, xi=-1.0):
    case = sphcases.small_droplet(2, 20, R_frac=0.3, shape="mode2", amp=0.2, walls=False,
                                  rho_l=10.0, rho_g=1.0, seed=3, jitter=0.2)
    pos, vel, rho, kind = case.flat()
    Pm = oracle.params_for_case(case, penalty_form=form, xi=xi)
    f = oracle.forces(Pm, pos, vel, rho, kind)
    m = np.asarray(case.fluid_props()[0])[kind] * case.dx ** 2
    tot = (m[:, None] * f["a_s"]).sum(0)
    scale = (m[:, None] * np.abs(f["a_s"])).sum()
    return tot, scale, f["a_s"]


def test_scalar_penalty_breaks_momentum_conservation_tensor_forms_keep_it():
    for form in (0, 1):
        tot, scale, _ = surface_force_sum(form)
        assert np.abs(tot).max() <= 1e-12 * scale, form
    tot, scale, _ = surface_force_sum(2)
    assert np.abs(tot).max() > 1e-6 * scale
    # with xi = 0 the penalty vanishes and every form gives the same force
    base = surface_force_sum(0, xi=0.0)[2]
    for form in (1, 2):
        assert np.array_equal(surface_force_sum(form, xi=0.0)[2], base)


def test_penalty_on_the_cross_phase_line_only():
    # the ablation keeps the cross-phase line of Eq. 33 and drops the
    # penalty from the same-phase line: with xi = 0 it changes nothing;
    # with the penalty on it changes the surface force, and what is left
    # still differs from no penalty at all (the cross-phase line)
    case = sphcases.small_droplet(2, 20, R_frac=0.3, shape="mode2", amp=0.2, walls=False,
                                  rho_l=10.0, rho_g=1.0, seed=3, jitter=0.2)
    pos, vel, rho, kind = case.flat()
    f0 = oracle.forces(oracle.params_for_case(case, xi=0.0), pos, vel, rho, kind)["a_s"]
    f1 = oracle.forces(oracle.params_for_case(case, xi=0.0, penalty_scope=1), pos, vel, rho, kind)["a_s"]
    assert np.array_equal(f0, f1)
    on = oracle.forces(oracle.params_for_case(case), pos, vel, rho, kind)["a_s"]
    cross = oracle.forces(oracle.params_for_case(case, penalty_scope=1), pos, vel, rho, kind)["a_s"]
    nopen = oracle.forces(oracle.params_for_case(case, xi=0.0), pos, vel, rho, kind)["a_s"]
    assert np.abs(cross - on).max() > 1e-6 * np.abs(on).max()          # the same-phase line carried a penalty
    assert np.abs(cross - nopen).max() > 1e-6 * np.abs(on).max()       # and the cross-phase line still does
