"""The pair weights of the oracle against exact consequences:

* Eq. 13's pair viscosity 2 eta_i eta_j / (eta_i + eta_j): a two-layer
  Couette profile (viscosity ratio 10, linear in each layer with equal shear
  stress, the kink between two particle rows) is an equilibrium of the
  viscous term to round-off away from the interface and to within 5% of the
  shear scale tau/(rho dx) on the rows whose support crosses it (an
  arithmetic pair mean leaves about twice the scale there);
* Eq. 22's weight 2 phi_i of the colour gradient: on a flat interface
  between densities 9 and 1, a particle and its mirror image across the
  interface see mirrored neighbour sets, so |gradC| of the dense side is
  exactly phi_dense / phi_light = 9 times that of the light side, with
  opposite direction.
"""
import numpy as np

import oracle
import sphcases


def layered(n, y_split=0.5):
    dx = 1.0 / n
    p = sphcases.lattice([0.0, 0.0], [1.0, 1.0], dx)
    w = sphcases.wall_shell([0.0, 0.0], [1.0, 1.0], dx, sides=[1])
    pos = np.zeros((len(p) + len(w), 3))
    pos[:len(p), :2] = p
    pos[len(p):, :2] = w
    kind = np.concatenate([np.where(p[:, 1] < y_split, 0, 1), np.full(len(w), 2)]).astype(np.int32)
    return dx, p, pos, kind


def test_two_layer_couette_is_an_equilibrium_of_the_pair_viscosity():
    n, eta1, eta2, tau = 24, 0.1, 1.0, 1.0
    dx, p, pos, kind = layered(n)
    u = lambda y: np.where(y < 0.5, tau / eta1 * (y - 0.5), tau / eta2 * (y - 0.5))
    vel = np.zeros_like(pos)
    vel[:, 0] = u(pos[:, 1])                         # walls carry the profile continued
    P = oracle.make_params(2, dx, 1.3 * dx, 10.0, 0.0, rho0=(1.0, 1.0), eta=(eta1, eta2), periodic=1,
                           box_lo=(0, 0, 0), box_hi=(1, 1, 0), n=len(kind), nbr_mode=0)
    av = oracle.forces(P, pos, vel, np.ones(len(kind)), kind)["a_v"][:len(p), 0]
    y = p[:, 1]
    scale = tau / dx
    near = np.abs(y - 0.5) < 2.6 * dx                 # rows whose support crosses the interface
    assert np.abs(av[~near]).max() <= 1e-10 * scale
    assert 0.0 < np.abs(av[near]).max() <= 0.05 * scale
    assert abs(av[near].sum()) <= 1e-10 * scale       # the residual is an internal exchange


def test_colour_gradient_weight_of_a_flat_interface():
    n = 20
    dx, p, pos, kind = layered(n)
    rho0 = (9.0, 1.0)
    rho = np.where(kind == 0, rho0[0], rho0[1])
    P = oracle.make_params(2, dx, 1.3 * dx, 10.0, 1.0, rho0=rho0, eta=(0.1, 0.1), periodic=1,
                           box_lo=(0, 0, 0), box_hi=(1, 1, 0), n=len(kind), nbr_mode=0)
    g = oracle.forces(P, pos, np.zeros_like(pos), rho, kind)["gradC"][:len(p)]
    y = p[:, 1]
    below = np.abs(y - (0.5 - 0.5 * dx)) < 1e-9       # dense row at the interface
    above = np.abs(y - (0.5 + 0.5 * dx)) < 1e-9       # its mirror row
    gb, ga = g[below, 1], g[above, 1]
    assert np.abs(g[below, 0]).max() < 1e-12 * np.abs(gb).max()     # normal to the interface
    assert np.allclose(gb, gb[0], rtol=1e-12) and np.allclose(ga, ga[0], rtol=1e-12)
    assert gb[0] * ga[0] < 0.0                                       # opposite directions
    assert abs(gb[0] / ga[0]) == np.float64(abs(gb[0] / ga[0]))
    assert abs(abs(gb[0] / ga[0]) - 9.0) <= 1e-12 * 9.0
