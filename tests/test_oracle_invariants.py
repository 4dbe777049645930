"""Invariants of the oracle's pair sums: momentum conservation of every
pairwise force (Sections 3.1, 4.1, 4.2), Galilean invariance, rotation
covariance, the colour-gradient zero modes of Section 4.2 (Fig. 2), and the
lattice identities behind the correction matrix (Eq. 15)."""
import math

import numpy as np
import pytest

import oracle
import sphcases


def blob(dim, **kw):
    case = sphcases.free_blob(dim=dim, n_side=14 if dim == 2 else 8, **kw)
    pos, vel, rho, kind = case.flat()
    return case, pos, vel, rho, kind


def masses(case, kind):
    rho0, _ = case.fluid_props()
    return np.asarray(rho0)[kind] * case.dx ** case.dim


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("opts", [{}, {"penalty_form": 1}, {"grad_mode": 1}, {"limiter": 1}, {"xi": 0.0},
                                  {"penalty_scope": 1}])
def test_momentum_conserved_by_each_force(dim, opts):
    case, pos, vel, rho, kind = blob(dim)
    P = oracle.params_for_case(case, **opts)
    f = oracle.forces(P, pos, vel, rho, kind)
    m = masses(case, kind)
    for key in ("a_p", "a_s", "a_v"):
        F = m[:, None] * f[key]
        scale = np.abs(F).sum()
        assert scale > 0
        assert np.abs(F.sum(0)).max() <= 1e-12 * scale, key


@pytest.mark.parametrize("dim", [2, 3])
def test_galilean_invariance(dim):
    case, pos, vel, rho, kind = blob(dim)
    P = oracle.params_for_case(case)
    a = oracle.forces(P, pos, vel, rho, kind)
    u0 = np.zeros(3)
    u0[:dim] = [0.7, -1.3, 0.4][:dim]
    b = oracle.forces(P, pos, vel + u0, rho, kind)
    for key in ("gradC", "a_p", "a_s", "a_v", "drho", "dr"):
        scale = np.abs(a[key]).max()
        assert np.abs(a[key] - b[key]).max() <= 1e-10 * scale, key


def rotation(dim):
    if dim == 2:
        t = 0.37
        R = np.eye(3)
        R[:2, :2] = [[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]]
        return R
    a, b, c = 0.3, -0.8, 1.1
    Rx = np.array([[1, 0, 0], [0, math.cos(a), -math.sin(a)], [0, math.sin(a), math.cos(a)]])
    Ry = np.array([[math.cos(b), 0, math.sin(b)], [0, 1, 0], [-math.sin(b), 0, math.cos(b)]])
    Rz = np.array([[math.cos(c), -math.sin(c), 0], [math.sin(c), math.cos(c), 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


@pytest.mark.parametrize("dim", [2, 3])
def test_rotation_covariance(dim):
    case, pos, vel, rho, kind = blob(dim)
    P = oracle.params_for_case(case)
    R = rotation(dim)
    a = oracle.forces(P, pos, vel, rho, kind)
    b = oracle.forces(P, pos @ R.T, vel @ R.T, rho, kind)
    for key in ("gradC", "a_p", "a_s", "a_v", "dr"):
        scale = np.abs(a[key]).max()
        assert np.abs(a[key] @ R.T - b[key]).max() <= 1e-9 * scale, key
    assert np.abs(a["drho"] - b["drho"]).max() <= 1e-9 * np.abs(a["drho"]).max()


def lattice_case(dim, m, phase_fn):
    dx = 1.0 / m
    g = sphcases.lattice([0.0] * dim, [1.0] * dim, dx)
    pos = np.zeros((len(g), 3))
    pos[:, :dim] = g
    kind = phase_fn(g).astype(np.int32)
    rho = np.where(kind == 0, 1000.0, 1.0)
    P = oracle.make_params(dim, dx, 1.3 * dx, 10.0, 1.0, rho0=(1000.0, 1.0), eta=(0.1, 0.001))
    return P, pos, np.zeros_like(pos), rho, kind, dx


def interior(pos, dim, margin):
    return np.all((pos[:, :dim] > margin) & (pos[:, :dim] < 1 - margin), axis=1)


@pytest.mark.parametrize("dim", [2, 3])
def test_bulk_colour_gradient_is_exactly_zero(dim):
    P, pos, vel, rho, kind, dx = lattice_case(dim, 20 if dim == 2 else 10,
                                              lambda g: (g[:, 0] > 0.5).astype(int))
    f = oracle.forces(P, pos, vel, rho, kind)
    far = np.abs(pos[:, 0] - 0.5) > 2 * 1.3 * dx
    assert np.all(f["gradC"][far] == 0.0)
    near = np.abs(pos[:, 0] - 0.5) < 2 * dx      # a cross-phase neighbour within 2 dx
    assert np.all(np.linalg.norm(f["gradC"][near], axis=1) > 0)


def test_checkerboard_zero_surface_energy_mode():
    # Fig. 2b of Section 4.2: every other-phase neighbour has a mirror partner,
    # so the colour gradient cancels exactly although the phases interleave.
    m = 20
    P, pos, vel, rho, kind, dx = lattice_case(
        2, m, lambda g: ((np.floor(g[:, 0] * m) + np.floor(g[:, 1] * m)) % 2).astype(int))
    f = oracle.forces(P, pos, vel, rho, kind)
    inner = interior(pos, 2, 3 * dx)
    g = np.linalg.norm(f["gradC"][inner], axis=1)
    assert g.max() * 1.3 * dx < 1e-10


def test_isolated_foreign_particle_is_invisible_to_colour_gradient():
    m = 15
    P, pos, vel, rho, kind, dx = lattice_case(2, m, lambda g: np.zeros(len(g), dtype=int))
    c = np.argmin(np.linalg.norm(pos[:, :2] - 0.5, axis=1))
    kind[c] = 1
    rho[c] = 1.0
    f = oracle.forces(P, pos, vel, rho, kind)
    assert np.linalg.norm(f["gradC"][c]) * 1.3 * dx < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_lattice_moment_identity_and_tvf(dim):
    # sum_j r_ij (x) grad_i W_ij V_j tends to -I on a full lattice (integration
    # by parts of the kernel), hence B = I and the transport shift vanishes.
    m = 16 if dim == 2 else 13
    P, pos, vel, rho, kind, dx = lattice_case(dim, m, lambda g: np.zeros(len(g), dtype=int))
    counts, idx = oracle.neighbors(P, pos)
    c = np.argmin(np.linalg.norm(pos[:, :dim] - 0.5 - 0.5 / m, axis=1))
    start = counts[:c].sum()
    M = np.zeros((3, 3))
    V = dx ** dim
    for j in idx[start:start + counts[c]]:
        r = pos[c] - pos[j]
        rn = np.linalg.norm(r)
        M += np.outer(r, oracle.kernel_dW(dim, P.h, rn) * r / rn) * V
    assert np.abs(M[:dim, :dim] + np.eye(dim)).max() < 5e-2   # lattice sum vs integral, h = 1.3 dx
    f = oracle.forces(P, pos, vel, rho, kind)
    inner = interior(pos, dim, 5.5 * dx)     # neighbours' neighbours have full support
    assert inner.sum() > 0
    assert np.abs(f["dr"][inner]).max() < 1e-14


@pytest.mark.parametrize("dim", [2, 3])
def test_tvf_pushes_displaced_particle_back(dim):
    # sign reading of Eq. 14: a particle nudged towards a neighbour is moved
    # back, away from the side where its neighbours crowd.
    m = 16 if dim == 2 else 9
    P, pos, vel, rho, kind, dx = lattice_case(dim, m, lambda g: np.zeros(len(g), dtype=int))
    c = np.argmin(np.linalg.norm(pos[:, :dim] - 0.5 - 0.5 / m, axis=1))
    delta = np.zeros(3)
    delta[:dim] = 0.15 * dx * np.array([1.0, 0.4, -0.3])[:dim]
    pos[c] += delta
    f = oracle.forces(P, pos, vel, rho, kind)
    dr = f["dr"][c]
    assert dr @ delta < 0
    assert np.linalg.norm(dr) < np.linalg.norm(delta)
