"""GPU edge cases against the FP64 oracle and the exact answers the method
has for them: one fluid phase (every surface term vanishes), fluid at rest
(stays at rest; the substep count follows the clipping of Eqs. 16-18), a
lone particle (no neighbours: it drifts at its velocity), a handful of
particles split over four or eight lanes each in 32-thread blocks (a
ragged, mostly empty tile), coincident particles (reported, not divided
by), and the closed forms of an isolated cross-phase pair and of a fluid
particle beside a wall particle."""
import numpy as np
import pytest

import oracle
import sphcases

pytestmark = pytest.mark.gpu

S = pytest.importorskip("paper_2503_16082_gb300")


def run_both(case, precision, n_adv, **kw):
    h = S.case_from_spec(case, precision=precision, **kw)
    try:
        info = S.step(h, n_adv)
        g = {k: S.read_fields(h, f, case.dim) for k, f in (("pos", S.FIELD_POS), ("vel", S.FIELD_VEL),
                                                           ("rho", S.FIELD_RHO), ("gradC", S.FIELD_GRADC))}
    finally:
        S.destroy(h)
    pos, vel, rho, kind = case.flat()
    P = oracle.params_for_case(case)
    p1, v1, r1, oinfo, gC, _ = oracle.run(P, pos, vel, rho, kind, n_adv)
    d = case.dim
    o = {"pos": p1[:, :d], "vel": v1[:, :d], "rho": r1, "gradC": gC[:, :d]}
    return g, o, info, oinfo, pos[:, :d], kind


def close(a, b, tol):
    scale = np.abs(b).max()
    return np.abs(a - b).max() <= tol * max(scale, 1e-300)


def one_phase(dim, n_side, jitter, vel_amp, seed=5):
    dx = 1.0 / n_side
    lo, hi = [0.0] * dim, [1.0] * dim
    p = sphcases.lattice(lo, hi, dx)
    rng = np.random.default_rng(seed)
    p = p + rng.uniform(-jitter, jitter, p.shape) * dx
    vel = rng.uniform(-vel_amp, vel_amp, p.shape) if vel_amp > 0 else None
    phases = [sphcases.Phase("fluid", p, rho0=1.0, eta=0.01, vel=vel),
              sphcases.Phase("wall", sphcases.wall_shell(lo, hi, dx))]
    case = sphcases.Case(name="one_phase", dim=dim, lo=lo, hi=hi, dx=dx, gamma=1.0, c0=10.0,
                         h_factor=1.3, xi=-1.0, phases=phases)
    if dim == 3:
        case.cfl_ac = 0.4
    return case


@pytest.mark.parametrize("dim", [2, 3])
def test_one_fluid_phase_against_oracle(dim):
    case = one_phase(dim, 20 if dim == 2 else 10, 0.15, 0.1)
    g, o, info, oinfo, pos0, kind = run_both(case, 64, 1)
    assert info["n_sub"] == oinfo["n_sub"] > 1
    assert np.all(g["gradC"] == 0.0)                   # Eq. 22 sums over the other fluid only
    fl = kind < 2
    assert close(g["pos"][fl] - pos0[fl], o["pos"][fl] - pos0[fl], 1e-12)
    assert close(g["vel"][fl], o["vel"][fl], 1e-12)
    assert close(g["rho"][fl] - 1.0, o["rho"][fl] - 1.0, 1e-12)


@pytest.mark.parametrize("precision", [32, 64])
def test_fluid_at_rest_stays_at_rest(precision):
    # a perfect lattice at rest inside its wall lattice: no pressure, no
    # viscous force, a transport shift that cancels; the advection step has
    # no velocity term, so the substeps follow the acoustic and surface
    # criteria and the last one is clipped exactly as in the oracle
    case = one_phase(2, 16, 0.0, 0.0)
    h = S.case_from_spec(case, precision=precision)
    info = S.step(h, 2)
    vel = S.read_fields(h, S.FIELD_VEL, 2)
    pos = S.read_fields(h, S.FIELD_POS, 2)
    S.destroy(h)
    pos0, vel0, rho0, kind = case.flat()
    P = oracle.params_for_case(case)
    _, _, _, oinfo, _, _ = oracle.run(P, pos0, vel0, rho0, kind, 2)
    assert info["n_sub"] == oinfo["n_sub"]
    assert info["t"] == pytest.approx(oinfo["t"], rel=1e-12)
    eps = 1e-12 if precision == 64 else 1e-5
    assert np.abs(vel).max() <= eps * case.c0
    assert np.abs(pos - pos0[:, :2]).max() <= eps * case.dx


@pytest.mark.parametrize("precision", [32, 64])
def test_lone_particle_drifts_at_its_velocity(precision):
    dim = 2
    v = np.array([[0.02, -0.01]])
    phases = [sphcases.Phase("fluid", np.array([[0.5, 0.5]]), rho0=1.0, eta=0.01, vel=v)]
    case = sphcases.Case(name="lone", dim=dim, lo=[0.0, 0.0], hi=[1.0, 1.0], dx=0.05, gamma=1.0,
                         c0=10.0, h_factor=1.3, xi=-1.0, phases=phases)
    h = S.case_from_spec(case, precision=precision)
    info = S.step(h, 3)
    pos = S.read_fields(h, S.FIELD_POS, dim)
    vel = S.read_fields(h, S.FIELD_VEL, dim)
    rho = S.read_fields(h, S.FIELD_RHO, dim)
    S.destroy(h)
    assert info["n_sub"] > 0 and info["t"] > 0
    # no neighbour, no force: the velocity keeps its stored value exactly
    assert np.array_equal(vel, v if precision == 64 else v.astype(np.float32).astype(np.float64))
    assert rho[0] == 1.0
    # x = x0 + v t up to the rounding of n_sub drift steps (FP32: of a
    # cell-relative position)
    tol = 1e-10 if precision == 64 else 1e-3
    assert np.abs(pos - (0.5 + v * info["t"])).max() <= tol * np.abs(v * info["t"]).max()


@pytest.mark.parametrize("lanes", [1, 4, 8])
def test_handful_of_particles_ragged_tile(lanes):
    # nine fluid particles of two phases in 32-thread blocks split over
    # L lanes each: one tile, mostly empty, every lane group ragged
    rng = np.random.default_rng(9)
    dx = 0.05
    base = np.array([[0.5, 0.5]]) + dx * np.array([[i, j] for i in range(3) for j in range(3)])
    p = base + rng.uniform(-0.1, 0.1, base.shape) * dx
    vel = rng.uniform(-0.05, 0.05, p.shape)
    inner = np.zeros(len(p), bool)
    inner[4] = True
    phases = [sphcases.Phase("fluid", p[inner], rho0=1000.0, eta=0.1, vel=vel[inner]),
              sphcases.Phase("fluid", p[~inner], rho0=1.0, eta=0.001, vel=vel[~inner])]
    case = sphcases.Case(name="handful", dim=2, lo=[0.0, 0.0], hi=[1.0, 1.0], dx=dx, gamma=1.0,
                         c0=10.0, h_factor=1.3, xi=-1.0, phases=phases)
    g, o, info, oinfo, pos0, kind = run_both(case, 64, 1, lanes=lanes, block=32)
    assert info["n_sub"] == oinfo["n_sub"]
    assert np.abs(o["gradC"]).max() > 0
    for key in ("vel", "gradC"):
        assert close(g[key], o[key], 1e-12), key
    assert close(g["pos"] - pos0, o["pos"] - pos0, 1e-12)


def test_coincident_particles_are_reported():
    case = one_phase(2, 12, 0.0, 0.0)
    fl = case.phases[0]
    fl.pos = np.vstack([fl.pos, fl.pos[:1]])            # a second particle on the first
    h = S.case_from_spec(case, precision=64)
    info = S.step(h, 1, check=False)
    assert info["rc"] == S.ERR_COINCIDENT
    assert S.case_info(h)["status"] == S.ERR_COINCIDENT
    S.destroy(h)


def test_isolated_cross_phase_pair_first_substep():
    # two particles of different fluids at rest, viscous enough that one
    # advection step is one substep: v after it is dt times the penalty
    # acceleration of the hand-reduced Eqs. 22-33,
    # a_i = -(4 phi_i phi_j xi gamma / (rho_i r)) (1 - |W'| V r) W' V e_ij
    import math
    dx, rho_a, rho_b, gamma, r = 0.1, 10.0, 1.0, 1.0, 0.1
    h = 1.3 * dx
    case = sphcases.Case(name="pair", dim=2, lo=[0.0, 0.0], hi=[1.0, 1.0], dx=dx, gamma=gamma, c0=10.0,
                         h_factor=1.3, xi=-1.0,
                         phases=[sphcases.Phase("fluid", np.array([[0.5, 0.5]]), rho0=rho_a, eta=50.0),
                                 sphcases.Phase("fluid", np.array([[0.5 + r, 0.5]]), rho0=rho_b, eta=5.0)])
    h_ = S.case_from_spec(case, precision=64)
    try:
        info = S.step(h_, 1)
        vel = S.read_fields(h_, S.FIELD_VEL, 2)
    finally:
        S.destroy(h_)
    assert info["n_sub"] == 1
    a = 7.0 / (4.0 * math.pi * h * h)
    q = r / h
    dW = -5.0 * a * q * (1.0 - q / 2.0) ** 3 / h
    xi = 1.3 * math.log10(rho_a / rho_b) + 0.6
    phi_i, phi_j, V = rho_a / (rho_a + rho_b), rho_b / (rho_a + rho_b), dx * dx
    coef = -4.0 * phi_i * phi_j * xi * gamma / r * (1.0 - abs(dW) * V * r)
    want_i = info["t"] * coef * dW * V / rho_a * -1.0          # x component; e_ij = (-1, 0)
    want_j = info["t"] * coef * dW * V / rho_b
    assert vel[0, 0] == pytest.approx(want_i, rel=1e-12)
    assert vel[1, 0] == pytest.approx(want_j, rel=1e-12)
    assert abs(vel[0, 1]) < 1e-15 and abs(vel[1, 1]) < 1e-15


@pytest.mark.parametrize("u,a,rho_eps", [(0.7, 0.2, 0.01), (3.0, 0.0, 0.0)])
def test_fluid_particle_beside_a_wall_particle_first_substep(u, a, rho_eps):
    # one fluid particle and one wall particle, viscous enough that one
    # advection step is one substep: v after it is v0 + dt (a_p + a_v) of
    # the hand-reduced wall reading (mirror state U_R = 2 U_w - U_L, Eq. 11's
    # limiter at beta = 0.3 and clipped at 1, Eq. 13 with eta_i and v_i - v_w),
    # and rho after it follows Eq. 6 with v* = v_w and the kicked velocity
    import math
    dx, c0, rho0, eta, r = 0.1, 10.0, 1.0, 50.0, 0.09
    h = 1.3 * dx
    w, b = 0.25, -0.15
    case = sphcases.Case(name="wall_pair", dim=2, lo=[0.0, 0.0], hi=[1.0, 1.0], dx=dx, gamma=1.0, c0=c0,
                         h_factor=1.3, xi=-1.0,
                         phases=[sphcases.Phase("fluid", np.array([[0.5, 0.5]]), rho0=rho0, eta=eta,
                                                vel=np.array([[u, w]]), rho=np.array([rho0 * (1.0 + rho_eps)])),
                                 sphcases.Phase("wall", np.array([[0.5 + r, 0.5]]), wall_vel=(a, b, 0.0))])
    h_ = S.case_from_spec(case, precision=64)
    try:
        info = S.step(h_, 1)
        vel = S.read_fields(h_, S.FIELD_VEL, 2)
        rho = S.read_fields(h_, S.FIELD_RHO, 2)
    finally:
        S.destroy(h_)
    assert info["n_sub"] == 1
    dt = info["t"]
    q = r / h
    dW = -5.0 * 7.0 / (4.0 * math.pi * h * h) * q * (1.0 - q / 2.0) ** 3 / h
    V = dx * dx
    rho_i = rho0 * (1.0 + rho_eps)
    dU = 2.0 * (u - a)
    beta = min(3.0 * max(dU / c0, 0.0), 1.0)
    Ps = c0 * c0 * (rho_i - rho0) + beta * rho_i * c0 * dU / 2.0
    e = np.array([-1.0, 0.0])
    vij = np.array([u - a, w - b])
    acc = -(2.0 / rho_i) * Ps * dW * e * V + (2.0 / rho_i) * eta * vij / r * dW * V
    v1 = np.array([u, w]) + dt * acc
    assert vel[0] == pytest.approx(v1, rel=1e-12)
    assert np.array_equal(vel[1], [a, b])                      # the wall keeps its velocity
    drho = 2.0 * rho_i * float((v1 - np.array([a, b])) @ e) * dW * V
    assert rho[0] - rho_i == pytest.approx(dt * drho, rel=1e-10)
