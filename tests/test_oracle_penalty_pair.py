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


# ---------------------------------------------------------------------------
# The same-phase line of Eq. 33, S_ij e = (Pi_i + Pi_j) e + xi gamma T-bar C-hat e / r
# (C_ij = 0), through the oracle's pair entry point, which is the routine its
# force loop calls for every fluid pair.  For a pair of one phase with
# colour gradients G_i n_i and G_j n_j, Eqs. 24-30 reduce by hand to:
#   Pi e = gamma G (e - n (n.e));  grad C-bar = (G_i n_i + G_j n_j) / 2;
#   C-hat e = -r |grad C-bar| (nbar.e) nbar      (contraction A A^T / |A|, the default)
#           = -r |grad C-bar| e                  (A^T A / |A|, penalty_form 1)
#           = -r (grad C-bar . e) e              (the scalar Eq. 29, penalty_form 2);
#   T-bar c = c - (n_i (n_i.c) + n_j (n_j.c)) / 2.
# Three configurations give closed forms that do not repeat those steps:
# ---------------------------------------------------------------------------
def rotation(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    return q * np.sign(np.linalg.det(q))


SAME_PHASE_GAMMA, SAME_PHASE_XI = 0.7, 2.5


def same_phase_params(dim, form):
    return oracle.make_params(dim, 0.1, 0.13, 10.0, SAME_PHASE_GAMMA, rho0=(3.0, 1.0), eta=(0.1, 0.1),
                              xi=SAME_PHASE_XI, penalty_form=form)


@pytest.mark.parametrize("form", [0, 1, 2])
@pytest.mark.parametrize("kind", [0, 1])
def test_same_phase_normals_across_the_pair(form, kind):
    """n_i = n_j = n perpendicular to e: the stresses pass e unchanged,
    grad C-bar has no component along e, so the default and the scalar
    contraction give no penalty while A^T A/|A| repels along the pair:
    S e = gamma (G_i + G_j) e, times (1 - xi/2) for A^T A/|A|."""
    g, xi = SAME_PHASE_GAMMA, SAME_PHASE_XI
    for dim, R in ((2, np.eye(3)), (3, rotation(3))):
        P = same_phase_params(dim, form)
        n, e = R @ np.array([0.0, 1.0, 0.0]), R @ np.array([1.0, 0.0, 0.0])
        Gi, Gj, r = 4.0, 2.5, 0.11
        out = oracle.surface_pair(P, kind, kind, (Gi * n)[:dim], (Gj * n)[:dim], e[:dim], r)
        want = g * (Gi + Gj) * (1.0 - xi / 2.0 if form == 1 else 1.0) * e[:dim]
        assert out == pytest.approx(want, rel=1e-13, abs=1e-13 * np.abs(want).max())


@pytest.mark.parametrize("form", [0, 1, 2])
@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_same_phase_normals_along_the_pair(form, sign):
    """n_i = n_j = n = +-e: Pi e = 0 and C-hat e lies along n, which T-bar
    removes, for every contraction: S e = 0 (the projection of Eq. 33 keeps
    the same-phase penalty tangential)."""
    for dim, R in ((2, np.eye(3)), (3, rotation(4))):
        P = same_phase_params(dim, form)
        e = R @ np.array([1.0, 0.0, 0.0])
        n = sign * e
        out = oracle.surface_pair(P, 0, 0, (3.0 * n)[:dim], (1.2 * n)[:dim], e[:dim], 0.09)
        assert np.abs(out).max() <= 1e-14


@pytest.mark.parametrize("form", [0, 1, 2])
@pytest.mark.parametrize("alpha,beta", [(0.4, 0.0), (0.9, 0.3), (0.25, 1.2), (1.1, -0.7)])
def test_same_phase_mirrored_normals(form, alpha, beta):
    """n_i = (cos a, sin a), n_j = (cos a, -sin a), G_i = G_j = G and
    e = (cos b, sin b) in a plane: grad C-bar = G cos a x, T-bar x =
    sin^2 a x and T-bar e = (sin^2 a cos b, cos^2 a sin b), so
      A A^T/|A|:  S e = gamma G (sin^2 a cos b (2 - xi cos a), 2 cos^2 a sin b)
      A^T A/|A|:  S e = gamma G (2 - xi cos a) (sin^2 a cos b, cos^2 a sin b)
      scalar:     S e = gamma G (2 - xi cos a cos b) (sin^2 a cos b, cos^2 a sin b)."""
    g, xi, G, r = SAME_PHASE_GAMMA, SAME_PHASE_XI, 3.3, 0.07
    ca, sa, cb, sb = math.cos(alpha), math.sin(alpha), math.cos(beta), math.sin(beta)
    if form == 0:
        want2 = g * G * np.array([sa * sa * cb * (2.0 - xi * ca), 2.0 * ca * ca * sb])
    elif form == 1:
        want2 = g * G * (2.0 - xi * ca) * np.array([sa * sa * cb, ca * ca * sb])
    else:
        want2 = g * G * (2.0 - xi * ca * cb) * np.array([sa * sa * cb, ca * ca * sb])
    for dim, R in ((2, np.eye(3)), (3, rotation(5))):
        P = same_phase_params(dim, form)
        ni = R @ np.array([ca, sa, 0.0])
        nj = R @ np.array([ca, -sa, 0.0])
        e = R @ np.array([cb, sb, 0.0])
        want = (R @ np.array([want2[0], want2[1], 0.0]))[:dim]
        out = oracle.surface_pair(P, 1, 1, (G * ni)[:dim], (G * nj)[:dim], e[:dim], r)
        assert out == pytest.approx(want, rel=1e-12, abs=1e-12 * g * G)


def test_same_phase_penalty_scope_and_xi():
    """The same-phase penalty is the only difference between xi = 0, the
    printed scope and the cross-phase-only ablation: with the mirrored
    normals the three give 2 gamma G sin^2 a cos b x-components
    (xi = 0 and cross-only) and the full closed form (printed scope)."""
    G, r, alpha = 2.0, 0.05, 0.6
    ni = np.array([math.cos(alpha), math.sin(alpha)])
    nj = np.array([math.cos(alpha), -math.sin(alpha)])
    e = np.array([1.0, 0.0])
    base = dict(rho0=(3.0, 1.0), eta=(0.1, 0.1))
    full = oracle.surface_pair(oracle.make_params(2, 0.1, 0.13, 10.0, 1.0, xi=2.0, **base), 0, 0, G * ni, G * nj, e, r)
    zero = oracle.surface_pair(oracle.make_params(2, 0.1, 0.13, 10.0, 1.0, xi=0.0, **base), 0, 0, G * ni, G * nj, e, r)
    cross = oracle.surface_pair(oracle.make_params(2, 0.1, 0.13, 10.0, 1.0, xi=2.0, penalty_scope=1, **base),
                                0, 0, G * ni, G * nj, e, r)
    s2 = math.sin(alpha) ** 2
    assert zero == pytest.approx([2.0 * G * s2, 0.0], abs=1e-14)
    assert cross == pytest.approx(zero, abs=1e-15)
    assert full == pytest.approx([G * s2 * (2.0 - 2.0 * math.cos(alpha)), 0.0], abs=1e-14)


def test_force_loop_uses_the_pair_term():
    """Wiring: on a small mixed cluster at rest, each particle's a^s from the
    force loop equals the sum over its neighbours of the pair entry point's
    S_ij e_ij times W'(r) V_j / rho_i (with the loop's own colour
    gradients)."""
    rng = np.random.default_rng(8)
    dx = 0.1
    h = 1.3 * dx
    pos = np.zeros((12, 3))
    pos[:, :2] = rng.uniform(0.0, 3 * dx, size=(12, 2))
    kind = np.array([0] * 7 + [1] * 5, dtype=np.int32)
    rho = np.where(kind == 0, 5.0, 1.0) * (1.0 + 0.01 * rng.normal(size=12))
    P = oracle.make_params(2, dx, h, 10.0, 0.8, rho0=(5.0, 1.0), eta=(0.1, 0.01), n=12, tvf_alpha=0.0)
    out = oracle.forces(P, pos, np.zeros((12, 3)), rho, kind)
    gC = out["gradC"]
    mass = np.where(kind == 0, 5.0, 1.0) * dx * dx
    for i in range(12):
        a = np.zeros(2)
        for j in range(12):
            rv = pos[i, :2] - pos[j, :2]
            r = float(np.linalg.norm(rv))
            if j == i or not (0.0 < r < 2 * h):
                continue
            Se = oracle.surface_pair(P, kind[i], kind[j], gC[i, :2], gC[j, :2], rv / r, r)
            a += Se * oracle.kernel_dW(2, h, r) * (mass[j] / rho[j]) / rho[i]
        assert out["a_s"][i, :2] == pytest.approx(a, rel=1e-11, abs=1e-12 * max(np.abs(out["a_s"]).max(), 1e-300))


# ---------------------------------------------------------------------------
# The stresses of the cross-phase line of Eq. 33 (Eq. 26 with the penalty
# off, xi = 0): S_ij e = w_i Pi_i e + w_j Pi_j e with Pi e = gamma G (e - n (n.e))
# (Eq. 24).  As printed w_i = 2 phi_j, w_j = 2 phi_i (phi of Eq. 23); the
# reading stress_weights = 1 takes each stress with its own particle's weight,
# w_i = 2 phi_i, w_j = 2 phi_j.  Normals at an angle to e so that both stresses
# act; fluids of rest density 3 and 1, so the two weights differ.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("weights", [0, 1])
def test_cross_phase_stress_weights(weights):
    g = 0.9
    rho_a, rho_b = 3.0, 1.0
    for dim, R in ((2, np.eye(3)), (3, rotation(5))):
        P = oracle.make_params(dim, 0.1, 0.13, 10.0, g, rho0=(rho_a, rho_b), eta=(0.1, 0.1), xi=0.0,
                               stress_weights=weights)
        e = R @ np.array([1.0, 0.0, 0.0])
        a_i, a_j = 0.4, 1.1                           # angles of n_i, n_j from e
        n_i = R @ np.array([math.cos(a_i), math.sin(a_i), 0.0])
        n_j = R @ np.array([math.cos(a_j), -math.sin(a_j), 0.0])
        Gi, Gj, r = 3.0, 1.7, 0.09
        for ki, kj in ((0, 1), (1, 0)):
            out = oracle.surface_pair(P, ki, kj, (Gi * n_i)[:dim], (-Gj * n_j)[:dim], e[:dim], r)
            phi = {0: rho_a / (rho_a + rho_b), 1: rho_b / (rho_a + rho_b)}
            w_i, w_j = (2 * phi[ki], 2 * phi[kj]) if weights else (2 * phi[kj], 2 * phi[ki])
            pi_e = g * Gi * (e - n_i * (n_i @ e))
            pj_e = g * Gj * (e - n_j * (n_j @ e))     # the sign of grad C_j drops out of Pi_j
            want = (w_i * pi_e + w_j * pj_e)[:dim]
            assert out == pytest.approx(want, rel=1e-13, abs=1e-13 * np.abs(want).max()), (dim, ki, kj)


def test_cross_phase_stress_weights_agree_at_density_ratio_one_and_conserve_momentum():
    """At equal rest densities every 2 phi is 1 and the two readings are the
    same sum; at density ratio 1000 both keep m_i a_i + m_j a_j = 0 pair by
    pair, so the total surface force on a jittered cluster vanishes."""
    rng = np.random.default_rng(21)
    dx = 0.1
    pos = np.zeros((16, 3))
    pos[:, :2] = rng.uniform(0.0, 3 * dx, size=(16, 2))
    kind = np.array([0] * 9 + [1] * 7, dtype=np.int32)
    for rho0 in ((1.0, 1.0), (1000.0, 1.0)):
        rho = np.where(kind == 0, rho0[0], rho0[1]) * (1.0 + 0.01 * rng.normal(size=16))
        res = []
        for w in (0, 1):
            P = oracle.make_params(2, dx, 1.3 * dx, 10.0, 0.8, rho0=rho0, eta=(0.1, 0.1), n=16, tvf_alpha=0.0,
                                   stress_weights=w)
            a_s = oracle.forces(P, pos, np.zeros((16, 3)), rho, kind)["a_s"]
            m = np.where(kind == 0, rho0[0], rho0[1]) * dx * dx
            total = (m[:, None] * a_s).sum(axis=0)
            assert np.abs(total).max() <= 1e-12 * np.abs(m[:, None] * a_s).max()
            res.append(a_s)
        if rho0[0] == rho0[1]:
            assert np.array_equal(res[0], res[1])
        else:
            assert not np.allclose(res[0], res[1])


# ---------------------------------------------------------------------------
# The own-fluid correction reading of the same-phase line (surface_corr = 1):
# S_ij (B^k_i + B^k_j)/2 grad_i W_ij, B^k Eq. 15's correction matrix summed
# over the particle's own fluid.
# ---------------------------------------------------------------------------
def mixed_cluster(seed, n_a=9, n_b=7):
    rng = np.random.default_rng(seed)
    dx = 0.1
    pos = np.zeros((n_a + n_b, 3))
    pos[:, :2] = rng.uniform(0.0, 3 * dx, size=(n_a + n_b, 2))
    kind = np.array([0] * n_a + [1] * n_b, dtype=np.int32)
    return dx, pos, kind, rng


def test_own_fluid_correction_matrix():
    """B^k equals Eq. 15's B where every neighbour is of the particle's own
    fluid, and differs from it where the other fluid is near."""
    case_pos = np.array([[x, y, 0.0] for x in np.arange(8) * 0.1 for y in np.arange(8) * 0.1])
    kind = np.where(case_pos[:, 0] < 0.35, 0, 1).astype(np.int32)
    rho = np.where(kind == 0, 3.0, 1.0)
    P = oracle.make_params(2, 0.1, 0.13, 10.0, 1.0, rho0=(3.0, 1.0), eta=(0.1, 0.1), n=len(case_pos))
    B, Bk = oracle.correction_matrices(P, case_pos, np.zeros_like(case_pos), rho, kind)
    far = np.abs(case_pos[:, 0] - 0.35) > 0.3          # no other-fluid neighbour within 2h = 0.26
    near = np.abs(case_pos[:, 0] - 0.35) < 0.1
    assert far.any() and near.any()
    assert np.array_equal(B[far], Bk[far])
    assert np.abs(B[near] - Bk[near]).max() > 0.1


def test_own_fluid_correction_conserves_momentum_and_is_wired():
    """At density ratio 1000 the corrected pair term stays antisymmetric
    (the mean of the two matrices), so the total surface force of a jittered
    cluster vanishes; and each particle's a^s equals the sum of the pair
    matrix applied to (B^k_i + B^k_j)/2 e_ij for same-phase pairs and to e_ij
    for the others, times W'(r) V_j / rho_i."""
    dx, pos, kind, rng = mixed_cluster(31)
    n = len(pos)
    rho0 = (1000.0, 1.0)
    rho = np.where(kind == 0, rho0[0], rho0[1]) * (1.0 + 0.01 * rng.normal(size=n))
    h = 1.3 * dx
    P = oracle.make_params(2, dx, h, 10.0, 0.8, rho0=rho0, eta=(0.1, 0.1), n=n, tvf_alpha=0.0, surface_corr=1)
    out = oracle.forces(P, pos, np.zeros((n, 3)), rho, kind)
    a_s, gC = out["a_s"], out["gradC"]
    m = np.where(kind == 0, rho0[0], rho0[1]) * dx * dx
    assert np.abs((m[:, None] * a_s).sum(axis=0)).max() <= 1e-12 * np.abs(m[:, None] * a_s).max()
    _, Bk = oracle.correction_matrices(P, pos, np.zeros((n, 3)), rho, kind)
    mass = np.where(kind == 0, rho0[0], rho0[1]) * dx * dx
    for i in range(n):
        a = np.zeros(2)
        for j in range(n):
            rv = pos[i, :2] - pos[j, :2]
            r = float(np.linalg.norm(rv))
            if j == i or not (0.0 < r < 2 * h):
                continue
            e = rv / r
            v = 0.5 * (Bk[i, :2, :2] + Bk[j, :2, :2]) @ e if kind[i] == kind[j] else e
            Sv = oracle.surface_pair_apply(P, kind[i], kind[j], gC[i, :2], gC[j, :2], e, r, v)
            a += Sv * oracle.kernel_dW(2, h, r) * (mass[j] / rho[j]) / rho[i]
        assert a_s[i, :2] == pytest.approx(a, rel=1e-11, abs=1e-12 * np.abs(a_s).max())
    plain = oracle.forces(oracle.make_params(2, dx, h, 10.0, 0.8, rho0=rho0, eta=(0.1, 0.1), n=n, tvf_alpha=0.0),
                          pos, np.zeros((n, 3)), rho, kind)["a_s"]
    assert not np.allclose(plain, a_s)
