"""Integral observables on the GPU path, against the oracle and against the
closed forms the paper and textbooks give:

* the Young-Laplace jump (Eq. 37) of a static drop: GPU time average equals
  the oracle's within 1%, and both equal gamma / R within the resolution
  error of R = 10 dp;
* the 2D drop of §5.1 (velocity of Eq. 34): the GPU's shape-anisotropy
  signal equals the oracle's while the two FP64 trajectories still coincide
  (the flow is chaotic: last-bit differences grow over thousands of
  substeps); at density ratio 1 with the paper's V0 = 10, the paper's own
  check: the centre of mass of the drop's upper-right quarter converges
  with resolution (R/dp 12, 24, 48);
* the Laplace jump against resolution (R = 10, 20, 40 dp): within 5% with
  full Riemann dissipation; with the default limiter it does not converge
  (an expected failure that states the measured values);
* total momentum of a wall-free run is conserved to FP32 rounding.
"""
import math

import numpy as np
import pytest

import oracle
import sphcases
from paper_2503_16082_gb300 import observables as ob

pytestmark = pytest.mark.gpu

S = pytest.importorskip("paper_2503_16082_gb300")


def laplace_case():
    return sphcases.small_droplet(2, 40, R_frac=0.25, rho_l=1.0, rho_g=1.0, mu_l=0.05,
                                  mu_g=0.05, c0=20.0)


def laplace_series_gpu(case, precision, t_from, t_to, chunk=20):
    h = S.case_from_spec(case, precision=precision)
    phase = S.read_fields(h, S.FIELD_PHASE, 2)
    out = []
    t = 0.0
    while t < t_to:
        info = S.step(h, chunk)
        t = info["t"]
        if t > t_from:
            dp, R = ob.laplace_jump(S.read_fields(h, S.FIELD_POS, 2), S.read_fields(h, S.FIELD_PRESSURE, 2),
                                    phase, case.dx, case.h_factor * case.dx)
            out.append(dp * R / case.gamma)
    S.destroy(h)
    return np.array(out)


def laplace_series_oracle(case, t_from, t_to, chunk=20):
    pos, vel, rho, kind = case.flat()
    P = oracle.params_for_case(case)
    rho0 = np.asarray(case.fluid_props()[0])[np.minimum(kind, 1)]
    out = []
    t = 0.0
    while t < t_to:
        pos, vel, rho, info, _, _ = oracle.run(P, pos, vel, rho, kind, chunk)
        t += info["t"]
        if t > t_from:
            p = case.c0 ** 2 * (rho - rho0)
            dp, R = ob.laplace_jump(pos[:, :2], p, kind, case.dx, case.h_factor * case.dx)
            out.append(dp * R / case.gamma)
    return np.array(out)


@pytest.mark.parametrize("precision", [64, 32])
def test_laplace_jump_gpu_vs_oracle_and_closed_form(precision):
    case = laplace_case()
    g = laplace_series_gpu(case, precision, 0.2, 0.45)
    o = laplace_series_oracle(case, 0.2, 0.45)
    assert len(g) == len(o) > 5
    gm, om = g.mean(), o.mean()
    assert abs(gm - om) <= 0.01 * abs(om), (gm, om)
    assert 0.8 < gm < 1.3, gm


def period_series_gpu(case, t_end, precision=64, chunk=10):
    h = S.case_from_spec(case, precision=precision)
    phase = S.read_fields(h, S.FIELD_PHASE, 2)
    ts, an = [], []
    t = 0.0
    while t < t_end:
        info = S.step(h, chunk)
        t = info["t"]
        ts.append(t)
        an.append(ob.anisotropy(S.read_fields(h, S.FIELD_POS, 2), phase))
    S.destroy(h)
    return np.array(ts), np.array(an)


def quarter_centroid_series(r_over_dp, precision=64, t_end=0.5, every=2, lanes=4):
    """Section 5.1, density ratio 1, V0 = 10 (the paper's values; the peak
    initial speed is V0/e, so c0 = 10 x 3.7 = 37): centre of mass of the
    particles that start in the drop's upper-right quarter, against time."""
    case = sphcases.oscillating_2d(ratio=1.0, R_over_dp=r_over_dp, V0=10.0, c0=37.0)
    liq = case.phases[0].pos
    sel = np.where((liq[:, 0] > 0.5) & (liq[:, 1] > 0.5))[0]
    h = S.case_from_spec(case, precision=precision, lanes=lanes, block=64)
    ts, xs = [0.0], [liq[sel].mean(0)]
    info = S.case_info(h)
    while info["t"] < t_end:
        info = S.step(h, every)
        ts.append(info["t"])
        xs.append(S.read_fields(h, S.FIELD_POS, 2)[sel].mean(0))
    S.destroy(h)
    tg = np.linspace(0.0, t_end - 0.01, 200)
    xs = np.array(xs)
    return np.stack([np.interp(tg, ts, xs[:, 0]), np.interp(tg, ts, xs[:, 1])], axis=1)


def test_oscillating_drop_quarter_centroid_converges():
    # the paper's own check of the ratio-1 drop (Section 5.1): the quarter's
    # centre of mass at three resolutions.  Measured (FP64 = oracle): the
    # largest gap between R/dp 24 and 48 is 0.74e-3 to 1.03e-3 (depending on
    # the build's summation order), smaller than between 12 and 24, against
    # an excursion of 0.016.  The flow amplifies summation-order differences:
    # at R/dp 24 and 48 reordering the sums alone moves the curve by up to
    # 0.76e-3, so the bar on the 24-48 gap is twice that, 8% of the excursion
    a, b, c = (quarter_centroid_series(r) for r in (12, 24, 48))
    d1, d2 = np.abs(a - b).max(), np.abs(b - c).max()
    excursion = c[:, 0].max() - c[:, 0].min()
    assert excursion > 0.01
    assert d2 < d1, (d1, d2)
    assert d2 < 0.08 * excursion, (d2, excursion)


def test_fp32_quarter_centroid_within_the_fp64_summation_order_spread():
    # the same observable as the FP32 path's precision bar, at R/dp = 24.
    # FP64 runs that differ only in summation order (1, 2 or 8 lanes per
    # particle against 4) already differ (the flow amplifies last-bit
    # differences): measured 0.38e-3 to 0.76e-3 for one reordering,
    # depending on the build's rounding, against an excursion of 0.016.
    # FP32 differs from FP64 (4 lanes) by 0.64e-3 to 0.76e-3.  The bar: FP32
    # within three times the largest FP64 reordering and within 10% of the
    # excursion
    a = quarter_centroid_series(24, 64)
    spread = max(np.abs(a - quarter_centroid_series(24, 64, lanes=n)).max() for n in (1, 2, 8))
    d32 = np.abs(a - quarter_centroid_series(24, 32)).max()
    excursion = a[:, 0].max() - a[:, 0].min()
    assert spread > 0.0
    assert d32 < 3.0 * spread, (d32, spread)
    assert d32 < 0.10 * excursion, (d32, excursion)


def laplace_jump_resolution(n_side, **params):
    """Time-averaged Delta p R / gamma of the viscous 2D drop (density and
    viscosity ratio 1, eta = 0.05, gamma = 1, R = n_side / 4 dp) over
    t in [0.4, 1.0], FP64."""
    case = sphcases.small_droplet(2, n_side, R_frac=0.25, rho_l=1.0, rho_g=1.0, mu_l=0.05, mu_g=0.05, c0=20.0)
    h = S.case_from_spec(case, precision=64, lanes=4, block=64, **params)
    phase = S.read_fields(h, S.FIELD_PHASE, 2)
    out = []
    info = S.case_info(h)
    while info["t"] < 1.0:
        info = S.step(h, 5)
        if info["t"] > 0.4:
            dp, R = ob.laplace_jump(S.read_fields(h, S.FIELD_POS, 2), S.read_fields(h, S.FIELD_PRESSURE, 2),
                                    phase, case.dx, case.h_factor * case.dx)
            out.append(dp * R / case.gamma)
    S.destroy(h)
    return float(np.mean(out))


def test_laplace_jump_with_full_riemann_dissipation():
    # with beta = 1 in Eq. 9 (full dissipation) the static drop settles and
    # Eq. 37 holds within 5% at R = 10, 20 and 40 dp (measured 1.006, 1.041,
    # 1.047: the error does not fall below the h = 1.3 dp smoothing's)
    for n in (40, 80, 160):
        x = laplace_jump_resolution(n, limiter=1)
        assert abs(x - 1.0) <= 0.05, (n / 4, x)


@pytest.mark.xfail(strict=True, reason="measured: with the dimensionless reading of the limiter of Eq. 11 the "
                                       "parasitic currents grow with resolution (peak speeds 0.27, 0.55, 0.80) and "
                                       "Delta p R / gamma is 1.07, 1.28, 1.25 at R = 10, 20, 40 dp")
def test_laplace_jump_converges_with_the_default_limiter():
    x = [laplace_jump_resolution(n) for n in (40, 80, 160)]
    err = [abs(v - 1.0) for v in x]
    assert err[2] < err[1] < err[0] and err[2] <= 0.05, x


def test_oscillating_drop_period_fp32_against_fp64():
    # the FP32 path's error on a dynamic observable, stated against FP64
    # (which equals the oracle): measured +1.3% to +2.8% over 2 periods
    case = sphcases.oscillating_2d(ratio=1.0)
    want = 2 * math.pi * math.sqrt(2 * 0.2 ** 3 * 1.0 / (6 * 1.0))
    p64 = ob.fit_period(*period_series_gpu(case, 2 * want, precision=64, chunk=5), want)
    p32 = ob.fit_period(*period_series_gpu(case, 2 * want, precision=32, chunk=5), want)
    assert abs(p32 - p64) <= 0.04 * p64, (p32, p64)


def test_oscillating_drop_signal_gpu_vs_oracle():
    case = sphcases.oscillating_2d(ratio=1000.0)
    ts, an = period_series_gpu(case, 0.05)
    pos, vel, rho, kind = case.flat()
    P = oracle.params_for_case(case)
    ots, oan = [], []
    t = 0.0
    while t < 0.05:
        pos, vel, rho, info, _, _ = oracle.run(P, pos, vel, rho, kind, 10)
        t += info["t"]
        ots.append(t)
        oan.append(ob.anisotropy(pos[:, :2], kind))
    ots, oan = np.array(ots), np.array(oan)
    assert len(ts) == len(ots) and np.allclose(ts, ots, rtol=1e-12)
    # ~530 advection steps / 2100 substeps: the FP64 trajectories coincide
    assert np.abs(an - oan).max() <= 1e-8 * np.abs(oan).max()


def test_momentum_conserved_without_walls():
    case = sphcases.free_blob(dim=2, n_side=24, vel_amp=0.05, rho_jitter=1e-6)
    h = S.case_from_spec(case, precision=32, tvf_alpha=0.0)
    v0 = S.read_fields(h, S.FIELD_VEL, 2)
    ph = S.read_fields(h, S.FIELD_PHASE, 2).astype(int)
    m = np.asarray(case.fluid_props()[0])[ph] * case.dx ** 2
    S.step(h, 5)
    v1 = S.read_fields(h, S.FIELD_VEL, 2)
    S.destroy(h)
    scale = (m * np.linalg.norm(v0, axis=1)).sum()
    assert np.abs(ob.momentum(v1, m) - ob.momentum(v0, m)).max() <= 1e-5 * scale


@pytest.mark.parametrize("precision", [64, 32])
def test_shear_drop_deformation_matches_taylor(precision):
    # Section 5.2: a drop in Couette flow, periodic in x, walls at +-U, equal
    # densities and viscosities, Re = 0.125; Taylor's D = Ca (19 + 16)/(16 + 16)
    # for a viscosity ratio of 1.  Measured at R = 12 dp: D = 0.0993 (-9%).
    case = sphcases.shear_drop_2d(0.1, t_end=20.0)
    h = S.case_from_spec(case, precision=precision)
    ds = []
    t = 0.0
    while t < 20.0:
        t = S.step(h, 400)["t"]
        if t >= 15.0:
            ds.append(ob.deformation_device(h, 2))
    assert S.diagnose(h)["n_nonfinite"] == 0
    S.destroy(h)
    D, ref = float(np.mean(ds)), ob.taylor_deformation(0.1)
    assert abs(D - ref) <= 0.15 * ref, (D, ref)


def test_impact_at_u0_10_reaches_the_papers_end_time_with_full_dissipation():
    # Section 5.4 in the paper's units at U0 = 10 (Re 2000, We 1000), d = 20
    # dp: with the low-dissipation limiter of Eq. 11 (the default reading) the
    # run stops at t = 1.1 of 4 (2.6 with walls that never pull); with
    # beta = 1 it reaches t = 4 with every particle finite
    case = sphcases.impact_sweep_case(10.0, 20)
    h = S.case_from_spec(case, precision=32, limiter=1)
    info = S.case_info(h)
    while info["t"] < case.t_end:
        info = S.step(h, 40)
    vel = S.read_fields(h, S.FIELD_VEL, 3)
    S.destroy(h)
    assert info["status"] == 0 and info["t"] >= case.t_end
    assert np.all(np.isfinite(vel))


def test_impact_at_highest_reynolds_and_weber_stays_finite():
    # Section 5.4 at U0 = 50 (Re = 1e4, We = 2.5e4), coarse (d = 10 dp), the
    # first fifth of the paper's end time: no numerical instability
    case = sphcases.impact_sweep_case(50.0, 10)
    h = S.case_from_spec(case, precision=32)
    t = 0.0
    while t < 0.02:
        info = S.step(h, 20)
        t = info["t"]
    dg = S.diagnose(h)
    pos = S.read_fields(h, S.FIELD_POS, 3)
    ph = S.read_fields(h, S.FIELD_PHASE, 3)
    S.destroy(h)
    assert info["status"] == 0 and dg["n_nonfinite"] == 0
    # the drop has hit the wall and spread beyond its initial radius
    assert np.sqrt(((pos[ph == 0, :2] - 4.0) ** 2).sum(1)).max() > 0.6


def lattice_gradient_factor_2d(h_over_dx=1.3):
    # m = -sum_j V_j x_ij^2 W'(r_ij) / r_ij over the lattice (Wendland C2)
    a = 7.0 / (4.0 * math.pi * h_over_dx ** 2)
    m = 0.0
    for i in range(-3, 4):
        for j in range(-3, 4):
            r = math.hypot(i, j)
            q = r / h_over_dx
            if 0.0 < r and q < 2.0:
                m += i * i / r * 5.0 * a * q * (1.0 - q / 2.0) ** 3 / h_over_dx
    return m


@pytest.mark.parametrize("precision", [32, 64])
def test_standing_sound_wave_period(precision):
    # a small density wave at rest in a periodic lattice: the period of the
    # standing wave is 2 pi / (c0 k m), m the lattice factor of the discrete
    # gradient, to O((k h)^2) (0.1% at 64 particles per wavelength)
    nx, ny, eps, c0 = 64, 8, 1e-3, 10.0
    dx = 1.0 / nx
    pos = sphcases.lattice([0.0, 0.0], [1.0, ny * dx], dx)
    k = 2.0 * math.pi
    rho = 1.0 + eps * np.cos(k * pos[:, 0])
    eta = 0.03 * (32.0 / nx) ** 2                   # sets the advection step only (Eq. 16)
    case = sphcases.Case(name="sound", dim=2, lo=[0.0, 0.0], hi=[1.0, ny * dx], dx=dx, gamma=0.0, c0=c0,
                         h_factor=1.3, xi=-1.0, periodic=3,
                         phases=[sphcases.Phase("fluid", pos, rho0=1.0, eta=eta, rho=rho)])
    h = S.case_from_spec(case, precision=precision)
    ts, amp = [0.0], [eps]
    try:
        for _ in range(40):
            info = S.step(h, 1)
            p = S.read_fields(h, S.FIELD_POS, 2)
            r = S.read_fields(h, S.FIELD_RHO, 2)
            ts.append(info["t"])
            amp.append(2.0 * np.mean((r - 1.0) * np.cos(k * p[:, 0])))
    finally:
        S.destroy(h)
    ratio = ob.fit_period(ts, amp, 1.0 / c0) * c0
    assert ratio == pytest.approx(1.0 / lattice_gradient_factor_2d(), rel=3e-3)


def test_box_mode_between_walls_period():
    # the lowest acoustic mode between two walls (periodic across them) has
    # the rigid-wall period 2 L / (c0 m) on the GPU as in the oracle
    nx, ny, eps, c0 = 64, 8, 1e-3, 10.0
    dx = 1.0 / nx
    lo, hi = [0.0, 0.0], [1.0, ny * dx]
    pos = sphcases.lattice(lo, hi, dx)
    k = math.pi
    eta = 0.03 * (32.0 / nx) ** 2
    case = sphcases.Case(name="box_mode", dim=2, lo=lo, hi=hi, dx=dx, gamma=0.0, c0=c0, h_factor=1.3,
                         xi=-1.0, periodic=2,
                         phases=[sphcases.Phase("fluid", pos, rho0=1.0, eta=eta, rho=1.0 + eps * np.cos(k * pos[:, 0])),
                                 sphcases.Phase("wall", sphcases.wall_shell(lo, hi, dx, sides=[0]))])
    h = S.case_from_spec(case, precision=64)
    ph = S.read_fields(h, S.FIELD_PHASE, 2)
    fl = ph == 0
    ts, amp = [0.0], [eps]
    try:
        for _ in range(60):
            info = S.step(h, 1)
            p = S.read_fields(h, S.FIELD_POS, 2)
            r = S.read_fields(h, S.FIELD_RHO, 2)
            ts.append(info["t"])
            amp.append(2.0 * np.mean((r[fl] - 1.0) * np.cos(k * p[fl, 0])))
    finally:
        S.destroy(h)
    ratio = ob.fit_period(ts, amp, 2.0 / c0) * c0 / 2.0
    assert ratio == pytest.approx(1.0 / lattice_gradient_factor_2d(), rel=1e-3)


def test_laplace_jump_3d_static_drop():
    # the 3D form of Eq. 37: dp = 2 gamma / R for a spherical drop (ratio 1,
    # the paper's viscous regime), R = 15 dp; measured 0.959 at t = 3.75
    case = sphcases.laplace_3d(dx=0.5 / 15.0)
    h = S.case_from_spec(case, precision=32)
    phase = S.read_fields(h, S.FIELD_PHASE, 3)
    samples = []
    try:
        for k in range(0, 1000, 50):
            S.step(h, 50)
            if k >= 800:
                dp, R = ob.laplace_jump(S.read_fields(h, S.FIELD_POS, 3), S.read_fields(h, S.FIELD_PRESSURE, 3),
                                        phase, case.dx, case.h_factor * case.dx)
                samples.append(dp * R / (2.0 * case.gamma))
    finally:
        S.destroy(h)
    assert 0.85 < np.mean(samples) < 1.15


def square_drop_jump(dp, **params):
    """Section 5.3: square drop of side l = 1 in a 2 x 2 box, density ratio
    1000, viscosity ratio 100, gamma = 1; Delta p averaged over t in
    [0.7, 1.0] against Eq. 37's gamma sqrt(pi) / l (FP64)."""
    case = sphcases.droplet_case("square", 2, [0, 0], [2, 2], dp, [1.0, 1.0], 1.0 / math.sqrt(math.pi),
                                 shape="square", rho_l=1.0, rho_g=1e-3, mu_l=0.05, mu_g=5e-4, sigma=1.0, c0=10.0)
    h = S.case_from_spec(case, precision=64, lanes=4, block=64, **params)
    phase = S.read_fields(h, S.FIELD_PHASE, 2)
    out = []
    info = S.case_info(h)
    while info["t"] < 1.0:
        info = S.step(h, 20)
        if info["t"] > 0.7:
            jump, _ = ob.laplace_jump(S.read_fields(h, S.FIELD_POS, 2), S.read_fields(h, S.FIELD_PRESSURE, 2),
                                      phase, case.dx, case.h_factor * case.dx)
            out.append(jump)
    S.destroy(h)
    return float(np.mean(out)) / math.sqrt(math.pi)


@pytest.mark.xfail(strict=True, reason="measured: at density ratio 1000 the jump is 0.60, 0.52, 0.41 of Eq. 37 at "
                                       "dp = 0.04, 0.02, 0.01 (0.69, 0.57, 0.45 with beta = 1), the paper reports "
                                       "close agreement at dp = 0.01; the printed weights 2 phi of Eqs. 22 and 26 "
                                       "give the liquid 0.70 of the CSF surface force at every resolution")
def test_square_drop_laplace_jump_at_density_ratio_1000():
    x = square_drop_jump(0.02)
    assert abs(x - 1.0) <= 0.10, x


def test_oscillating_drop_period_at_density_ratio_1000_with_the_own_fluid_correction():
    # the surface_corr reading (the same-phase line of Eq. 33 with the kernel
    # gradient corrected by the own-fluid matrices of Eq. 15) gives the liquid
    # the full surface force (0.98 of CSF, oracle pin): at R = 12 dp the period
    # is within 5% of Eq. 35 (measured +0.8%, +1.9%, +2.3% with 4, 1 and 8
    # lanes per particle).  At 24 dp it is 6-8% long and at 48 dp the signal
    # loses its regular oscillation, so this is not the paper's convergence
    case = sphcases.oscillating_2d(ratio=1000.0, R_over_dp=12, V0=1.0, gamma=0.5)
    tau = 2 * math.pi * math.sqrt(0.2 ** 3 * 1.0 / (6 * 0.5))
    h = S.case_from_spec(case, precision=64, lanes=4, block=64, surface_corr=1)
    phase = S.read_fields(h, S.FIELD_PHASE, 2)
    ts, an = [], []
    info = S.case_info(h)
    while info["t"] < 3 * tau:
        info = S.step(h, 5)
        ts.append(info["t"])
        an.append(ob.anisotropy(S.read_fields(h, S.FIELD_POS, 2), phase))
    S.destroy(h)
    period = ob.fit_period(ts, an, tau)
    assert abs(period - tau) <= 0.05 * tau, (period, tau)


@pytest.mark.xfail(strict=True, reason="measured: at density ratio 1000 (V0 = 1, gamma = 0.5) the fitted period is "
                                       "0.37-0.46 at R = 12 and 24 dp against Eq. 35's 0.324 (0.40-0.43 with "
                                       "beta = 1; the value moves with the build's rounding: the flow is chaotic); "
                                       "at gamma = 1 the signal has no regular period; the paper reports < 5% for "
                                       "every gamma")
def test_oscillating_drop_period_at_density_ratio_1000():
    case = sphcases.oscillating_2d(ratio=1000.0, R_over_dp=24, V0=1.0, gamma=0.5)
    tau = 2 * math.pi * math.sqrt(0.2 ** 3 * 1.0 / (6 * 0.5))
    h = S.case_from_spec(case, precision=64, lanes=4, block=64)
    phase = S.read_fields(h, S.FIELD_PHASE, 2)
    ts, an = [], []
    info = S.case_info(h)
    while info["t"] < 3 * tau:
        info = S.step(h, 5)
        ts.append(info["t"])
        an.append(ob.anisotropy(S.read_fields(h, S.FIELD_POS, 2), phase))
    S.destroy(h)
    period = ob.fit_period(ts, an, tau)
    assert abs(period - tau) <= 0.05 * tau, (period, tau)
