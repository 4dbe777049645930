"""Integral observables computed on the host from read-back fields.

* Laplace jump (Eq. 37): mean pressure of the drop's core (r < R_eff/2)
  minus mean pressure of the surrounding fluid farther than R_eff + 3h from
  the drop centre, with R_eff the radius of a disc/ball of the drop's volume.
* Oscillation period: zero crossings of the drop's shape anisotropy
  (I_xx - I_yy in 2D, I_zz - (I_xx + I_yy)/2 in 3D, second moments about the
  drop's centroid), mean spacing of same-direction crossings, linearly
  interpolated.
* Total momentum of the fluids.
* Interface disorder: the share of fluid particles whose fluid neighbours
  (r < 2h) belong mostly to the other fluid.  On a sharp interface every
  particle has at most about half of its neighbours across it; particles
  that have crossed into the other fluid, or interface particles arranged in
  a zero-surface-energy pattern (Section 4: the surface stress alone exerts
  no force on them), have more.
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np


def effective_radius(n_drop: int, dx: float, dim: int) -> float:
    vol = n_drop * dx ** dim
    return math.sqrt(vol / math.pi) if dim == 2 else (3.0 * vol / (4.0 * math.pi)) ** (1.0 / 3.0)


def laplace_jump(pos, p, phase, dx: float, h: float, drop_phase: int = 0, outer_phase: int = 1):
    """(dp, R_eff) of a drop given positions (n, dim), pressures and phase ids."""
    dim = pos.shape[1]
    drop = phase == drop_phase
    c = pos[drop].mean(axis=0)
    r = np.linalg.norm(pos - c, axis=1)
    Reff = effective_radius(int(drop.sum()), dx, dim)
    inner = drop & (r < 0.5 * Reff)
    outer = (phase == outer_phase) & (r > Reff + 3.0 * h)
    return float(p[inner].mean() - p[outer].mean()), Reff


def moments_from_diag(dg: dict, dim: int):
    """(centroid, covariance) of the phase-0 particles from device sums."""
    n = max(dg["count"][0], 1)
    c = np.array(dg["first"]) / n
    s = dg["second"]
    M = np.array([[s[0], s[3], s[4]], [s[3], s[1], s[5]], [s[4], s[5], s[2]]]) / n
    cov = M - np.outer(c, c)
    return c[:dim], cov[:dim, :dim]


def anisotropy_device(case, dim: int) -> float:
    """Shape anisotropy of the drop from FP64 device reductions."""
    from . import diagnose
    _, cov = moments_from_diag(diagnose(case), dim)
    if dim == 2:
        return float(cov[0, 0] - cov[1, 1])
    return float(cov[2, 2] - 0.5 * (cov[0, 0] + cov[1, 1]))


def laplace_jump_device(case, dim: int, dx: float, h: float):
    """(dp, R_eff) of the drop (phase 0) from two FP64 device reductions:
    the first gives the centroid and R_eff, the second the sampling sums."""
    from . import diagnose
    first = diagnose(case)
    c, _ = moments_from_diag(first, dim)
    Reff = effective_radius(int(first["count"][0]), dx, dim)
    dg = diagnose(case, tuple(c), 0.5 * Reff, Reff + 3.0 * h)
    return float(dg["p_in"] / max(dg["n_in"], 1) - dg["p_out"] / max(dg["n_out"], 1)), Reff


def deformation(cov) -> float:
    """Taylor deformation D = (a - b)/(a + b) of an elliptical drop from the
    covariance of its particles (a filled ellipse has eigenvalues a^2/4 and
    b^2/4 along its axes)."""
    lam = np.sort(np.linalg.eigvalsh(np.asarray(cov)))[::-1]
    a, b = math.sqrt(max(lam[0], 0.0)), math.sqrt(max(lam[-1], 0.0))
    return (a - b) / (a + b)


def deformation_device(case, dim: int = 2) -> float:
    """Deformation of the drop (phase 0) from FP64 device reductions."""
    from . import diagnose
    _, cov = moments_from_diag(diagnose(case), dim)
    return deformation(cov)


def taylor_deformation(Ca: float, visc_ratio: float = 1.0) -> float:
    """Taylor's small-deformation result D = Ca (19 l + 16) / (16 l + 16)."""
    return Ca * (19.0 * visc_ratio + 16.0) / (16.0 * visc_ratio + 16.0)


def anisotropy(pos, phase, drop_phase: int = 0) -> float:
    q = pos[phase == drop_phase]
    d = q - q.mean(axis=0)
    if q.shape[1] == 2:
        return float((d[:, 0] ** 2).mean() - (d[:, 1] ** 2).mean())
    return float((d[:, 2] ** 2).mean() - 0.5 * ((d[:, 0] ** 2).mean() + (d[:, 1] ** 2).mean()))


def period_from_signal(t: Sequence[float], s: Sequence[float]) -> float:
    """Mean spacing of upward zero crossings of s - mean(s); nan if < 2."""
    t = np.asarray(t, dtype=float)
    s = np.asarray(s, dtype=float)
    s = s - s.mean()
    ups = []
    for k in range(1, len(s)):
        if s[k - 1] < 0.0 <= s[k]:
            f = -s[k - 1] / (s[k] - s[k - 1])
            ups.append(t[k - 1] + f * (t[k] - t[k - 1]))
    if len(ups) < 2:
        return float("nan")
    return float(np.mean(np.diff(ups)))


def stray_fraction(pos, phase, h: float, fluid_phases=(0, 1)) -> float:
    """Share of fluid particles with more than half of their fluid
    neighbours (0 < r < 2h) from the other fluid phase."""
    from scipy.spatial import cKDTree

    fl = np.isin(phase, fluid_phases)
    q = np.asarray(pos)[fl]
    ph = np.asarray(phase)[fl]
    if len(q) == 0:
        return 0.0
    pairs = cKDTree(q).query_pairs(2.0 * h, output_type="ndarray")
    if len(pairs) == 0:
        return 0.0
    n_all = np.zeros(len(q))
    n_other = np.zeros(len(q))
    cross = (ph[pairs[:, 0]] != ph[pairs[:, 1]]).astype(float)
    for c in (0, 1):
        np.add.at(n_all, pairs[:, c], 1.0)
        np.add.at(n_other, pairs[:, c], cross)
    return float(np.mean(n_other > 0.5 * np.maximum(n_all, 1.0)))


def momentum(vel, mass) -> np.ndarray:
    return (np.asarray(mass)[:, None] * vel).sum(axis=0)


def period_2d_drop(R: float, rho_drop: float, gamma: float) -> float:
    """Eq. 35: tau = 2 pi sqrt(R^3 rho / (6 gamma)) (drop in a much lighter fluid)."""
    return 2.0 * math.pi * math.sqrt(R ** 3 * rho_drop / (6.0 * gamma))


def period_lamb_3d(R: float, rho_in: float, rho_out: float, gamma: float) -> float:
    """Lamb's n = 2 mode of a drop in a second fluid: w^2 = 24 gamma / (R^3 (3 rho_in + 2 rho_out))."""
    return 2.0 * math.pi / math.sqrt(24.0 * gamma / (R ** 3 * (3.0 * rho_in + 2.0 * rho_out)))


def fit_period(t: Sequence[float], s: Sequence[float], guess: float, skip: float = 0.05) -> float:
    """Period of s(t) ~ c + exp(-l t) (a cos w t + b sin w t), fitted by a grid
    search over (w, l) around 2 pi / guess with linear least squares for
    (a, b, c), then refined by a simplex search from the best grid point;
    the first `skip` fraction of the record is ignored."""
    from scipy.optimize import minimize

    t = np.asarray(t, dtype=float)
    s = np.asarray(s, dtype=float)
    keep = t >= t[0] + skip * (t[-1] - t[0])
    t, s = t[keep], s[keep]
    w0 = 2.0 * math.pi / guess

    def resid(x):
        w, lam = x
        e = np.exp(-lam * (t - t[0]))
        A = np.stack([np.ones_like(t), e * np.cos(w * t), e * np.sin(w * t)], axis=1)
        coef, *_ = np.linalg.lstsq(A, s, rcond=None)
        return float(((A @ coef - s) ** 2).sum())

    best = (np.inf, (w0, 0.0))
    for w in np.linspace(0.3 * w0, 3.0 * w0, 541):
        for lam in np.linspace(0.0, 2.0 * w0, 21):
            r = resid((w, lam))
            if r < best[0]:
                best = (r, (w, lam))
    x = minimize(resid, np.array(best[1]), method="Nelder-Mead",
                 options={"xatol": 1e-7 * w0, "fatol": 1e-14 * max(best[0], 1e-300), "maxiter": 400}).x
    w = x[0] if resid(x) <= best[0] else best[1][0]
    return 2.0 * math.pi / w
