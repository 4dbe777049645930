"""Run the paper-shaped workloads on the GPU and report their observables.

  python -m paper_2503_16082_gb300.validate laplace_2d [--precision 64] [--adv 500]
  python -m paper_2503_16082_gb300.validate laplace_3d [--ratio3d 1] [--dx3d 0.05]
  python -m paper_2503_16082_gb300.validate oscillating_3d [--periods 1.5]
  python -m paper_2503_16082_gb300.validate impact_3d [--t-end 2]
  python -m paper_2503_16082_gb300.validate oscillating_2d [--ratio 1000] [--r-over-dp 12] [--xi 0]
  python -m paper_2503_16082_gb300.validate shear_drop [--ca 0.1] [--t-end 20] [--r-over-dp 12]
  python -m paper_2503_16082_gb300.validate impact_sweep [--res 20] [--u0 0.5 1 5 10 50]

Each prints one JSON line.  laplace_2d: Young-Laplace jump (Eq. 37)
averaged over the last 20% of the run, against gamma / R_eff.  oscillating_*:
period of the drop's shape anisotropy against Eq. 35 (2D, ratio >> 1), the
equal-density textbook value (2D, ratio 1) or Lamb's n = 2 value (3D).
The 2D drop also reports the interface disorder (share of fluid particles
whose neighbours belong mostly to the other fluid) at the end of the run and
its maximum over the run; --xi 0 switches the penalty of Eqs. 29-33 off.
impact_3d: whether the run stays finite to t_end, with its substep count.
impact_sweep: Section 5.4's impact in the paper's units for each U0 (Re up to
1e4, We up to 2.5e4): whether the run stays finite to the paper's end time,
and the drop's final spread along the wall (--wall-form 1: walls push and
never pull).
shear_drop: Taylor deformation of the drop of Section 5.2 (periodic in x,
walls at +-U) averaged over the last 25% of the run, against Taylor's
D = Ca (19 l + 16)/(16 l + 16) with l = 1.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import sphcases  # noqa: E402

import paper_2503_16082_gb300 as S  # noqa: E402
from paper_2503_16082_gb300 import observables as ob  # noqa: E402


def launch(args) -> dict:
    """Launch shape of the sweeps (speed only: block size, lanes per
    particle) and the penalty-scope ablation flag."""
    kw = {}
    if getattr(args, "penalty_scope", 0):
        kw["penalty_scope"] = args.penalty_scope
    if getattr(args, "wall_form", 0):
        kw["wall_form"] = args.wall_form
    if getattr(args, "stress_weights", 0):
        kw["stress_weights"] = args.stress_weights
    if getattr(args, "surface_corr", 0):
        kw["surface_corr"] = args.surface_corr
    if getattr(args, "limiter", None) is not None:
        kw["limiter"] = args.limiter
    if args.block:
        kw["block"] = args.block
    if args.lanes:
        kw["lanes"] = args.lanes
    return kw


def laplace(args, dim=2):
    case = sphcases.laplace_2d() if dim == 2 else sphcases.laplace_3d(ratio=args.ratio3d, dx=args.dx3d)
    h = S.case_from_spec(case, precision=args.precision, **launch(args))
    phase = S.read_fields(h, S.FIELD_PHASE, dim)
    samples = []
    t0 = time.perf_counter()
    every = 10
    for k in range(0, args.adv, every):
        info = S.step(h, every, check=False)
        if info["rc"]:
            break
        if k >= 0.8 * args.adv:
            dp, R = ob.laplace_jump(S.read_fields(h, S.FIELD_POS, dim), S.read_fields(h, S.FIELD_PRESSURE, dim),
                                    phase, case.dx, case.h_factor * case.dx)
            samples.append(dp * R / ((dim - 1) * case.gamma))     # Eq. 37: (d - 1) gamma / R
    wall = time.perf_counter() - t0
    vmax = float(np.abs(S.read_fields(h, S.FIELD_VEL, dim)).max())
    S.destroy(h)
    return {"workload": f"laplace_{dim}d", "precision": args.precision, "adv": info["n_adv"],
            **({"ratio": args.ratio3d, "dx": case.dx, "particles": case.n} if dim == 3 else {}),
            "substeps": info["n_sub"], "t": info["t"], "status": info["status"],
            "dp_R_over_dm1_gamma_mean": float(np.mean(samples)) if samples else None,
            "dp_R_over_dm1_gamma_std": float(np.std(samples)) if samples else None,
            "exact": 1.0, "vmax_end": vmax, "wall_s": round(wall, 2)}


def oscillating(args, dim):
    if dim == 3:
        if args.ratio == 1000.0:
            rho_in, rho_out = 1000.0, 1.0
            case = sphcases.oscillating_3d()
        else:      # drop density 1, viscosity 0.01 (light damping), outer fluid rho/ratio, eta/ratio
            rho_in, rho_out = 1.0, 1.0 / args.ratio
            case = sphcases.oscillating_3d(rho_l=rho_in, rho_g=rho_out, mu_l=0.01, mu_g=0.01 / args.ratio)
        R = 0.5
        tau = ob.period_lamb_3d(R, rho_in, rho_out, case.gamma)
    else:
        case = sphcases.oscillating_2d(ratio=args.ratio, R_over_dp=args.r_over_dp)
        tau = ob.period_2d_drop(0.2, 1.0, 1.0) * (math.sqrt(2.0) if args.ratio == 1 else 1.0)
    if args.xi is not None:
        case.xi = args.xi
    h = S.case_from_spec(case, precision=args.precision, **launch(args))
    phase = S.read_fields(h, S.FIELD_PHASE, dim)
    hk = case.h_factor * case.dx
    ts, an, stray = [], [], []
    t0 = time.perf_counter()
    t_end = args.periods * tau
    info = S.case_info(h)
    while info["t"] < t_end:
        info = S.step(h, args.every, check=False)
        if info["rc"]:
            break
        ts.append(info["t"])
        pos = S.read_fields(h, S.FIELD_POS, dim)
        an.append(ob.anisotropy(pos, phase))
        if dim == 2 and len(ts) % 10 == 1:
            stray.append(ob.stray_fraction(pos, phase, hk))
    wall = time.perf_counter() - t0
    if dim == 2:
        stray.append(ob.stray_fraction(S.read_fields(h, S.FIELD_POS, dim), phase, hk))
    S.destroy(h)
    s = np.array(an) - np.mean(an)
    cr = [ts[k - 1] + (ts[k] - ts[k - 1]) * (-s[k - 1]) / (s[k] - s[k - 1])
          for k in range(1, len(s)) if np.sign(s[k]) != np.sign(s[k - 1]) and s[k] != s[k - 1]]
    period = ob.fit_period(ts, an, tau) if len(ts) > 10 else float("nan")
    return {"workload": f"oscillating_{dim}d", "precision": args.precision, "ratio": args.ratio,
            "adv": info["n_adv"], "substeps": info["n_sub"], "t": info["t"], "status": info["status"],
            "zero_crossings": [round(c, 4) for c in cr], "period": period, "theory": tau,
            "rel_error": (period - tau) / tau if period == period else None,
            "anisotropy_amplitude": float(np.abs(s).max()) if len(s) else None,
            "series": [[round(ts[k], 5), float(an[k])] for k in range(0, len(ts), max(1, len(ts) // 200))],
            **({"R_over_dp": args.r_over_dp, "xi": case.xi, "penalty_scope": args.penalty_scope,
                "stray_end": stray[-1], "stray_max": max(stray)}
               if dim == 2 else {}),
            "wall_s": round(wall, 2)}


def impact(args):
    case = sphcases.impact_3d()
    h = S.case_from_spec(case, precision=args.precision, **launch(args))
    t0 = time.perf_counter()
    info = S.case_info(h)
    while info["t"] < args.t_end:
        info = S.step(h, 10, check=False)
        if info["rc"]:
            break
    wall = time.perf_counter() - t0
    vel = S.read_fields(h, S.FIELD_VEL, 3)
    S.destroy(h)
    return {"workload": "impact_3d", "precision": args.precision, "particles": case.n,
            "adv": info["n_adv"], "substeps": info["n_sub"], "t": info["t"], "status": info["status"],
            "finite": bool(np.isfinite(vel).all()), "vmax": float(np.abs(vel).max()),
            "particle_substeps_per_s": case.n_fluid * info["n_sub"] / wall, "wall_s": round(wall, 2)}


def shear(args):
    case = sphcases.shear_drop_2d(args.ca, t_end=args.t_end, R_over_dp=args.r_over_dp)
    h = S.case_from_spec(case, precision=args.precision, **launch(args))
    ts, ds = [], []
    t0 = time.perf_counter()
    info = S.case_info(h)
    while info["t"] < args.t_end:
        info = S.step(h, args.every_shear, check=False)
        if info["rc"]:
            break
        ts.append(info["t"])
        ds.append(ob.deformation_device(h, 2))
    wall = time.perf_counter() - t0
    dg = S.diagnose(h)
    S.destroy(h)
    ts, ds = np.array(ts), np.array(ds)
    tail = ts >= 0.75 * ts[-1] if len(ts) else ts
    D = float(ds[tail].mean()) if len(ts) else float("nan")
    ref = ob.taylor_deformation(args.ca)
    return {"workload": "shear_drop_2d", "precision": args.precision, "Ca": args.ca, "Re": case.meta["Re"],
            "R_over_dp": args.r_over_dp,
            "particles": case.n, "adv": info["n_adv"], "substeps": info["n_sub"], "t": info["t"],
            "status": info["status"], "D": D, "D_std_tail": float(ds[tail].std()) if len(ts) else None,
            "taylor": ref, "rel_error": (D - ref) / ref, "n_nonfinite": dg["n_nonfinite"],
            "D_series": [[round(float(t), 3), round(float(d), 5)] for t, d in zip(ts[::max(1, len(ts) // 20)], ds[::max(1, len(ts) // 20)])],
            "wall_s": round(wall, 2)}


def impact_sweep(args):
    out = []
    for U0 in args.u0:
        case = sphcases.impact_sweep_case(U0, args.res)
        h = S.case_from_spec(case, precision=args.precision, **launch(args))
        t_end = case.t_end * args.t_frac
        t0 = time.perf_counter()
        info = S.case_info(h)
        while info["t"] < t_end:
            info = S.step(h, 20, check=False)
            if info["rc"]:
                break
        wall = time.perf_counter() - t0
        pos = S.read_fields(h, S.FIELD_POS, 3)
        vel = S.read_fields(h, S.FIELD_VEL, 3)
        ph = S.read_fields(h, S.FIELD_PHASE, 3)
        dg = S.diagnose(h)
        S.destroy(h)
        drop = ph == 0
        spread = float(np.sqrt(((pos[drop, :2] - 4.0) ** 2).sum(1)).max()) / 0.5
        out.append({"U0": U0, "Re": case.meta["Re"], "We": case.meta["We"], "particles": case.n,
                    "t": info["t"], "t_end": t_end, "status": info["status"], "adv": info["n_adv"],
                    "substeps": info["n_sub"], "finite": bool(np.isfinite(vel).all()) and dg["n_nonfinite"] == 0,
                    "spread_over_R0": round(spread, 3),
                    "drop_height": round(float(pos[drop, 2].max()), 4),
                    "particle_substeps_per_s": case.n_fluid * info["n_sub"] / wall, "wall_s": round(wall, 2)})
        print(json.dumps(out[-1]), flush=True)
    return {"workload": "impact_sweep", "precision": args.precision, "d_over_dp": args.res, "runs": out}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=["laplace_2d", "laplace_3d", "oscillating_3d", "oscillating_2d", "impact_3d", "shear_drop",
                                         "impact_sweep"])
    ap.add_argument("--res", type=int, default=20, help="impact_sweep: d / dp")
    ap.add_argument("--u0", type=float, nargs="+", default=[0.5, 1.0, 5.0, 10.0, 50.0])
    ap.add_argument("--t-frac", type=float, default=1.0, help="impact_sweep: fraction of the end time")
    ap.add_argument("--ca", type=float, default=0.1)
    ap.add_argument("--every-shear", type=int, default=200)
    ap.add_argument("--precision", type=int, default=None, choices=[32, 64])
    ap.add_argument("--adv", type=int, default=500)
    ap.add_argument("--periods", type=float, default=1.5)
    ap.add_argument("--every", type=int, default=5)
    ap.add_argument("--ratio", type=float, default=1000.0)
    ap.add_argument("--r-over-dp", type=int, default=12, help="oscillating_2d, shear_drop: R / dp")
    ap.add_argument("--ratio3d", type=float, default=1.0, help="laplace_3d: density ratio (1 or 1000)")
    ap.add_argument("--dx3d", type=float, default=0.05, help="laplace_3d: particle spacing (R = 0.5)")
    ap.add_argument("--block", type=int, default=0, help="threads per block of the sweeps (0: library default)")
    ap.add_argument("--lanes", type=int, default=0, choices=[0, 1, 2, 4, 8],
                    help="lanes per particle (0: library default); small 2D cases run faster with 4")
    ap.add_argument("--xi", type=float, default=None, help="penalty coefficient (default: from the density ratio)")
    ap.add_argument("--penalty-scope", type=int, default=0, choices=[0, 1],
                    help="0: the penalty on both lines of Eq. 33; 1: on the cross-phase line only (ablation)")
    ap.add_argument("--limiter", type=int, default=None, choices=[0, 1, 2, 3],
                    help="Eq. 11 reading (0 dimensionless low-dissipation, 1 beta = 1, 2 beta = 0, 3 as printed)")
    ap.add_argument("--wall-form", type=int, default=0, choices=[0, 1],
                    help="wall pairs: 0 mirror state as it comes, 1 no suction (max(P*, 0))")
    ap.add_argument("--stress-weights", type=int, default=0, choices=[0, 1],
                    help="cross-phase surface stress: 0 2phi_j Pi_i + 2phi_i Pi_j as printed, 1 each by its own phi")
    ap.add_argument("--surface-corr", type=int, default=0, choices=[0, 1],
                    help="same-phase surface line: 0 grad W as printed, 1 corrected by the own-fluid matrices of Eq. 15")
    ap.add_argument("--t-end", type=float, default=None, help="impact_3d: 2.0, shear_drop: 20.0")
    args = ap.parse_args(argv)
    if args.t_end is None:
        args.t_end = 20.0 if args.workload == "shear_drop" else 2.0
    if args.precision is None:
        args.precision = 64 if args.workload in ("laplace_2d", "oscillating_2d", "shear_drop") else 32
    if args.workload == "laplace_2d":
        out = laplace(args)
    elif args.workload == "laplace_3d":
        out = laplace(args, 3)
    elif args.workload == "oscillating_3d":
        out = oscillating(args, 3)
    elif args.workload == "oscillating_2d":
        out = oscillating(args, 2)
    elif args.workload == "shear_drop":
        out = shear(args)
    elif args.workload == "impact_sweep":
        out = impact_sweep(args)
    else:
        out = impact(args)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
