"""Seeded synthetic inputs for the multiphase SPH pair sweep.

This module only places particles and labels them: lattice positions, phase
membership from a shape test, wall layers, initial velocities and the physical
parameters of each workload.  It holds none of the method's arithmetic (no
kernel, no Riemann solver, no surface stress, no time step), so both the CUDA
library's tests and the CPU oracle can take their inputs from here.

Workloads (sizes follow the paper's test problems, §5, scaled as stated):

* ``laplace_2d``      static circular droplet in a closed 2D box (Eq. 37 check)
* ``oscillating_3d``  3D droplet with a mode-2 perturbation (Lamb period check)
* ``impact_3d``       3D droplet hitting a no-slip wall at Re=1e4, We=2.5e4
* ``oscillating_2d``  the 2D oscillating drop of §5.1 with the velocity of Eq. 34
* ``batch_cases``     many independent 2D/3D droplet relaxation cases
* ``served_stream``   Poisson arrival stream of droplet cases

All lattices place particles at ``lo + (i + 1/2) dx``.  No-slip walls are three
layers of lattice particles outside the box (three layers cover the kernel
support 2h = 2.6 dx).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Sequence

import numpy as np

WALL_LAYERS = 3


@dataclasses.dataclass
class Phase:
    """One group of particles added with one call (one fluid, or one wall)."""

    kind: str                      # "fluid" or "wall"
    pos: np.ndarray                # (n, dim) float64
    rho0: float = 0.0              # reference density (fluid)
    eta: float = 0.0               # dynamic viscosity (fluid)
    vel: Optional[np.ndarray] = None   # (n, dim) initial velocity, None = rest
    rho: Optional[np.ndarray] = None   # (n,) initial density, None = rho0
    wall_vel: Sequence[float] = (0.0, 0.0, 0.0)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


@dataclasses.dataclass
class Case:
    """A full problem statement: box, resolution, fluids, walls, interface."""

    name: str
    dim: int
    lo: Sequence[float]
    hi: Sequence[float]
    dx: float
    gamma: float
    c0: float = 10.0
    h_factor: float = 1.3
    xi: float = -1.0              # < 0: derive from the density ratio
    cfl_ac: float = 0.6           # factor of the acoustic time-step criterion
    phases: List[Phase] = dataclasses.field(default_factory=list)
    t_end: Optional[float] = None  # physical end time of the workload, if any
    meta: dict = dataclasses.field(default_factory=dict)
    periodic: int = 0             # bit a set: axis a is periodic on [lo[a], hi[a])

    @property
    def n(self) -> int:
        return sum(p.n for p in self.phases)

    @property
    def n_fluid(self) -> int:
        return sum(p.n for p in self.phases if p.kind == "fluid")

    def flat(self):
        """Concatenate phases in insertion order.

        Returns ``pos (n,3)``, ``vel (n,3)``, ``rho (n,)``, ``kind (n,) int32``
        where kind is 0/1 for the first/second fluid and 2 for walls.  Wall
        particles carry their wall velocity in ``vel``; their ``rho`` entry is
        the first fluid's reference density and is never used.
        """
        n = self.n
        pos = np.zeros((n, 3))
        vel = np.zeros((n, 3))
        rho = np.zeros(n)
        kind = np.zeros(n, dtype=np.int32)
        off = 0
        fluid_no = 0
        rho_ref = next((p.rho0 for p in self.phases if p.kind == "fluid"), 1.0)
        for p in self.phases:
            s = slice(off, off + p.n)
            pos[s, : self.dim] = p.pos
            if p.kind == "fluid":
                if p.vel is not None:
                    vel[s, : self.dim] = p.vel
                rho[s] = p.rho if p.rho is not None else p.rho0
                kind[s] = fluid_no
                fluid_no += 1
            else:
                vel[s, : self.dim] = np.asarray(p.wall_vel, dtype=float)[: self.dim]
                rho[s] = rho_ref
                kind[s] = 2
            off += p.n
        return pos, vel, rho, kind

    def fluid_props(self):
        """(rho0[2], eta[2]) of the fluid phases in insertion order."""
        fl = [p for p in self.phases if p.kind == "fluid"]
        rho0 = [p.rho0 for p in fl] + [1.0] * (2 - len(fl))
        eta = [p.eta for p in fl] + [1.0] * (2 - len(fl))
        return rho0[:2], eta[:2]


# ----------------------------------------------------------------------------
# lattices
# ----------------------------------------------------------------------------

def lattice(lo: Sequence[float], hi: Sequence[float], dx: float) -> np.ndarray:
    """Cell-centred lattice filling the box [lo, hi] with spacing dx."""
    dim = len(lo)
    axes = []
    for a in range(dim):
        m = int(round((hi[a] - lo[a]) / dx))
        axes.append(lo[a] + (np.arange(m) + 0.5) * dx)
    grids = np.meshgrid(*axes, indexing="ij")
    return np.stack([g.ravel() for g in grids], axis=1)


def wall_shell(lo: Sequence[float], hi: Sequence[float], dx: float,
               layers: int = WALL_LAYERS,
               sides: Optional[Sequence[int]] = None) -> np.ndarray:
    """Lattice particles in ``layers`` rows outside the box.

    ``sides`` lists the axes that are closed by walls (default: all).  The
    shell continues the interior lattice so wall and fluid spacing agree.
    """
    dim = len(lo)
    sides = list(range(dim)) if sides is None else list(sides)
    big_lo = [lo[a] - (layers * dx if a in sides else 0.0) for a in range(dim)]
    big_hi = [hi[a] + (layers * dx if a in sides else 0.0) for a in range(dim)]
    p = lattice(big_lo, big_hi, dx)
    inside = np.ones(len(p), dtype=bool)
    for a in range(dim):
        inside &= (p[:, a] > lo[a]) & (p[:, a] < hi[a])
    return p[~inside]


# ----------------------------------------------------------------------------
# shapes (phase membership)
# ----------------------------------------------------------------------------

def _legendre(n: int, x: np.ndarray) -> np.ndarray:
    if n == 0:
        return np.ones_like(x)
    if n == 1:
        return x
    if n == 2:
        return 0.5 * (3 * x * x - 1)
    if n == 3:
        return 0.5 * (5 * x ** 3 - 3 * x)
    raise ValueError(n)


def shape_mask(pos: np.ndarray, center: Sequence[float], R: float,
               shape: str = "circle", amp: float = 0.0) -> np.ndarray:
    """Particles inside the droplet.

    shape: ``circle`` (circle/sphere), ``mode2``/``mode3`` (surface
    r = R (1 + amp cos(n theta)) in 2D, r = R (1 + amp P_n(cos theta)) in 3D,
    theta measured from the last axis), ``square`` (square of side R sqrt(pi)
    in 2D, cube of side R (4 pi / 3)^(1/3) in 3D: the same area/volume as the
    circle/sphere of radius R).
    """
    dim = pos.shape[1]
    d = pos - np.asarray(center, dtype=float)[:dim]
    r = np.sqrt((d * d).sum(axis=1))
    if shape == "circle":
        return r < R
    if shape in ("mode2", "mode3"):
        n = 2 if shape == "mode2" else 3
        with np.errstate(invalid="ignore", divide="ignore"):
            if dim == 2:
                th = np.arctan2(d[:, 1], d[:, 0])
                rs = R * (1.0 + amp * np.cos(n * th))
            else:
                c = np.where(r > 0, d[:, 2] / np.where(r > 0, r, 1.0), 1.0)
                rs = R * (1.0 + amp * _legendre(n, c))
        return r < rs
    if shape == "square":
        side = R * math.sqrt(math.pi) if dim == 2 else R * (4.0 * math.pi / 3.0) ** (1.0 / 3.0)
        return np.all(np.abs(d) < 0.5 * side, axis=1)
    raise ValueError(shape)


# ----------------------------------------------------------------------------
# generic droplet-in-box builder
# ----------------------------------------------------------------------------

def droplet_case(name: str, dim: int, lo, hi, dx: float, center, R: float, *,
                 shape: str = "circle", amp: float = 0.0,
                 rho_l: float = 1000.0, rho_g: float = 1.0,
                 mu_l: float = 0.1, mu_g: float = 0.001,
                 sigma: float = 1.0, c0: float = 10.0,
                 drop_vel: Optional[Sequence[float]] = None,
                 vel_fn: Optional[Callable[[np.ndarray], np.ndarray]] = None,
                 walls: bool = True, t_end: Optional[float] = None,
                 xi: float = -1.0, h_factor: float = 1.3) -> Case:
    """A droplet (fluid 0) inside a second fluid (fluid 1) in a walled box."""
    lo = [float(v) for v in lo][:dim]
    hi = [float(v) for v in hi][:dim]
    p = lattice(lo, hi, dx)
    inside = shape_mask(p, center, R, shape, amp)
    liq = p[inside]
    gas = p[~inside]
    lvel = None
    if drop_vel is not None:
        lvel = np.tile(np.asarray(drop_vel, dtype=float)[:dim], (len(liq), 1))
    if vel_fn is not None:
        lvel = vel_fn(liq)
    phases = [Phase("fluid", liq, rho0=rho_l, eta=mu_l, vel=lvel),
              Phase("fluid", gas, rho0=rho_g, eta=mu_g)]
    if walls:
        phases.append(Phase("wall", wall_shell(lo, hi, dx)))
    return Case(name=name, dim=dim, lo=lo, hi=hi, dx=dx, gamma=sigma, c0=c0,
                h_factor=h_factor, xi=xi, phases=phases, t_end=t_end,
                meta=dict(center=list(center)[:dim], R=R, shape=shape, amp=amp))


def shear_drop_2d(Ca: float = 0.1, R: float = 1.0, L: float = 8.0, R_over_dp: int = 12,
                  rho: float = 1.0, eta: float = 1.0, U: float = 0.5,
                  t_end: float = 30.0) -> Case:
    """Drop in a Couette flow (Section 5.2): an L x L box periodic in x,
    no-slip walls at y = 0 and y = L moving with -U and +U, a drop of radius
    R at the centre with the same density and viscosity as the outer fluid.
    Shear rate G = 2U/L; the surface tension follows from the capillary number
    Ca = G eta R / gamma.  The fluid starts on the Couette profile.  The
    sound speed is ten times the larger of U and the capillary velocity
    sqrt(gamma / (rho R))."""
    dx = R / R_over_dp
    G = 2.0 * U / L
    gamma = G * eta * R / Ca
    c0 = 10.0 * max(U, math.sqrt(gamma / (rho * R)))
    lo, hi = [0.0, 0.0], [L, L]
    p = lattice(lo, hi, dx)
    inside = shape_mask(p, [0.5 * L, 0.5 * L], R)
    vel = np.zeros_like(p)
    vel[:, 0] = -U + G * p[:, 1]
    shell = wall_shell(lo, hi, dx, sides=[1])
    bottom = shell[shell[:, 1] < 0.0]
    top = shell[shell[:, 1] > L]
    phases = [Phase("fluid", p[inside], rho0=rho, eta=eta, vel=vel[inside]),
              Phase("fluid", p[~inside], rho0=rho, eta=eta, vel=vel[~inside]),
              Phase("wall", bottom, wall_vel=(-U, 0.0, 0.0)),
              Phase("wall", top, wall_vel=(U, 0.0, 0.0))]
    return Case(name=f"shear_drop_2d Ca={Ca:g}", dim=2, lo=lo, hi=hi, dx=dx, gamma=gamma, c0=c0,
                phases=phases, t_end=t_end, periodic=1,
                meta=dict(center=[0.5 * L, 0.5 * L], R=R, Ca=Ca, G=G, Re=rho * G * R * R / eta, U=U))


def periodic_blob(dim: int = 2, n_side: int = 24, seed: int = 0, jitter: float = 0.1,
                  vel_amp: float = 0.05, R_frac: float = 0.3, periodic: Optional[int] = None,
                  rho_ratio: float = 1.0) -> Case:
    """A drop in a unit box that is periodic along every axis flagged in
    `periodic` (default: all) and walled along the others; jittered lattice
    and random velocities, for neighbour and parity checks across the wrap."""
    rng = np.random.default_rng(seed)
    per = (1 << dim) - 1 if periodic is None else periodic
    dx = 1.0 / n_side
    lo, hi = [0.0] * dim, [1.0] * dim
    p = lattice(lo, hi, dx)
    p = p + rng.uniform(-jitter, jitter, p.shape) * dx
    for a in range(dim):
        if (per >> a) & 1:
            p[:, a] = np.mod(p[:, a], 1.0)
    inside = shape_mask(p, [0.5] * dim, R_frac)
    vel = rng.uniform(-vel_amp, vel_amp, p.shape)
    phases = [Phase("fluid", p[inside], rho0=rho_ratio, eta=0.05, vel=vel[inside]),
              Phase("fluid", p[~inside], rho0=1.0, eta=0.05, vel=vel[~inside])]
    walled = [a for a in range(dim) if not (per >> a) & 1]
    if walled:
        phases.append(Phase("wall", wall_shell(lo, hi, dx, sides=walled)))
    return Case(name=f"periodic_blob_{dim}d", dim=dim, lo=lo, hi=hi, dx=dx, gamma=1.0, c0=20.0,
                phases=phases, periodic=per, cfl_ac=0.4 if dim == 3 else 0.6,
                meta=dict(center=[0.5] * dim, R=R_frac))


# ----------------------------------------------------------------------------
# the paper-shaped workloads
# ----------------------------------------------------------------------------

def laplace_2d(dx: float = 0.025, R: float = 0.5, box: float = 2.0) -> Case:
    """Static circular droplet (§5.3 check, Eq. 37): R = 0.5 in a 2x2 box,
    dx = R/20 (6400 fluid particles), rho 1000/1, mu 0.1/0.001, sigma 1."""
    c = [box / 2, box / 2]
    return droplet_case("laplace_2d", 2, [0, 0], [box, box], dx, c, R,
                        shape="circle", sigma=1.0)


def laplace_3d(dx: float = 0.05, R: float = 0.5, box: float = 2.0, ratio: float = 1.0,
               eta: float = 0.05) -> Case:
    """Static spherical droplet, the 3D form of the Laplace check: R = 0.5 in
    a 2x2x2 box, drop density 1 and outer density 1/ratio, viscosities eta
    and eta/ratio (ratio 1: the paper's viscous regime of its 2D checks),
    sigma 1; the jump is 2 sigma / R."""
    c = [box / 2] * 3
    case = droplet_case("laplace_3d", 3, [0, 0, 0], [box, box, box], dx, c, R, shape="circle",
                        rho_l=1.0, rho_g=1.0 / ratio, mu_l=eta, mu_g=eta / ratio, sigma=1.0)
    case.cfl_ac = 0.4
    return case


def oscillating_3d(dx: float = 0.02, R: float = 0.5, box: float = 2.0,
                   amp: float = 0.05, rho_l: float = 1000.0, rho_g: float = 1.0,
                   mu_l: float = 0.1, mu_g: float = 0.001) -> Case:
    """3D droplet with a mode-2 perturbation r < R(1 + 0.05 P2(cos theta)) in a
    2x2x2 box, dx = R/25 (1e6 fluid particles), rho 1000/1, mu 0.1/0.001,
    sigma 1, at rest (other densities and viscosities on request)."""
    c = [box / 2] * 3
    sigma = 1.0
    # linear (Lamb) n = 2 frequency for a drop inside a second fluid
    w2 = 24.0 * sigma / (R ** 3 * (3 * rho_l + 2 * rho_g))
    tau = 2 * math.pi / math.sqrt(w2)
    case = droplet_case("oscillating_3d", 3, [0] * 3, [box] * 3, dx, c, R,
                        shape="mode2", amp=amp, sigma=sigma, t_end=3 * tau,
                        rho_l=rho_l, rho_g=rho_g, mu_l=mu_l, mu_g=mu_g)
    # the gas surface-tension term binds the acoustic step at c0 dt / h = 0.38
    # with the printed factor, at the edge of the 3D interface stability limit
    case.cfl_ac = 0.4
    return case


def oscillating_2d(R: float = 0.2, R_over_dp: int = 12, ratio: float = 1000.0,
                   V0: float = 1.0, r0: float = 0.05, gamma: float = 1.0,
                   rho_k: float = 1.0, eta_k: float = 0.05, c0: float = 10.0) -> Case:
    """Oscillating drop of §5.1: R = 0.2 in a unit box, drop fluid rho_k = 1,
    eta_k = 0.05, surrounding fluid rho_k/ratio, eta_k/(ratio/10) (ratio 1000
    gives 1e-3 and 5e-4 as in the paper), gamma = 1, and the divergence-free
    initial velocity of Eq. 34 (V0, r0) about the drop centre."""
    dx = R / R_over_dp
    rho_l = rho_k / ratio
    eta_l = eta_k / (ratio / 10.0) if ratio > 1 else eta_k

    def vel_fn(p):
        d = p - 0.5
        r = np.sqrt((d * d).sum(axis=1))
        rs = np.where(r > 0, r, 1.0)
        ex = np.exp(-r / r0)
        vx = V0 * d[:, 0] / r0 * (1.0 - d[:, 1] ** 2 / (r0 * rs)) * ex
        vy = -V0 * d[:, 1] / r0 * (1.0 - d[:, 0] ** 2 / (r0 * rs)) * ex
        return np.stack([vx, vy], axis=1)

    case = droplet_case("oscillating_2d", 2, [0, 0], [1, 1], dx, [0.5, 0.5], R,
                        shape="circle", rho_l=rho_k, rho_g=rho_l, mu_l=eta_k, mu_g=eta_l,
                        sigma=gamma, c0=c0)
    for ph in case.phases:
        if ph.kind == "fluid":
            ph.vel = vel_fn(ph.pos)
    case.meta.update(V0=V0, r0=r0)
    return case


def impact_3d(dx: float = 1.0 / 60.0) -> Case:
    """Droplet D = 1 moving at U = 1 towards the wall z = 0, centred 0.6 above
    it in a 4x4x2 box; rho 1000/1, mu 0.1/0.001, sigma 0.04 (Re = 1e4,
    We = 2.5e4, Eq. 38); dx = D/60."""
    case = droplet_case("impact_3d", 3, [0, 0, 0], [4, 4, 2], dx, [2, 2, 0.6],
                        0.5, shape="circle", sigma=0.04,
                        drop_vel=[0, 0, -1.0], t_end=2.0)
    case.cfl_ac = 0.4      # the sound term binds the acoustic step here
    return case


def impact_sweep_case(U0: float, d_over_dp: int = 20) -> Case:
    """Section 5.4's impact in the paper's own units: a drop of diameter
    d = 1 resting on the wall z = 0 at the centre of an 8 x 8 x 1.5 box,
    moving down at U0; rho 1 / 0.001, mu 0.005 / 5e-5, gamma 0.1, so
    Re = 200 U0 and We = 10 U0^2; c0 = 10 U0.  The paper's end times: 4.0,
    and 0.1 for U0 = 50."""
    dx = 1.0 / d_over_dp
    case = droplet_case(f"impact_U{U0:g}", 3, [0, 0, 0], [8, 8, 1.5], dx, [4, 4, 0.5], 0.5,
                        rho_l=1.0, rho_g=0.001, mu_l=0.005, mu_g=5e-5, sigma=0.1, c0=10.0 * U0,
                        drop_vel=[0, 0, -U0], t_end=0.1 if U0 >= 50 else 4.0)
    case.cfl_ac = 0.4
    case.meta.update(U0=U0, Re=200.0 * U0, We=10.0 * U0 * U0)
    return case


def small_droplet(dim: int = 2, n_side: int = 24, R_frac: float = 0.3,
                  shape: str = "circle", amp: float = 0.0, sigma: float = 1.0,
                  rho_l: float = 1000.0, rho_g: float = 1.0,
                  mu_l: float = 0.1, mu_g: float = 0.001, c0: float = 10.0,
                  walls: bool = True, seed: Optional[int] = None,
                  jitter: float = 0.0, vel_amp: float = 0.0) -> Case:
    """A reduced droplet case sized for the CPU oracle (unit box).

    ``jitter`` displaces particles by a seeded uniform fraction of dx and
    ``vel_amp`` gives them seeded random velocities, so that parity tests
    exercise irregular pair geometry and all terms of the Riemann solver.
    """
    dx = 1.0 / n_side
    lo, hi = [0.0] * dim, [1.0] * dim
    case = droplet_case(f"small_{dim}d_{n_side}", dim, lo, hi, dx, [0.5] * dim,
                        R_frac, shape=shape, amp=amp, sigma=sigma, rho_l=rho_l,
                        rho_g=rho_g, mu_l=mu_l, mu_g=mu_g, c0=c0, walls=walls)
    if dim == 3:
        case.cfl_ac = 0.4      # coarse 3D cases are bound by the sound term
    if seed is not None and (jitter > 0 or vel_amp > 0):
        rng = np.random.default_rng(seed)
        for ph in case.phases:
            if ph.kind != "fluid":
                continue
            if jitter > 0:
                ph.pos = ph.pos + rng.uniform(-jitter, jitter, ph.pos.shape) * dx
            if vel_amp > 0:
                ph.vel = rng.uniform(-vel_amp, vel_amp, ph.pos.shape)
    return case


def free_blob(dim: int = 2, n_side: int = 14, seed: int = 7, jitter: float = 0.2,
              vel_amp: float = 0.3, rho_ratio: float = 1000.0,
              rho_jitter: float = 0.01) -> Case:
    """Two-phase blob without walls (momentum-conservation inputs): a jittered
    lattice, inner disc/ball of fluid 0 inside fluid 1, random velocities and
    densities, seeded."""
    dx = 1.0 / n_side
    rng = np.random.default_rng(seed)
    p = lattice([0.0] * dim, [1.0] * dim, dx)
    p = p + rng.uniform(-jitter, jitter, p.shape) * dx
    inside = shape_mask(p, [0.5] * dim, 0.3, "mode2", 0.15)
    phases = []
    for mask, rho0, eta in ((inside, rho_ratio, 0.1), (~inside, 1.0, 0.001)):
        q = p[mask]
        vel = rng.uniform(-vel_amp, vel_amp, q.shape)
        rho = rho0 * (1.0 + rng.uniform(-rho_jitter, rho_jitter, len(q)))
        phases.append(Phase("fluid", q, rho0=rho0, eta=eta, vel=vel, rho=rho))
    return Case(name=f"blob_{dim}d", dim=dim, lo=[0.0] * dim, hi=[1.0] * dim,
                dx=dx, gamma=1.0, c0=10.0, phases=phases)


# ----------------------------------------------------------------------------
# batched and served workloads
# ----------------------------------------------------------------------------

BATCH_SEED = 20250320
SERVE_SEED = 20250321


@dataclasses.dataclass
class CaseSpec:
    """A lazily built droplet case of the batched/served workloads."""

    index: int
    dim: int
    n_target: int
    R: float
    sigma: float
    shape: str
    amp: float
    arrival: float = 0.0

    def build(self) -> Case:
        box = 4.0 * self.R
        m = max(8, int(round(self.n_target ** (1.0 / self.dim))))
        dx = box / m
        c = [box / 2] * self.dim
        case = droplet_case(f"case{self.index}_{self.dim}d", self.dim,
                            [0.0] * self.dim, [box] * self.dim, dx, c, self.R,
                            shape=self.shape, amp=self.amp, sigma=self.sigma)
        case.meta["spec"] = dataclasses.asdict(self)
        case.cfl_ac = 0.4      # small or weakly tensioned cases are bound by the sound term
        return case


def _draw_specs(rng, n: int, n_lo: float, n_hi: float, p3: float = 0.5):
    specs = []
    for i in range(n):
        dim = 3 if rng.random() < p3 else 2
        n_t = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        R = rng.uniform(0.2, 0.5)
        sigma = math.exp(rng.uniform(math.log(0.1), math.log(10.0)))
        shape = ("square", "mode2", "mode3")[int(rng.integers(0, 3))]
        amp = rng.uniform(0.0, 0.2) if shape != "square" else 0.0
        specs.append(CaseSpec(i, dim, n_t, R, sigma, shape, amp))
    return specs


def batch_cases(n_cases: int = 512, seed: int = BATCH_SEED,
                n_lo: float = 2e3, n_hi: float = 2e5) -> List[CaseSpec]:
    """Independent 2D/3D droplet relaxation cases (dims 1:1, particle count
    log-uniform in [n_lo, n_hi], R ~ U[0.2, 0.5], sigma log-uniform in
    [0.1, 10], shape square / mode-2 / mode-3 with amplitude U[0, 0.2])."""
    rng = np.random.default_rng(seed)
    return _draw_specs(rng, n_cases, n_lo, n_hi)


def served_stream(n_requests: int, seed: int = SERVE_SEED, rate: float = 50.0,
                  n_lo: float = 5e3, n_hi: float = 2e6) -> List[CaseSpec]:
    """Poisson arrivals (mean ``rate`` per second) of droplet cases drawn like
    ``batch_cases`` but with particle counts log-uniform in [n_lo, n_hi]."""
    rng = np.random.default_rng(seed)
    specs = _draw_specs(rng, n_requests, n_lo, n_hi)
    t = 0.0
    for s in specs:
        t += rng.exponential(1.0 / rate)
        s.arrival = t
    return specs
