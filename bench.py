#!/usr/bin/env python3
"""Benchmark of the multiphase SPH pair-sweep path on GB300.

Workload (default): the 3D oscillating droplet -- sphere R = 0.5 with a
mode-2 perturbation of amplitude 0.05 R in a 2x2x2 box, dx = R/25
(1,000,000 fluid + 191,016 wall particles), density ratio 1000, viscosity
ratio 100, sigma = 1, at rest, FP32 pair arithmetic with FP64 reductions.

One timed step is one advection step of the dual-criteria scheme: cell-list
rebuild, correction matrix, viscous force + transport shift, then all its
acoustic substeps (~67 here), each with the criterion, colour gradient,
force + kick and continuity + drift sweeps.  The metric counts
particle-substeps: fluid particles times acoustic substeps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun) runs one independent replica per GPU ("replicas only":
a single case does not shard without a halo exchange); value is the sum of
all ranks' particle-substeps over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import sphcases  # noqa: E402

METRIC = "particle-substeps/s"

# ncu summaries record the DRAM traffic of a kernel together with a hash of
# the kernel sources it was taken on; the bench reports it only while the
# sources are unchanged
KERNEL_SOURCES = ("paper_2503_16082_gb300/csrc/sphst_kernels.cuh", "paper_2503_16082_gb300/csrc/sphst_internal.cuh")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(summary: str, kernel: str, key: str = "traffic_bytes_per_launch"):
    """DRAM bytes (or another recorded per-launch count, `key`) of `kernel`
    from a profiles/ summary, or None if the summary is missing or was taken
    on other kernel sources."""
    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"source_sha256:\s*([0-9a-f]+)", text)
    if not m or m.group(1) != kernel_source_hash():
        return None
    m = re.search(re.escape(key) + r"\[" + re.escape(kernel) + r"\]:\s*([0-9]+)", text)
    return int(m.group(1)) if m else None
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12     # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz
# algorithmic flops per neighbour pair, counted from the formulas (adds and
# multiplies 1, fused multiply-adds 2, divisions and square roots 1):
FP64_PEAK_TFLOPS = 1.25      # nominal FP64 (non-tensor) rate of a GB300
FLOPS_PAIR_B = 59            # geometry + Riemann pressure, every pair (sweep B)
FLOPS_PAIR_B_SURF = 110      # surface stress + penalty, pairs touching the interface (sweep S)
L2_BYTES = 129 * 10**6       # L2 of a GB300; a case smaller than twice this is flushed between timed steps


def workload(name: str):
    if name == "oscillating_3d":
        return sphcases.oscillating_3d()
    if name == "laplace_2d":
        return sphcases.laplace_2d()
    if name == "impact_3d":
        return sphcases.impact_3d()
    raise SystemExit(f"unknown workload {name}")


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.first = 0
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)

    def _lines(self) -> int:
        try:
            with open(self.path) as f:
                return sum(1 for _ in f)
        except OSError:
            return 0

    def start(self):
        """Start sampling every 100 ms; returns once the first sample is in,
        and marks the samples before the timed region as not under load."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t0 = time.time()
        while self._lines() == 0 and time.time() - t0 < 3.0 and self.proc.poll() is None:
            time.sleep(0.02)
        self.first = self._lines()

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for k, line in enumerate(open(self.path)):
            parts = [p.strip() for p in line.split(",")]
            if k >= self.first and len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if "Active" in r[5 + k] and "Not" not in r[5 + k]:
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ------------------------------------------------------------ distributed
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Dist:
    """Replica bookkeeping over torch.distributed.  A rank that dies or never
    arrives turns the others' next barrier or reduction into an error after
    `timeout_s` (SPHST_BENCH_PG_TIMEOUT_S, default 600 s) instead of a hang."""

    def __init__(self, backend: str, timeout_s: float = None):
        self.ws, self.rank, self.local = dist_env()
        self.pg = None
        if self.ws > 1:
            import datetime

            import torch.distributed as dist
            if timeout_s is None:
                timeout_s = float(os.environ.get("SPHST_BENCH_PG_TIMEOUT_S", "600"))
            dist.init_process_group(backend, timeout=datetime.timedelta(seconds=timeout_s))
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        return self._reduce(x, "max")

    def sum(self, x: float) -> float:
        return self._reduce(x, "sum")

    def _reduce(self, x, op):
        if not self.pg:
            return x
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX if op == "max" else self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def aggregate(dist: Dist, units: float, seconds: float):
    """Whole-job value: units summed over ranks / slowest rank's time."""
    total = dist.sum(units)
    tmax = dist.max(seconds)
    return total / tmax, tmax, total


# ----------------------------------------------------------- our arm
def run_ours(args, dist: Dist):
    import torch

    import paper_2503_16082_gb300 as S

    torch.cuda.set_device(dist.local)
    stream = torch.cuda.current_stream()
    spec = workload(args.workload)
    n_fluid = spec.n_fluid

    nbr_mode = S.NBR_CELLS if args.nbr == "cells" else S.NBR_LIST
    extra = {"block": args.block} if args.block else {}
    if args.lanes:
        extra["lanes"] = args.lanes
    if args.loop == "host":                      # every kernel a launch of its own (profilers see them)
        extra["loop_mode"] = S.LOOP_HOST
    h = S.case_from_spec(spec, precision=args.precision, nbr_mode=nbr_mode, **extra)
    S.set_stream(h, stream.cuda_stream)
    S.step(h, args.warmup)                       # engine set-up, graph capture, warm-up
    info0 = S.case_info(h)
    # a case whose state fits in L2 is evicted before each timed advection
    # step by writing a buffer twice the L2 size, outside the events
    state_bytes = S.footprint_bytes(S.params_from_spec(spec, args.precision, nbr_mode=nbr_mode, **extra), spec.n)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda") if state_bytes < 2 * L2_BYTES else None
    l2_note = (f"inputs larger than L2 ({state_bytes / 1e6:.0f} MB of case state on the device vs 129 MB L2)"
               if flush is None else
               f"L2 flushed before each timed step (case state {state_bytes / 1e6:.1f} MB; a 258 MB buffer "
               f"written between steps, outside the timed events)")

    clocks = ClockSampler(dist.local)
    clocks.start()
    dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if flush is None:
        ev0.record(stream)
        S.step(h, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
    else:
        ms = 0.0
        for _ in range(args.steps):
            flush.fill_(1)
            ev0.record(stream)
            S.step(h, 1)
            ev1.record(stream)
            torch.cuda.synchronize()
            ms += ev0.elapsed_time(ev1)
    dist.barrier()
    clk = clocks.stop()
    info1 = S.case_info(h)
    n_sub = info1["n_sub"] - info0["n_sub"]
    units = float(n_fluid) * n_sub
    value, tmax, total_units = aggregate(dist, units, ms / 1e3)
    # live per-kernel timing of one more advection step (events around each
    # launch on the same stream) for the roofline of the dominant kernel
    prof = S.profile_step(h)
    # kernels launched in the timed region, from the launch counts of that
    # step: set-up kernels + 1 closing kernel per advection step, the
    # per-substep kernels (criterion, A, S, B, C) per substep
    prof_sub = max(prof["criterion"][1], 1)
    per_step = prof["rebuild"][1] + prof["setup"][1] + 1
    per_sub = sum(prof[g][1] for g in ("criterion", "sweep_A", "sweep_S", "sweep_B", "sweep_C")) / prof_sub
    launches = int(round(args.steps * per_step + n_sub * per_sub))
    counts = S.debug_neighbor_counts(h)
    phase = S.read_fields(h, S.FIELD_PHASE, spec.dim)
    gradc = S.read_fields(h, S.FIELD_GRADC, spec.dim)
    kinds = [0 if p.kind == "fluid" else 2 for p in spec.phases]
    is_fluid = np.array([kinds[int(k)] < 2 for k in phase])
    iface = is_fluid & (np.abs(gradc).max(axis=1) > 0)
    pairs = int(counts[is_fluid].sum())
    pairs_surf = int(min(2 * counts[iface].sum(), pairs))
    b_ms, b_launches = prof["sweep_B"]
    b_avg = b_ms / max(b_launches, 1) / 1e3
    # sweep B carries the pressure pairs; with the neighbour list the surface
    # pairs run in sweep S, with the cell walk in B itself
    surf_in_b = args.nbr == "cells"
    flops = FLOPS_PAIR_B * pairs + (FLOPS_PAIR_B_SURF * pairs_surf if surf_in_b else 0)
    achieved = flops / b_avg / 1e12
    f32 = args.precision == 32
    peak = FP32_PEAK_TFLOPS if f32 else FP64_PEAK_TFLOPS
    roofline = {"bound": "alu",
                "kernel": f"k_sweep_B<{'float' if f32 else 'double'}, {spec.dim}, {'false' if surf_in_b else 'true'}>",
                "achieved": round(achieved, 3),
                "peak": round(peak, 2), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4),
                "traffic": (recorded_traffic(f"sweeps_{args.workload}_f{args.precision}_{args.nbr}.md", "k_sweep_B")
                            if f32 and not surf_in_b else None),
                "peak_source": ("derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz" if f32
                                else "nominal FP64 rate of a GB300"),
                "flops_per_launch": flops, "pairs": pairs, "pairs_surface": pairs_surf,
                "avg_launch_ms": round(b_avg * 1e3, 4)}
    # the issue roof beside the ALU one: warp instructions of one launch (ncu,
    # recorded with the traffic) over its live duration, against one warp
    # instruction per scheduler per cycle (152 SMs x 4 x 2.07 GHz)
    insts = (recorded_traffic(f"sweeps_{args.workload}_f{args.precision}_{args.nbr}.md", "k_sweep_B",
                              "warp_instructions_per_launch") if f32 and not surf_in_b else None)
    if insts:
        issue_peak = 152 * 4 * 2.07e9
        roofline["issue"] = {"warp_instructions": insts, "achieved": round(insts / b_avg / 1e12, 4),
                             "peak": round(issue_peak / 1e12, 4), "unit": "T warp-instructions/s",
                             "frac": round(insts / b_avg / issue_peak, 4)}
    try:                                   # measured FMA roof beside the derived one
        roofline["peak_measured_fma"] = round(S.fma_peak(args.precision)["tflops"], 2)
        roofline["frac_of_measured_fma"] = round(achieved / roofline["peak_measured_fma"], 4)
    except Exception as e:                 # noqa: BLE001 - report, keep the bench line
        roofline["peak_measured_fma"] = f"unavailable: {e}"
    if not surf_in_b and prof["sweep_S"][1]:
        s_avg = prof["sweep_S"][0] / prof["sweep_S"][1] / 1e3
        roofline["sweep_S"] = {"avg_launch_ms": round(s_avg * 1e3, 4),
                               "achieved": round(FLOPS_PAIR_B_SURF * pairs_surf / s_avg / 1e12, 3)}
    kernel_ms = {g: {"ms": round(m, 3), "launches": l} for g, (m, l) in prof.items()}
    S.destroy(h)

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2 = S.case_from_spec(spec, precision=args.precision, nbr_mode=nbr_mode, **extra)
        S.set_stream(h2, stream.cuda_stream)
        d2h = 0
        e_sub0 = 0
        # the result lands in pinned host memory, as a caller streaming it
        # out would keep it
        pinned = torch.empty(spec.n * spec.dim, dtype=torch.float64, pin_memory=True).numpy()
        for k in range(args.steps):
            S.step(h2, 1)
            pos = S.read_fields(h2, S.FIELD_POS, spec.dim, out=pinned)
            d2h += pos.nbytes
        e_sub = S.case_info(h2)["n_sub"] - e_sub0
        t1 = time.perf_counter()
        S.destroy(h2)
        e_val, _, _ = aggregate(dist, float(n_fluid) * e_sub, t1 - t0)
        h2d = spec.n * (3 + 3 + 1) * 8
        e2e = {"value": round(e_val, 1), "unit": METRIC,
               "h2d_bytes_per_step": int(h2d / max(args.steps, 1)),
               "d2h_bytes_per_step": int(d2h / max(args.steps, 1)),
               "note": "case upload + engine set-up + graph capture + K x (step, read positions into pinned host memory)"}

    return {
        "value": value, "ms_per_step": tmax * 1e3 / args.steps, "units": total_units,
        "n_sub": n_sub, "roofline": roofline, "e2e": e2e, "gpu_launches": launches,
        "clocks": clk, "kernel_ms": kernel_ms, "n_fluid": n_fluid, "n_total": spec.n, "l2": l2_note,
    }


# ------------------------------------------------------ CPU oracle sample
SAMPLE_SUBSTEPS = 4


def oracle_sample(spec, substeps: int = SAMPLE_SUBSTEPS):
    """Time the oracle as it stands on the full workload: one advection
    step's set-up (neighbour search, viscous force, transport shift) plus
    `substeps` acoustic substeps.  Returns (particle-substeps/s, seconds, threads)."""
    import oracle

    pos, vel, rho, kind = spec.flat()
    P = oracle.params_for_case(spec, max_substeps=substeps)
    t0 = time.perf_counter()
    _, _, _, info, _, _ = oracle.run(P, pos, vel, rho, kind, 1)
    dt = time.perf_counter() - t0
    return spec.n_fluid * info["n_sub"] / dt, dt, oracle.max_threads(), info["n_sub"]


def run_reference(args, dist: Dist):
    if dist.rank != 0:
        return None
    spec = workload(args.workload)
    for _ in range(args.warmup):
        oracle_sample(spec, 1)
    units = 0.0
    secs = 0.0
    threads = 0
    for _ in range(args.steps):
        rate, dt, threads, nsub = oracle_sample(spec)
        units += spec.n_fluid * nsub
        secs += dt
    value = units / secs
    return {"value": value, "ms_per_step": secs * 1e3 / max(args.steps, 1), "threads": threads,
            "sample": f"full {args.workload} ({spec.n} particles): per step one advection-step "
                      f"set-up + {SAMPLE_SUBSTEPS} acoustic substeps of the FP64 oracle"}


# ------------------------------------------------------ batched and served
def run_batch(args):
    """The batched workload: independent 2D/3D droplet cases advanced together in one
    engine (one graph per advection step), against the same cases stepped
    one at a time through the single-case path."""
    import torch

    import paper_2503_16082_gb300 as S

    torch.cuda.set_device(0)
    specs = sphcases.batch_cases(args.cases)
    cases = [sp.build() for sp in specs]
    # coarse 3D drops with strong tension cluster beyond the default list
    # capacity of 128 neighbours; the batch uses 192
    hs = [S.case_from_spec(c, precision=args.precision, max_neighbors=192 if c.dim == 3 else 0)
          for c in cases]
    state_bytes = sum(S.footprint_bytes(S.params_from_spec(c, args.precision, max_neighbors=192 if c.dim == 3 else 0),
                                        c.n) for c in cases)
    b = S.batch_create(args.precision)
    for h in hs:
        S.batch_add(b, h)
    S.batch_step(b, args.warmup)
    sub0 = [S.case_info(h)["n_sub"] for h in hs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S.batch_step(b, args.steps)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    units = sum(c.n_fluid * (S.case_info(h)["n_sub"] - s0) for c, h, s0 in zip(cases, hs, sub0))
    statuses = [S.case_info(h)["status"] for h in hs]
    for h in hs:
        S.batch_remove(b, h)
        S.destroy(h)
    S.batch_destroy(b)
    # the single-case path on a sample of the same cases
    k = min(args.plain_sample, len(cases))
    punits, psecs = 0, 0.0
    for c in cases[:k]:
        h = S.case_from_spec(c, precision=args.precision, max_neighbors=192 if c.dim == 3 else 0)
        S.step(h, args.warmup)
        s0 = S.case_info(h)["n_sub"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.step(h, args.steps)
        torch.cuda.synchronize()
        psecs += time.perf_counter() - t0
        punits += c.n_fluid * (S.case_info(h)["n_sub"] - s0)
        S.destroy(h)
    # the oracle as it stands on a bounded sample of the same cases (one
    # advection-step set-up + a few substeps each, about 10 s of host time)
    cpu = None
    if not args.no_cpu_baseline:
        cu, cs, used, threads = 0.0, 0.0, 0, 0
        for c in cases:
            _, secs, threads, nsub = oracle_sample(c)
            cu += c.n_fluid * nsub
            cs += secs
            used += 1
            if cs > 10.0 or used >= 16:
                break
        cpu = {"value": round(cu / cs, 1), "unit": METRIC, "cores": threads, "kind": "oracle",
               "sample": f"the batch's first {used} cases, each one advection-step set-up + "
                         f"{SAMPLE_SUBSTEPS} acoustic substeps of the FP64 oracle, {cs:.1f} s"}
    line = {"metric": METRIC, "mode": "batch", "value": round(units / dt, 1), "unit": METRIC,
            "cases": len(cases), "particles": int(sum(c.n for c in cases)),
            "fluid_particles": int(sum(c.n_fluid for c in cases)), "steps": args.steps,
            "warmup": args.warmup, "seconds": round(dt, 3), "failed_cases": int(sum(1 for x in statuses if x)),
            "failed_status": {str(x): int(sum(1 for y in statuses if y == x)) for x in set(statuses) if x},
            "failed_specs": [dict(dim=sp.dim, n=c.n, sigma=round(sp.sigma, 3), shape=sp.shape)
                             for sp, c, x in zip(specs, cases, statuses) if x][:8],
            "plain_single_case": {"value": round(punits / psecs, 1), "cases_sampled": k},
            "speedup_vs_plain": round((units / dt) / (punits / psecs), 2), "cpu_baseline": cpu,
            "dtype": "f32" if args.precision == 32 else "f64", "data": "synthetic",
            "config": {"workload": "batch_cases seed 20250320", "step": "one advection step of every case",
                       "l2": f"inputs larger than L2 ({state_bytes / 1e9:.1f} GB of case state vs 129 MB L2)"}}
    print(json.dumps(line), flush=True)


def run_serve(args):
    """The served workload: Poisson arrivals of droplet cases into the continuous-batching
    server; p50/p99 time from submission to result."""
    import torch

    import paper_2503_16082_gb300 as S
    from paper_2503_16082_gb300 import serve

    torch.cuda.set_device(0)
    specs = sphcases.served_stream(args.requests, rate=args.rate, n_hi=args.serve_n_hi)
    cases = [sp.build() for sp in specs]
    # capacity first: a batch of the stream's first cases, one advection step
    # each after a warm-up step; the offered load (arrival rate x mean fluid
    # particles x substeps per request) must stay below 0.9 of it, else the
    # substep count per request is lowered
    probe = cases[:min(len(cases), args.capacity_cases)]
    b = S.batch_create(args.precision)
    hs = [S.case_from_spec(c, precision=args.precision) for c in probe]
    for h in hs:
        S.batch_add(b, h)
    S.batch_step(b, 1)
    s0 = [S.case_info(h)["n_sub"] for h in hs]
    torch.cuda.synchronize()
    tc = time.perf_counter()
    S.batch_step(b, 2)
    torch.cuda.synchronize()
    tc = time.perf_counter() - tc
    capacity = sum(c.n_fluid * (S.case_info(h)["n_sub"] - s) for c, h, s in zip(probe, hs, s0)) / tc
    for h in hs:
        S.batch_remove(b, h)
        S.destroy(h)
    S.batch_destroy(b)
    mean_fluid = float(np.mean([c.n_fluid for c in cases]))
    n_sub = args.serve_substeps
    while n_sub > 1 and args.rate * mean_fluid * n_sub > 0.9 * capacity:
        n_sub -= 1
    offered = args.rate * mean_fluid * n_sub
    srv = serve.Server(precision=args.precision, budget_bytes=args.budget_gb * 1e9)
    srv.start()
    t0 = time.perf_counter()
    futs = []
    for sp, c in zip(specs, cases):
        delay = t0 + sp.arrival - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        futs.append(srv.submit(c, n_sub=n_sub))
    res = [f.result(timeout=3600) for f in futs]
    wall = time.perf_counter() - t0
    srv.stop()
    st = srv.stats()
    srv.close()
    lat = np.array([r.latency for r in res])
    line = {"metric": METRIC, "mode": "serve", "value": round(st["particle_substeps"] / wall, 1),
            "unit": METRIC, "requests": len(res), "arrival_rate_per_s": args.rate,
            "p50_latency_s": round(float(np.percentile(lat, 50)), 4),
            "p99_latency_s": round(float(np.percentile(lat, 99)), 4),
            "gpu_busy_fraction": round(st["busy_s"] / wall, 3), "rounds": st["rounds"],
            "failed": int(sum(1 for r in res if r.info["status"])),
            "substeps_per_request": n_sub, "substeps_requested": args.serve_substeps,
            "capacity": round(capacity, 1), "offered_load": round(offered, 1),
            "offered_fraction": round(offered / capacity, 3), "budget_gb": args.budget_gb,
            "particles_per_request_range": [5e3, args.serve_n_hi],
            "dtype": "f32" if args.precision == 32 else "f64", "data": "synthetic",
            "config": {"workload": "served_stream seed 20250321", "wall_s": round(wall, 2)}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="oscillating_3d")
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--nbr", default="list", choices=["list", "cells"],
                    help="neighbour source of the sweeps (list built per advection step, or cell walk)")
    ap.add_argument("--block", type=int, default=0, help="particles per tile / threads per block (0: library default)")
    ap.add_argument("--loop", default="graph", choices=["graph", "host"],
                    help="graph: one CUDA graph per advection step (the default, timed); host: the same kernels "
                         "launched one by one with a host check per substep, for profilers")
    ap.add_argument("--lanes", type=int, default=0, choices=[0, 1, 2, 4, 8],
                    help="lanes per particle in sweeps A, B, C with the list (0: library default, 1)")
    ap.add_argument("--mode", default="single", choices=["single", "batch", "serve"],
                    help="single: the headline line; batch / serve: the batched and served workloads")
    ap.add_argument("--cases", type=int, default=512)
    ap.add_argument("--plain-sample", type=int, default=32)
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--serve-substeps", type=int, default=128,
                    help="acoustic substeps per served request (lowered to keep the offered load below 0.9 of capacity)")
    ap.add_argument("--capacity-cases", type=int, default=24)
    ap.add_argument("--serve-n-hi", type=float, default=2e6)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "serve":
        return run_serve(args)

    ws, rank, local = dist_env()
    config = {"workload": args.workload, "particles": None, "fluid_particles": None,
              "step": "one advection step (rebuild + all acoustic substeps)",
              "l2": None,
              "parallelism": f"replicas x{max(ws, 1)}", "neighbours": args.nbr,
              "block": args.block or 128, "lanes": args.lanes or 1, "loop": args.loop}
    dtype = "f32" if args.precision == 32 else "f64"

    if args.impl == "reference":
        dist = Dist("gloo")                    # the oracle runs on the host: no NCCL needed
        res = run_reference(args, dist)
        dist.close()
        if res is None:
            return
        spec_n = workload(args.workload)
        config.update(particles=spec_n.n, fluid_particles=spec_n.n_fluid,
                      l2="not applicable: the oracle runs on the host cores")
        line = {"impl": "reference", "metric": METRIC, "value": round(res["value"], 1),
                "unit": METRIC, "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(res["ms_per_step"], 1), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": config,
                "cpu_baseline": {"value": round(res["value"], 1), "unit": METRIC, "cores": res["threads"],
                                 "kind": "oracle", "sample": res["sample"]},
                "e2e": {"value": round(res["value"], 1), "unit": METRIC,
                        "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    dist = Dist("nccl")
    res = run_ours(args, dist)
    config.update(particles=res["n_total"], fluid_particles=res["n_fluid"], l2=res["l2"],
                  substeps_per_step=round(res["n_sub"] / args.steps, 2))
    cpu = None
    if rank == 0 and ws <= 1 and not args.no_cpu_baseline:
        spec = workload(args.workload)
        rate, dt, threads, nsub = oracle_sample(spec)
        cpu = {"value": round(rate, 1), "unit": METRIC, "cores": threads, "kind": "oracle",
               "sample": f"full {args.workload}: one advection-step set-up + {nsub} acoustic "
                         f"substeps of the FP64 oracle, {dt:.1f} s"}
    dist.close()
    if rank != 0:
        return
    line = {"metric": METRIC, "value": round(res["value"], 1), "unit": METRIC, "n_gpus": max(ws, 1),
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(res["ms_per_step"], 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic", "config": config, "roofline": res["roofline"],
            "cpu_baseline": cpu, "e2e": res["e2e"], "gpu_launches": res["gpu_launches"],
            "clocks": res["clocks"], "kernel_ms_one_step": res["kernel_ms"]}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
