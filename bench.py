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
# sources are unchanged.  The hash covers the code, not the comments: line
# comments are dropped and each line's whitespace is normalised first.
KERNEL_SOURCES = ("paper_2503_16082_gb300/csrc/sphst_kernels.cuh", "paper_2503_16082_gb300/csrc/sphst_internal.cuh")


def _code_of(text: str) -> str:
    lines = []
    for line in text.splitlines():
        code = re.sub(r"//.*", "", line).strip()
        if code:
            lines.append(" ".join(code.split()))
    return "\n".join(lines)


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            h.update(_code_of(fh.read()).encode())
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
# FP32 lanes per SM of compute capability 10.x (GB300): the arithmetic roof
# is SMs x lanes x 2 flop (FMA) x peak SM clock, with the SM count and clock
# read from the device (sphst_device_info)
FP32_LANES_PER_SM = 128
ISSUE_PER_SM = 4             # warp schedulers per SM: one warp instruction each per cycle
# algorithmic flops per neighbour pair, counted from the formulas (adds and
# multiplies 1, fused multiply-adds 2, divisions and square roots 1):
FP64_PEAK_TFLOPS = 1.25      # nominal FP64 (non-tensor) rate of a GB300
FLOPS_PAIR_B = 59            # geometry + Riemann pressure, every pair (sweep B)
FLOPS_PAIR_B_SURF = 110      # surface stress + penalty, pairs touching the interface (sweep S)
L2_BYTES = 129 * 10**6       # L2 of a GB300; a case smaller than twice this is flushed between timed steps
HBM_FALLBACK_GBS = 6800.0    # one earlier copy-bandwidth measurement on a GB300, used without a measured one


def hbm_roof(traffic_bytes: int, launch_s: float, root: str | None = None) -> dict:
    """A kernel's DRAM bytes per launch (ncu) over its live launch time,
    against the measured HBM copy bandwidth of this GPU model
    (MEASURED_PEAKS.json beside this file), else a fallback figure."""
    path = os.path.join(root or ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            peak, src = float(json.load(f)["hbm_gbs"]), "measured copy bandwidth (MEASURED_PEAKS.json)"
    except (OSError, KeyError, TypeError, ValueError):
        peak, src = HBM_FALLBACK_GBS, "fallback: an earlier GB300 copy measurement"
    gbs = traffic_bytes / launch_s / 1e9
    return {"achieved": round(gbs, 1), "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4),
            "peak_source": src}


def device_roofs():
    """FP32 arithmetic roof (TFLOP/s) and warp-instruction issue roof
    (instructions/s) of the current GPU, from its SM count and peak SM
    clock as the device reports them."""
    import paper_2503_16082_gb300 as S

    info = S.device_info()
    sm, ghz = info["sm_count"], info["max_sm_clock_khz"] / 1e6
    return {"sm_count": sm, "max_sm_clock_mhz": round(ghz * 1e3, 1), "cc": list(info["cc"]),
            "fp32_tflops": sm * FP32_LANES_PER_SM * 2 * ghz * 1e9 / 1e12,
            "issue_per_s": sm * ISSUE_PER_SM * ghz * 1e9}


# Launch shape of a workload's line where it differs from the library's
# default of 128 threads per block (speed only: with one lane per particle
# no particle's sums depend on the block size, and the results are the same
# bit for bit).  The 3D drop in FP32 with the list: 256 threads 1.547e9
# particle-substeps/s against 1.516e9 with 128 (sweep C 0.244 against
# 0.255 ms per launch, B the same), 160: 1.532e9, 192: 1.517e9.
TUNED_BLOCK = {("oscillating_3d", 32, "list"): 256}
# the same for the batched workload (one engine of 512 cases): 256 threads
# 1.513-1.515e9 against 1.497-1.500e9 with 128, the work-list variant
# 1.443e9 against 1.394e9; its cases stepped one by one stay at the
# library's default (676 against 666 M particle-substeps/s at 256)
BATCH_BLOCK = 256


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
    roofs = device_roofs()
    peak = roofs["fp32_tflops"] if f32 else FP64_PEAK_TFLOPS
    roofline = {"bound": "alu",
                # the instantiation a one-case engine launches: <T, D, list, lanes, mode>
                # (mode 2: the case's constants in the launch parameters; the
                # cell-walk classes run mode 0)
                "kernel": (f"k_sweep_B<{'float' if f32 else 'double'}, {spec.dim}, {0 if surf_in_b else 1}, "
                           f"{1 if surf_in_b else (args.lanes or 1)}, {0 if surf_in_b else 2}>"),
                "achieved": round(achieved, 3),
                "peak": round(peak, 2), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4),
                "traffic": (recorded_traffic(f"sweeps_{args.workload}_f{args.precision}_{args.nbr}.md", "k_sweep_B")
                            if f32 and not surf_in_b else None),
                "peak_source": (f"derived from the device: {roofs['sm_count']} SMs x {FP32_LANES_PER_SM} FP32 "
                                f"lanes x 2 flop x {roofs['max_sm_clock_mhz']:.0f} MHz (peak SM clock)" if f32
                                else "nominal FP64 rate of a GB300"),
                "device": {k: roofs[k] for k in ("sm_count", "max_sm_clock_mhz", "cc")},
                "flops_per_launch": flops, "pairs": pairs, "pairs_surface": pairs_surf,
                "avg_launch_ms": round(b_avg * 1e3, 4)}
    # the HBM roof beside the ALU one: the recorded DRAM bytes of one launch
    # over its live duration (the list sweeps reuse their neighbours' records
    # from L1 and L2, so HBM is not what holds them)
    if roofline["traffic"]:
        roofline["hbm"] = hbm_roof(roofline["traffic"], b_avg)
    # the issue roof beside the ALU one: warp instructions of one launch (ncu,
    # recorded with the traffic) over its live duration, against one warp
    # instruction per scheduler per cycle (SMs x 4 x peak SM clock)
    insts = (recorded_traffic(f"sweeps_{args.workload}_f{args.precision}_{args.nbr}.md", "k_sweep_B",
                              "warp_instructions_per_launch") if f32 and not surf_in_b else None)
    if insts:
        issue_peak = roofs["issue_per_s"]
        roofline["issue"] = {"warp_instructions": insts, "achieved": round(insts / b_avg / 1e12, 4),
                             "peak": round(issue_peak / 1e12, 4), "unit": "T warp-instructions/s",
                             "frac": round(insts / b_avg / issue_peak, 4)}
    # the L1 throughput of the same launch (ncu, recorded with the traffic):
    # the list sweeps' gathers are what holds them
    l1 = (recorded_traffic(f"sweeps_{args.workload}_f{args.precision}_{args.nbr}.md", "k_sweep_B",
                           "l1tex_throughput_permille") if f32 and not surf_in_b else None)
    if l1:
        roofline["l1"] = {"throughput_frac": l1 / 1000.0,
                          "metric": "l1tex__throughput.avg.pct_of_peak_sustained_active (ncu)"}
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
# acoustic substeps per advection step of each workload, as the GPU measures
# them over the bench's timed steps (the 3D drop: the default 20 after the
# default 3 warm-up steps; the 2D static drop: 20 after 5; the impact: 5
# after 3): the reference arm rates the oracle at this many substeps per
# advection step, since it cannot afford whole advection steps of the full
# case
SUBSTEPS_PER_STEP = {"oscillating_3d": 36.25, "laplace_2d": 31.45, "impact_3d": 3.0}


_ALL_THREADS = []


def oracle_time(spec, substeps: int, threads: int = 0):
    """Seconds the oracle as it stands takes for one advection step's set-up
    (neighbour search, correction matrix, viscous force, transport shift)
    plus `substeps` acoustic substeps of the full workload; (seconds,
    substeps run, threads used).  threads = 0: all host threads (the OpenMP
    default seen at the first call; a thread count set for one run stays
    set in the process, so it is always passed explicitly)."""
    import oracle

    if not _ALL_THREADS:
        _ALL_THREADS.append(oracle.max_threads())
    threads = threads or _ALL_THREADS[0]
    pos, vel, rho, kind = spec.flat()
    P = oracle.params_for_case(spec, max_substeps=substeps, n_threads=threads)
    t0 = time.perf_counter()
    _, _, _, info, _, _ = oracle.run(P, pos, vel, rho, kind, 1)
    return time.perf_counter() - t0, info["n_sub"], threads


def oracle_split(spec, k: int = SAMPLE_SUBSTEPS):
    """The oracle's set-up and per-substep costs, from one run with one
    substep and one with k: per substep = (t_k - t_1) / (k - 1), set-up =
    t_1 - per substep."""
    t1, n1, threads = oracle_time(spec, 1)
    tk, nk, _ = oracle_time(spec, k)
    per_sub = max(tk - t1, 0.0) / max(nk - n1, 1)
    return {"setup_s": max(t1 - per_sub, 0.0), "substep_s": per_sub, "threads": threads,
            "seconds": t1 + tk, "runs": f"set-up + {n1} and set-up + {nk} substeps"}


def oracle_rate(spec, split, substeps_per_step: float) -> float:
    """particle-substeps/s of whole advection steps of `substeps_per_step`
    substeps, from the measured set-up and per-substep costs."""
    return spec.n_fluid * substeps_per_step / (split["setup_s"] + substeps_per_step * split["substep_s"])


def cpu_baseline(spec, substeps_per_step: float, one_thread: bool = True):
    """The oracle on the host cores, rated at the GPU's own substeps per
    advection step; with one_thread, also set-up + 1 substep on one thread
    (the all-core rate divided by the measured speed-up of that run)."""
    sp = oracle_split(spec)
    rate = oracle_rate(spec, sp, substeps_per_step)
    out = {"value": round(rate, 1), "unit": METRIC, "cores": sp["threads"], "kind": "oracle",
           "setup_s": round(sp["setup_s"], 3), "substep_s": round(sp["substep_s"], 4),
           "substeps_per_step": substeps_per_step,
           "sample": (f"full {spec.name} ({spec.n} particles): {sp['runs']} of the FP64 oracle "
                      f"({sp['seconds']:.1f} s); rated as whole advection steps of {substeps_per_step} "
                      f"substeps = set-up + that many substeps")}
    if one_thread:
        t1, _, _ = oracle_time(spec, 1, threads=1)
        speedup = t1 / (sp["setup_s"] + sp["substep_s"])
        out["one_thread"] = {"value": round(rate / speedup, 1), "setup_plus_1_substep_s": round(t1, 2),
                             "speedup_all_cores": round(speedup, 2),
                             "method": "set-up + 1 substep timed on 1 thread; the all-core rate divided by "
                                       "that run's speed-up"}
    return out


def run_reference(args, dist: Dist):
    """The oracle, timed as it stands: every timed step runs set-up + 1
    substep and set-up + SAMPLE_SUBSTEPS substeps, and the value rates the
    summed set-up and per-substep costs at the workload's substeps per
    advection step."""
    if dist.rank != 0:
        return None
    spec = workload(args.workload)
    for _ in range(args.warmup):
        oracle_time(spec, 1)
    setup = sub = secs = 0.0
    threads = 0
    for _ in range(args.steps):
        sp = oracle_split(spec)
        setup += sp["setup_s"]
        sub += sp["substep_s"]
        secs += sp["seconds"]
        threads = sp["threads"]
    n = max(args.steps, 1)
    split = {"setup_s": setup / n, "substep_s": sub / n}
    S_sub = SUBSTEPS_PER_STEP.get(args.workload, float(SAMPLE_SUBSTEPS))
    value = oracle_rate(spec, split, S_sub)
    return {"value": value, "ms_per_step": (split["setup_s"] + S_sub * split["substep_s"]) * 1e3,
            "threads": threads, "substeps_per_step": S_sub, "measured_s": secs,
            "setup_s": split["setup_s"], "substep_s": split["substep_s"],
            "sample": f"full {args.workload} ({spec.n} particles): per timed step set-up + 1 and set-up + "
                      f"{SAMPLE_SUBSTEPS} acoustic substeps of the FP64 oracle; value and ms_per_step rate "
                      f"whole advection steps of {S_sub} substeps (set-up + {S_sub} x per-substep cost)"}


# ------------------------------------------------------ batched and served
def batch_measure(precision: int = 32, n_cases: int = 512, steps: int = 20, warmup: int = 3,
                  plain_sample: int = 32, cpu: bool = True, cpu_cases: int = 16, block: int = BATCH_BLOCK):
    """The batched workload: independent 2D/3D droplet cases advanced
    together in one engine (one graph per advection step), against the same
    cases stepped one at a time through the single-case path.  Each case's
    arithmetic is the same alone and in the batch (bitwise, tested), so the
    two paths reach every observable with the same error.  Host-timed
    around each synchronising step call."""
    import torch

    import paper_2503_16082_gb300 as S

    torch.cuda.set_device(0)
    specs = sphcases.batch_cases(n_cases)
    cases = [sp.build() for sp in specs]
    # coarse 3D drops with strong tension cluster beyond the default list
    # capacity of 128 neighbours; the batch uses 192
    kw = [dict(max_neighbors=192 if c.dim == 3 else 0) for c in cases]
    kw_batch = [dict(k, **({"block": block} if block else {})) for k in kw]
    state_bytes = sum(S.footprint_bytes(S.params_from_spec(c, precision, **k), c.n) for c, k in zip(cases, kw_batch))

    def run(work_lists: int):
        hs = [S.case_from_spec(c, precision=precision, work_lists=work_lists, **k) for c, k in zip(cases, kw_batch)]
        b = S.batch_create(precision)
        for h in hs:
            S.batch_add(b, h)
        S.batch_step(b, warmup)
        sub0 = [S.case_info(h)["n_sub"] for h in hs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.batch_step(b, steps)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        subs = [S.case_info(h)["n_sub"] - s0 for h, s0 in zip(hs, sub0)]
        stats = [S.case_info(h)["status"] for h in hs]
        for h in hs:
            S.batch_remove(b, h)
            S.destroy(h)
        S.batch_destroy(b)
        return secs, subs, stats

    # the default launch (one block per tile of every member each substep)
    # and the work-list variant (the active members' tiles listed each
    # substep, the sweeps' blocks striding over the list)
    dt, subs, statuses = run(0)
    units = sum(c.n_fluid * n for c, n in zip(cases, subs))
    dt_w, subs_w, _ = run(1)
    units_w = sum(c.n_fluid * n for c, n in zip(cases, subs_w))
    # the single-case path on a sample of the same cases
    k = min(plain_sample, len(cases))
    punits, psecs = 0, 0.0
    for c, kk in zip(cases[:k], kw[:k]):
        h = S.case_from_spec(c, precision=precision, **kk)
        S.step(h, warmup)
        s0 = S.case_info(h)["n_sub"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.step(h, steps)
        torch.cuda.synchronize()
        psecs += time.perf_counter() - t0
        punits += c.n_fluid * (S.case_info(h)["n_sub"] - s0)
        S.destroy(h)
    # the oracle as it stands on the first cases: set-up and per-substep
    # costs measured per case, rated at that case's substeps per advection
    # step on the GPU (about 10 s of host time)
    cpu_line = None
    if cpu:
        cu = cs = spent = 0.0
        used, threads = 0, 0
        for c, n, x in zip(cases, subs, statuses):
            if x or n == 0:
                continue
            sp = oracle_split(c)
            per_step = n / steps
            cu += c.n_fluid * per_step
            cs += sp["setup_s"] + per_step * sp["substep_s"]
            spent += sp["seconds"]
            threads = sp["threads"]
            used += 1
            if spent > 10.0 or used >= cpu_cases:
                break
        cpu_line = {"value": round(cu / cs, 1) if cs > 0 else None, "unit": METRIC, "cores": threads,
                    "kind": "oracle",
                    "sample": f"the batch's first {used} healthy cases: set-up + 1 and set-up + {SAMPLE_SUBSTEPS} "
                              f"substeps of the FP64 oracle each ({spent:.1f} s), rated at each case's substeps "
                              f"per advection step on the GPU"}
    return {"metric": METRIC, "value": round(units / dt, 1), "unit": METRIC,
            "cases": len(cases), "particles": int(sum(c.n for c in cases)),
            "fluid_particles": int(sum(c.n_fluid for c in cases)), "steps": steps,
            "warmup": warmup, "seconds": round(dt, 3), "failed_cases": int(sum(1 for x in statuses if x)),
            "failed_status": {str(x): int(sum(1 for y in statuses if y == x)) for x in set(statuses) if x},
            "failed_specs": [dict(index=sp.index, dim=sp.dim, n=c.n, sigma=round(sp.sigma, 3), shape=sp.shape,
                                  status=x) for sp, c, x in zip(specs, cases, statuses) if x][:8],
            "plain_single_case": {"value": round(punits / psecs, 1), "cases_sampled": k},
            "speedup_vs_plain": round((units / dt) / (punits / psecs), 2),
            "work_list_variant": {"value": round(units_w / dt_w, 1), "seconds": round(dt_w, 3),
                                  "note": "the active members' tiles listed each substep and the sweeps' blocks "
                                          "striding over the list (work_lists = 1); same results bit for bit"},
            "same_results_as_plain": "bitwise per case (tested), so equal Laplace-pressure error",
            "cpu_baseline": cpu_line, "timing": "host clock around synchronising step calls",
            "dtype": "f32" if precision == 32 else "f64", "data": "synthetic",
            "config": {"workload": f"batch_cases seed {sphcases.BATCH_SEED}", "step": "one advection step of every case",
                       "block": block or 128, "plain_block": 128,
                       "l2": f"inputs larger than L2 ({state_bytes / 1e9:.1f} GB of case state vs 129 MB L2)"}}


def run_batch(args):
    line = batch_measure(args.precision, args.cases, args.steps, args.warmup, args.plain_sample,
                         cpu=not args.no_cpu_baseline, block=args.block or BATCH_BLOCK)
    line["mode"] = "batch"
    print(json.dumps(line), flush=True)


def serve_measure(precision: int = 32, requests: int = 200, rate: float = 50.0, n_hi: float = 2e6,
                  substeps: int = 128, capacity_cases: int = 24, budget_gb: float = 150.0):
    """The served workload: Poisson arrivals of droplet cases into the
    continuous-batching server; p50/p99 time from submission to result."""
    import torch

    import paper_2503_16082_gb300 as S
    from paper_2503_16082_gb300 import serve

    torch.cuda.set_device(0)
    specs = sphcases.served_stream(requests, rate=rate, n_hi=n_hi)
    cases = [sp.build() for sp in specs]
    # capacity first: a batch of the stream's first cases, one advection step
    # each after a warm-up step; the offered load (arrival rate x mean fluid
    # particles x substeps per request) must stay below 0.9 of it, else the
    # substep count per request is lowered
    probe = cases[:min(len(cases), capacity_cases)]
    b = S.batch_create(precision)
    hs = [S.case_from_spec(c, precision=precision) for c in probe]
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
    n_sub = substeps
    while n_sub > 1 and rate * mean_fluid * n_sub > 0.9 * capacity:
        n_sub -= 1
    offered = rate * mean_fluid * n_sub
    srv = serve.Server(precision=precision, budget_bytes=budget_gb * 1e9)
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
    return {"metric": METRIC, "value": round(st["particle_substeps"] / wall, 1),
            "unit": METRIC, "requests": len(res), "arrival_rate_per_s": rate,
            "p50_latency_s": round(float(np.percentile(lat, 50)), 4),
            "p99_latency_s": round(float(np.percentile(lat, 99)), 4),
            "gpu_busy_fraction": round(st["busy_s"] / wall, 3), "rounds": st["rounds"],
            "failed": int(sum(1 for r in res if r.info["status"])),
            "substeps_per_request": n_sub, "substeps_requested": substeps,
            "capacity": round(capacity, 1), "offered_load": round(offered, 1),
            "offered_fraction": round(offered / capacity, 3), "budget_gb": budget_gb,
            "particles_per_request_range": [5e3, n_hi],
            "dtype": "f32" if precision == 32 else "f64", "data": "synthetic",
            "config": {"workload": f"served_stream seed {sphcases.SERVE_SEED}", "wall_s": round(wall, 2)}}


def run_serve(args):
    line = serve_measure(args.precision, args.requests, args.rate, args.serve_n_hi, args.serve_substeps,
                         args.capacity_cases, args.budget_gb)
    line["mode"] = "serve"
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
    ap.add_argument("--batch-steps", type=int, default=5,
                    help="timed advection steps of the batch object in the default line")
    ap.add_argument("--no-batch", action="store_true", help="leave the batch object out of the default line")
    ap.add_argument("--no-serve", action="store_true", help="leave the serve object out of the default line")
    ap.add_argument("--no-one-thread", action="store_true", help="skip the one-thread oracle run")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if not args.block and not args.lanes:
        args.block = TUNED_BLOCK.get((args.workload, args.precision, args.nbr), 0)
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
                      l2="not applicable: the oracle runs on the host cores",
                      substeps_per_step=res["substeps_per_step"])
        line = {"impl": "reference", "metric": METRIC, "value": round(res["value"], 1),
                "unit": METRIC, "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(res["ms_per_step"], 1), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": config,
                "cpu_baseline": {"value": round(res["value"], 1), "unit": METRIC, "cores": res["threads"],
                                 "kind": "oracle", "sample": res["sample"],
                                 "setup_s": round(res["setup_s"], 3), "substep_s": round(res["substep_s"], 4),
                                 "measured_s": round(res["measured_s"], 1)},
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
        cpu = cpu_baseline(workload(args.workload), round(res["n_sub"] / args.steps, 2),
                           one_thread=not args.no_one_thread)
    # the batched and served workloads on the same GPU, bounded in time
    extra = {}
    if rank == 0 and ws <= 1 and args.precision == 32 and args.workload == "oscillating_3d":
        if not args.no_batch:
            extra["batch"] = batch_measure(32, args.cases, args.batch_steps, 3, args.plain_sample,
                                           cpu=not args.no_cpu_baseline)
        if not args.no_serve:
            extra["serve"] = serve_measure(32, args.requests, args.rate, args.serve_n_hi, args.serve_substeps,
                                           args.capacity_cases, args.budget_gb)
    dist.close()
    if rank != 0:
        return
    line = {"metric": METRIC, "value": round(res["value"], 1), "unit": METRIC, "n_gpus": max(ws, 1),
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(res["ms_per_step"], 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic", "config": config, "roofline": res["roofline"],
            "cpu_baseline": cpu, "e2e": res["e2e"], "gpu_launches": res["gpu_launches"],
            "clocks": res["clocks"], "kernel_ms_one_step": res["kernel_ms"]}
    line.update(extra)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
