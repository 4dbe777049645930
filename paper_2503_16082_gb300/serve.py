"""Continuous-batching server for droplet and bubble solves.

Requests (a case description plus a stopping rule) arrive at any time.  One
scheduling round:

1. retires members that reached their stopping rule (their fields are read
   back, the case leaves the batch and is released);
2. admits queued requests, first come first served, while their device
   footprint (``sphst_footprint_bytes``) fits the memory budget next to the
   resident members and the engine's particle limit holds;
3. advances every member by one advection step with one ``sphst_batch_step``
   (all members share one launch sequence; each keeps its own time steps).

Membership changes take effect at the next batch step; particle state stays
on the device between rounds.  Latency is measured from submission to the
round that retired the request.  Everything numerical runs in the CUDA
library; this module only schedules.
"""
from __future__ import annotations

import collections
import concurrent.futures
import dataclasses
import threading
import time
from typing import Deque, Dict, List, Optional, Sequence

import numpy as np

from . import (FIELD_POS, FIELD_RHO, FIELD_VEL, MAX_LIST_ENGINE_PARTICLES, OK, SphstError, batch_add, batch_create,
               batch_destroy, batch_remove, batch_step, case_from_spec, case_info, default_params,
               destroy, footprint_bytes, read_fields)


@dataclasses.dataclass
class Result:
    """What a retired request returns."""

    fields: Dict[int, np.ndarray]
    info: dict
    submitted: float
    admitted: float
    finished: float

    @property
    def latency(self) -> float:
        return self.finished - self.submitted

    @property
    def queued(self) -> float:
        return self.admitted - self.submitted


@dataclasses.dataclass
class _Request:
    rid: int
    spec: object
    n_adv: Optional[int]
    t_end: Optional[float]
    n_sub: Optional[int]
    params: dict
    submitted: float
    future: concurrent.futures.Future
    footprint: int = 0
    handle: object = None
    admitted: float = 0.0
    done_steps: int = 0


class Server:
    """Admission by device-memory budget and particle count, one shared
    batch, FIFO queue.  An error in the background loop fails every queued
    and resident request with it and stops the loop."""

    def __init__(self, precision: int = 32, budget_bytes: float = 150e9,
                 fields: Sequence[int] = (FIELD_POS, FIELD_VEL, FIELD_RHO),
                 max_members: int = 4096, max_particles: int = MAX_LIST_ENGINE_PARTICLES):
        self.precision = precision
        self.budget = float(budget_bytes)
        self.max_particles = int(max_particles)
        self.resident_particles = 0
        self.error: Optional[BaseException] = None
        self.fields = tuple(fields)
        self.max_members = max_members
        self.batch = batch_create(precision)
        self.queue: Deque[_Request] = collections.deque()
        self.members: List[_Request] = []
        self.resident_bytes = 0
        self.lock = threading.Lock()
        self.next_id = 0
        self.particle_substeps = 0
        self.busy_seconds = 0.0
        self.rounds = 0
        self.results: List[Result] = []
        self._thread = None
        self._stop = threading.Event()

    # ------------------------------------------------------------ requests
    def footprint(self, spec, params: Optional[dict] = None) -> int:
        p = default_params(dim=spec.dim, precision=self.precision, dx=spec.dx)
        for k, v in (params or {}).items():
            setattr(p, k, v)
        return footprint_bytes(p, spec.n)

    def submit(self, spec, n_adv: Optional[int] = None, t_end: Optional[float] = None,
               n_sub: Optional[int] = None, **params) -> concurrent.futures.Future:
        """Queue a solve; it stops after n_adv advection steps, or at the first
        advection-step boundary with t >= t_end, or with at least n_sub
        acoustic substeps done (whichever rule is given first)."""
        if n_adv is None and t_end is None and n_sub is None:
            raise ValueError("give n_adv, t_end or n_sub")
        fut: concurrent.futures.Future = concurrent.futures.Future()
        with self.lock:
            r = _Request(self.next_id, spec, n_adv, t_end, n_sub, params, time.perf_counter(), fut)
            r.footprint = self.footprint(spec, params)
            if r.footprint > self.budget:
                fut.set_exception(SphstError(-8, f"request needs {r.footprint} B, budget {self.budget:.0f} B"))
                return fut
            if spec.n > self.max_particles:
                fut.set_exception(SphstError(-1, f"request has {spec.n} particles, an engine holds "
                                                 f"{self.max_particles}"))
                return fut
            if self.error is not None:
                fut.set_exception(self.error)
                return fut
            self.next_id += 1
            self.queue.append(r)
        return fut

    # ------------------------------------------------------------- rounds
    def _finished(self, r: _Request, info: dict) -> bool:
        if info["status"] != OK:
            return True
        if r.n_adv is not None and r.done_steps >= r.n_adv:
            return True
        if r.n_sub is not None and info["n_sub"] >= r.n_sub:
            return True
        return r.t_end is not None and info["t"] >= r.t_end

    def _retire(self, now: float) -> None:
        keep = []
        for r in self.members:
            info = case_info(r.handle)
            if not self._finished(r, info):
                keep.append(r)
                continue
            fields = {f: read_fields(r.handle, f, r.spec.dim) for f in self.fields}
            batch_remove(self.batch, r.handle)
            destroy(r.handle)
            self.resident_bytes -= r.footprint
            self.resident_particles -= r.spec.n
            res = Result(fields, info, r.submitted, r.admitted, now)
            self.results.append(res)
            r.future.set_result(res)
        self.members = keep

    def _admit(self, now: float) -> int:
        admitted = 0
        with self.lock:
            while (self.queue and len(self.members) < self.max_members
                   and self.resident_bytes + self.queue[0].footprint <= self.budget
                   and self.resident_particles + self.queue[0].spec.n <= self.max_particles):
                r = self.queue.popleft()
                try:
                    r.handle = case_from_spec(r.spec, precision=self.precision, **r.params)
                    batch_add(self.batch, r.handle)
                except Exception as e:          # noqa: BLE001 - report to the caller
                    r.future.set_exception(e)
                    continue
                r.admitted = now
                self.resident_bytes += r.footprint
                self.resident_particles += r.spec.n
                self.members.append(r)
                admitted += 1
        return admitted

    def step(self) -> int:
        """One scheduling round; returns the number of members stepped."""
        now = time.perf_counter()
        self._retire(now)
        self._admit(now)
        if not self.members:
            return 0
        before = {r.rid: case_info(r.handle)["n_sub"] for r in self.members}
        t0 = time.perf_counter()
        batch_step(self.batch, 1)
        self.busy_seconds += time.perf_counter() - t0
        self.rounds += 1
        for r in self.members:
            r.done_steps += 1
            self.particle_substeps += r.spec.n_fluid * (case_info(r.handle)["n_sub"] - before[r.rid])
        return len(self.members)

    def idle(self) -> bool:
        with self.lock:
            return not self.queue and not self.members

    def run_until_idle(self, timeout: Optional[float] = None) -> None:
        t0 = time.perf_counter()
        while not self.idle():
            if self.step() == 0:
                self._retire(time.perf_counter())
            if timeout is not None and time.perf_counter() - t0 > timeout:
                raise TimeoutError("server did not drain")
        self._retire(time.perf_counter())

    # ------------------------------------------------------- background loop
    def start(self) -> None:
        def loop():
            try:
                while not self._stop.is_set():
                    if self.step() == 0:
                        self._retire(time.perf_counter())
                        time.sleep(0.0005)
            except BaseException as e:      # noqa: BLE001 - handed to every waiting caller
                self.fail_all(e)
        self._thread = threading.Thread(target=loop, daemon=True)
        self._thread.start()

    def fail_all(self, e: BaseException) -> None:
        """Record `e` and fail every queued and resident request with it."""
        with self.lock:
            self.error = e
            pending = list(self.queue) + list(self.members)
            self.queue.clear()
        for r in pending:
            if not r.future.done():
                r.future.set_exception(e)

    def stop(self) -> None:
        self._stop.set()
        if self._thread:
            self._thread.join()
        self._thread = None

    def close(self) -> None:
        self.stop()
        for r in self.members:
            batch_remove(self.batch, r.handle)
            destroy(r.handle)
        self.members = []
        batch_destroy(self.batch)

    # ---------------------------------------------------------- statistics
    def stats(self) -> dict:
        lat = np.array([r.latency for r in self.results]) if self.results else np.zeros(1)
        return {"completed": len(self.results),
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "particle_substeps": int(self.particle_substeps),
                "busy_s": self.busy_seconds, "rounds": self.rounds}
