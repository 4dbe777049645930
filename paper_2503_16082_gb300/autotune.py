"""Launch-configuration autotuner for the pair sweeps.

Three choices change only speed, never the physics:

* ``block``: particles per tile = threads per block of every sweep (a multiple
  of 32 in 32..256; the sweeps are compiled for at most 256 threads per
  block).  Each particle's sums do not depend on it.
* ``nbr_mode``: neighbour list built once per advection step, or the cell walk
  every sweep.  The two visit the same pairs; the list orders other-phase
  neighbours first, so results agree to the rounding of a reordered sum.
* ``lanes``: lanes per particle in the per-substep sweeps with the list (1, 2,
  4 or 8, i.e. 32, 16, 8 or 4 particles per warp).  The lanes split the list and
  add their partial sums in a fixed order (the results differ from one lane by
  the rounding of the reordered sum, within the parity tolerances).
  More lanes put a small case on more SMs and more warps.

``Tuner.best(spec)`` times every candidate on the case itself (one advection
step to set up and warm, then ``adv`` timed steps), keeps the fastest in
particle-substeps per second, and caches it under a key of dimension,
precision and size bucket (floor of log2 of the particle count), so cases of
similar size reuse the answer.  The table is a JSON file when a path is given.
Timing goes through the library's own step; nothing here computes physics.
"""
from __future__ import annotations

import json
import math
import os
import time
from typing import Callable, Dict, Iterable, Optional, Sequence, Tuple

BLOCKS = (32, 64, 128, 256)
LANES = (1, 2, 4, 8)


def bucket_key(dim: int, precision: int, n: int) -> str:
    """Cache key: dimension, precision and log2 size bucket."""
    return f"d{dim}-p{precision}-n{int(math.log2(max(int(n), 1)))}"


class Tuner:
    def __init__(self, path: Optional[str] = None, blocks: Sequence[int] = BLOCKS,
                 nbr_modes: Optional[Sequence[int]] = None, adv: int = 2,
                 measure: Optional[Callable[..., float]] = None, lanes: Sequence[int] = LANES):
        from . import NBR_CELLS, NBR_LIST
        self.path = path
        self.blocks = tuple(blocks)
        self.lanes = tuple(lanes)
        self._list = NBR_LIST
        self.nbr_modes = tuple(nbr_modes) if nbr_modes is not None else (NBR_LIST, NBR_CELLS)
        self.adv = adv
        self.measure = measure or self._measure
        self.table: Dict[str, dict] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.table = json.load(f)

    def candidates(self) -> Iterable[Tuple[int, int, int]]:
        """(block, nbr_mode, lanes); lanes > 1 only with the list and at
        least 16 particles per block."""
        for m in self.nbr_modes:
            for b in self.blocks:
                for L in (self.lanes if m == self._list else (1,)):
                    if L == 1 or b // L >= 16:
                        yield b, m, L

    def _measure(self, spec, precision: int, block: int, nbr_mode: int, lanes: int = 1) -> float:
        """Particle-substeps per second of `adv` advection steps after one
        warm-up step (engine set-up and graph capture excluded)."""
        from . import case_from_spec, case_info, destroy, step
        h = case_from_spec(spec, precision=precision, block=block, nbr_mode=nbr_mode, lanes=lanes)
        try:
            step(h, 1)
            s0 = case_info(h)["n_sub"]
            t0 = time.perf_counter()
            step(h, self.adv)
            dt = time.perf_counter() - t0
            subs = case_info(h)["n_sub"] - s0
        finally:
            destroy(h)
        return spec.n_fluid * subs / max(dt, 1e-9)

    def tune(self, spec, precision: int = 32) -> dict:
        results = []
        for block, mode, lanes in self.candidates():
            rate = self.measure(spec, precision, block, mode, lanes)
            results.append({"block": block, "nbr_mode": mode, "lanes": lanes, "rate": rate})
        best = max(results, key=lambda r: r["rate"])
        entry = {"block": best["block"], "nbr_mode": best["nbr_mode"], "lanes": best["lanes"],
                 "rate": best["rate"], "tried": results, "n": int(spec.n)}
        self.table[bucket_key(spec.dim, precision, spec.n)] = entry
        self.save()
        return entry

    def best(self, spec, precision: int = 32) -> dict:
        """{'block': b, 'nbr_mode': m, 'lanes': L} for this case, tuning on a
        cache miss."""
        e = self.table.get(bucket_key(spec.dim, precision, spec.n))
        if e is None:
            e = self.tune(spec, precision)
        return {"block": int(e["block"]), "nbr_mode": int(e["nbr_mode"]), "lanes": int(e.get("lanes", 1))}

    def save(self) -> None:
        if not self.path:
            return
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.table, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)
