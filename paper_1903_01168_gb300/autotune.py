"""Measured choice of the fused kernel's tile height per lattice size class.

The fused kernel works on strips 128 columns wide; the planner cuts the rows of
every strip into segments, and a thread block marches down its segments.  A
segment re-reads a 4-row halo, so short segments waste bandwidth, while long
ones leave streaming multiprocessors idle on small lattices.  Very small
lattices may even run faster on the node-parallel two-pass kernel.  The shortest
segment a lattice may be cut into (`plan_rows`) and the kernel are therefore
chosen per size class by timing, not by rule: every candidate runs a few steps on
the device, timed with CUDA events on the stream it runs on, and the fastest
wins.

A size class is (storage type, collision, equilibrium, nx and ny rounded up to
powers of two).  Tuning a single lattice times it alone; tuning for a batch
times the members of each class together as a small batch, so the choice is the
one that pays inside a batched launch.  A whole batch also gets its planner's
row cost model tuned (`tune_row_overhead`): how much of a full strip row a
narrow strip's row costs, which decides how many rows each block receives.

The plan never changes what a node computes, so every candidate gives
bit-identical results; only the time differs.
"""
from __future__ import annotations

import json
import math
import os

from . import lbm as L

PLAN_CANDIDATES = (8, 16, 32, 64)
ROW_OVERHEAD_CANDIDATES = (0.0, 0.5, 1.0, 2.0, 4.0)
CLASS_SAMPLE = 4          # members of a class timed together when tuning a batch


def _pow2(n: int) -> int:
    return 1 << max(0, int(math.ceil(math.log2(max(1, n)))))


def size_class(nx: int, ny: int, storage: int = 0, collision: int = 0, equilibrium: int = 0) -> str:
    return f"s{storage}-c{collision}-e{equilibrium}-x{_pow2(nx)}-y{_pow2(ny)}"


def class_of(nx: int, ny: int, params: dict) -> str:
    return size_class(nx, ny, params.get("storage", 0), params.get("collision", 0), params.get("equilibrium", 0))


def _event_ms(run, steps: int) -> float:
    """Mean milliseconds of run(steps) on torch's current stream (after a warm-up)."""
    import torch
    run(max(2, steps // 4))
    torch.cuda.current_stream().synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    run(steps)
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def _start(nx, ny, params, choice):
    """A lattice of this size with a static bubble, on torch's current stream."""
    kw = dict(params)
    kw.update(choice)
    s = L.Simulation(nx, ny, torch_memory=True, **kw)
    s.init_bubble(nx / 2.0, ny / 2.0, max(2.0, min(nx, ny) / 5.0))
    return s


class Autotuner:
    """Table of size class -> {"kernel", "plan_rows", "ms", "timings"}, optionally
    kept in a JSON file so that tuning runs once per device and build."""

    def __init__(self, cache_path: str | None = None, steps: int = 30,
                 candidates=PLAN_CANDIDATES, try_twopass: bool = True):
        self.cache_path = cache_path
        self.steps = int(steps)
        self.candidates = tuple(candidates)
        self.try_twopass = try_twopass
        self.table: dict[str, dict] = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.table = json.load(f)

    def save(self):
        if not self.cache_path:
            return
        tmp = self.cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.table, f, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)

    def _choices(self, batched: bool):
        out = [dict(kernel=L.LBM_KERNEL_FUSED, plan_rows=r) for r in self.candidates]
        if self.try_twopass and not batched:
            out.append(dict(kernel=L.LBM_KERNEL_TWOPASS, plan_rows=0))
        return out

    def _record(self, key, timings):
        ms, best = min(timings, key=lambda x: x[0])
        self.table[key] = dict(best, ms=ms, timings={f"{'fused' if c['kernel'] == L.LBM_KERNEL_FUSED else 'twopass'}"
                                                     f"/{c['plan_rows']}": t for t, c in timings})
        return self.table[key]

    def tune_single(self, nx: int, ny: int, **params) -> dict:
        """Fastest (kernel, plan_rows) for one lattice of this size class run alone."""
        key = "single-" + class_of(nx, ny, params)
        if key not in self.table:
            timings = []
            for c in self._choices(batched=False):
                s = _start(nx, ny, params, c)
                try:
                    timings.append((_event_ms(s.step, self.steps), c))
                finally:
                    s.close()
            self._record(key, timings)
        return self.table[key]

    def tune_batch(self, members) -> dict:
        """members: list of (nx, ny, params) that will run as one batch.  For each
        size class among them, time up to CLASS_SAMPLE of its members together as
        a batch under every candidate plan_rows; returns {class: choice}."""
        by_class: dict[str, list] = {}
        for nx, ny, params in members:
            by_class.setdefault("batch-" + class_of(nx, ny, params), []).append((nx, ny, params))
        for key, group in by_class.items():
            if key in self.table:
                continue
            sample = group[:CLASS_SAMPLE]
            timings = []
            for c in self._choices(batched=True):
                sims = [_start(nx, ny, params, c) for nx, ny, params in sample]
                try:
                    b = L.Batch(sims)
                    try:
                        timings.append((_event_ms(lambda n: b.step(n, use_graph=False), self.steps), c))
                    finally:
                        b.close()
                finally:
                    for s in sims:
                        s.close()
            self._record(key, timings)
        return {k: self.table[k] for k in by_class}

    def params_for(self, nx: int, ny: int, batched: bool, **params) -> dict:
        """`params` with the tuned kernel and plan_rows of this size class (the
        batch table when batched), unchanged if the class was never tuned."""
        key = ("batch-" if batched else "single-") + class_of(nx, ny, params)
        out = dict(params)
        c = self.table.get(key)
        if c is not None:
            out["plan_rows"] = int(c["plan_rows"])
            if not batched:
                out["kernel"] = int(c["kernel"])
        return out


def tune_row_overhead(sims, candidates=ROW_OVERHEAD_CANDIDATES, steps: int = 20) -> tuple[float, dict]:
    """Planner cost of a strip row beyond its busy warps, timed on the batch itself.

    The balanced plan shares the strip rows of all members among the resident
    blocks by cost; how much a narrow strip's row costs relative to a full one
    depends on the mix of lattice widths, so each candidate is timed on the
    whole batch (direct launches on torch's current stream).  The members'
    states advance by (steps + warm-up) x len(candidates) steps: re-initialise
    them afterwards.  Returns (best, {candidate: ms per step})."""
    timings = {}
    for c in candidates:
        b = L.Batch(sims, row_overhead=float(c))
        try:
            timings[float(c)] = _event_ms(lambda n: b.step(n, use_graph=False), steps)
        finally:
            b.close()
    best = min(timings, key=timings.get)
    return best, timings
