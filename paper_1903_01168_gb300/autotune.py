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
times the whole batch while the plan_rows of one class at a time varies, so the
choice is the one that pays inside that batched launch.  A whole batch also gets
its work plan
tuned (`tune_plan`): one segment per block (split) or equal shares of row cost
over several segments per block (balanced), each with a row cost model (how
much of a full strip row a narrow strip's row costs).

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
# (plan kind, row overhead) pairs timed on a whole batch
PLAN_OPTION_CANDIDATES = tuple((L.LBM_PLAN_SPLIT, o) for o in (0.0, 1.0, 4.0)) + \
    tuple((L.LBM_PLAN_BALANCED, o) for o in ROW_OVERHEAD_CANDIDATES)


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

    def tune_batch(self, sims, steps: int = 20, gain: float = 0.02) -> dict:
        """Per size class plan_rows and the plan options of one batch, timed on
        the batch itself (the members of a class alone would neither fill the GPU
        nor share it as they do in the batch).

        Coordinate descent: start from the default plan for every member; for
        each size class (largest share of nodes first) try every candidate
        plan_rows for that class's members with the others fixed, and keep one
        that is at least `gain` faster.  Then time the plan kinds and row costs
        (`tune_plan`) with the chosen plan_rows.  The members' states advance:
        re-initialise them afterwards.  Returns {"classes": {class: plan_rows},
        "member_plan_rows": [...], "plan": kind, "row_overhead": r, "ms": t}; the
        class table is also stored under "batch-<class>" keys."""
        keys = [class_of(s.nx, s.ny, {"storage": s.params.storage, "collision": s.params.collision,
                                      "equilibrium": s.params.equilibrium}) for s in sims]
        rows = [0] * len(sims)

        def timed(member_rows, kind=L.LBM_PLAN_AUTO, ovh=None):
            b = L.Batch(sims, row_overhead=ovh, plan=kind, member_plan_rows=member_rows)
            try:
                return _event_ms(lambda n: b.step(n, use_graph=False), steps)
            finally:
                b.close()

        best = timed(rows)
        weight = {}
        for s, k in zip(sims, keys):
            weight[k] = weight.get(k, 0) + s.nx * s.ny
        chosen = {}
        for k in sorted(weight, key=weight.get, reverse=True):
            pick = 0
            for r in self.candidates:
                if r == 8:
                    continue   # the default (0 = 8) is the incumbent
                trial = [r if kk == k else v for kk, v in zip(keys, rows)]
                t = timed(trial)
                if t < best * (1.0 - gain):
                    best, pick = t, r
            rows = [pick if kk == k else v for kk, v in zip(keys, rows)]
            chosen[k] = pick if pick else 8
            self.table["batch-" + k] = {"kernel": L.LBM_KERNEL_FUSED, "plan_rows": chosen[k]}
        (kind, ovh), timings = tune_plan(sims, steps=steps, member_plan_rows=rows)
        return {"classes": chosen, "member_plan_rows": rows, "plan": kind, "row_overhead": ovh,
                "ms": timings[(kind, ovh)]}

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


def tune_plan(sims, candidates=PLAN_OPTION_CANDIDATES, steps: int = 20,
              member_plan_rows=None) -> tuple[tuple[int, float], dict]:
    """Work plan of a batch, timed on the batch itself.

    Each candidate (plan kind, row overhead) plans the strip rows of all members
    differently; which is fastest depends on the mix of lattice sizes (how many
    128-column strips there are per resident block, how narrow their last strips
    are), so each is timed on the whole batch with direct launches on torch's
    current stream.  The members' states advance by (steps + warm-up) x
    len(candidates) steps: re-initialise them afterwards.  Returns
    (best (kind, overhead), {(kind, overhead): ms per step})."""
    timings = {}
    for kind, ovh in candidates:
        b = L.Batch(sims, row_overhead=float(ovh), plan=int(kind), member_plan_rows=member_plan_rows)
        try:
            timings[(int(kind), float(ovh))] = _event_ms(lambda n: b.step(n, use_graph=False), steps)
        finally:
            b.close()
    best = min(timings, key=timings.get)
    return best, timings
