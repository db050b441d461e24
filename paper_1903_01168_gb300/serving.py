"""Continuous-batching serving loop for colour-gradient LBM simulation requests.

A request is a simulation spec (lattice, physics, boundary conditions, storage
type, number of steps) with an arrival time.  The server:

  * admits arrived requests into device memory in arrival order while the sum
    of the resident state bytes stays within an HBM budget; a request that does
    not fit waits, and later ones that fit are admitted past it (backfill).
    Admitted simulations stay resident until they are done;
  * chooses the active set among the resident simulations: in arrival order,
    while their lattice nodes stay within `max_active_nodes`, about what keeps
    every SM busy in one launch, again letting later ones that fit pass one that
    does not (the oldest always runs).  The members of a batch advance in
    lockstep, one step per launch, so a batch larger than the GPU only slows every
    member down: the cap keeps the GPU full while the oldest requests run at full
    speed, close to first come first served, and small lattices that would leave
    the GPU idle alone share it;
  * advances the active simulations together, one batched fused-kernel launch
    per time step and storage type, replaying a graph of `graph_steps` steps; each
    simulation carries its own stop step, so one that finishes inside a chunk
    simply stops there while the others go on;
  * between chunks retires the finished simulations (their diagnostics are read
    back), frees their memory, admits new arrivals and recomputes the active set,
    so new requests join work already on the device.

`run_sequential` is the baseline: the same requests one at a time through the
plain single-simulation FP32 path.  Both report the time from arrival to result
(p50 / p99) and the aggregate MLUPS over the whole trace.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import lbm as L
from .workloads import SimSpec

STORAGE_BYTES = {0: 144, 1: 104, 2: 104}


@dataclass
class Request:
    rid: int
    arrival: float
    spec: SimSpec


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    nodes: int
    steps: int                 # steps run (fewer than requested if the run failed)
    diag: dict = field(default_factory=dict)
    failed: bool = False       # the state went non-finite; the request was retired early

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def state_bytes(spec: SimSpec) -> int:
    """Device bytes a simulation of this spec keeps resident (both state buffers)."""
    p = params_of(spec)
    return L.lbm_bytes_required(spec.nx, spec.ny, p)


class Admission:
    """Admission into device memory under a byte budget (host logic only): in
    arrival order, letting later requests that fit pass one that does not."""

    def __init__(self, budget_bytes: int):
        self.budget = int(budget_bytes)
        self.resident = 0

    def fits(self, nbytes: int) -> bool:
        return self.resident + nbytes <= self.budget

    def take(self, waiting: deque, now: float, size_of) -> list:
        """Remove from `waiting` and return, in arrival order, the requests that
        have arrived by `now` and fit the budget, skipping those that do not."""
        out, keep = [], deque()
        while waiting:
            r = waiting.popleft()
            if r.arrival > now:
                keep.append(r)
                continue
            nb = size_of(r)
            if nb > self.budget:
                raise ValueError(f"request {r.rid} needs {nb} bytes, more than the whole budget")
            if self.fits(nb):
                self.resident += nb
                out.append(r)
            else:
                keep.append(r)
        waiting.extend(keep)
        return out

    def release(self, nbytes: int):
        self.resident -= int(nbytes)
        assert self.resident >= 0


def active_set(order: list, nodes_of, cap: int | None) -> list:
    """The requests (ids in priority order) that run in the next chunk: in order,
    while their nodes stay within `cap`, skipping one that would exceed it; the
    first always runs, alone if it exceeds the cap by itself."""
    act, tot = [], 0
    for rid in order:
        n = nodes_of(rid)
        if act and cap is not None and tot + n > cap:
            continue
        act.append(rid)
        tot += n
    return act


def params_of(spec: SimSpec) -> L.lbm_params:
    kw = dict(gamma=spec.gamma, tau_r=spec.tau_r, tau_b=spec.tau_b, sigma=spec.sigma, beta=spec.beta,
              gx=spec.gx, gy=spec.gy, bc_x=spec.bc_x, bc_y=spec.bc_y, storage=spec.storage,
              u_in_r=spec.u_in_r, u_in_b=spec.u_in_b, p_out=spec.p_out,
              inlet_period_r=spec.inlet_period_r, inlet_period_b=spec.inlet_period_b,
              collision=spec.collision, equilibrium=spec.equilibrium)
    return L.make_params(**kw)


def start_simulation(spec: SimSpec, storage: int | None = None) -> L.Simulation:
    """Create and initialise the simulation a request describes."""
    p = params_of(spec)
    kw = {name: getattr(p, name) for name in L.PARAM_NAMES}
    if storage is not None:
        kw["storage"] = storage
    s = L.Simulation(spec.nx, spec.ny, **kw)
    if spec.geometry == "bubble":
        s.init_bubble(*spec.bubble)
    elif spec.geometry == "slug":
        n, length, height = spec.slug
        s.init_slug(int(n), length, height, True)
    else:
        # open channel: liquid (heavy phase) at rest; the inlet injects the segments
        ones = np.full((spec.ny, spec.nx), spec.gamma)
        zeros = np.zeros((spec.ny, spec.nx))
        s.init_fields(ones, zeros, zeros, zeros)
    return s


def _stats(results: list[Result], makespan: float) -> dict:
    lat = np.array([r.latency for r in results])
    work = sum(r.nodes * r.steps for r in results)
    return {"requests": len(results), "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
            "makespan_s": makespan, "mlups": work / makespan / 1e6, "updates": work,
            "failed": sum(1 for r in results if r.failed)}


def _failed(diag: dict) -> bool:
    return diag.get("nonfinite", 0) != 0


class Server:
    """Continuous-batching server on the current CUDA device."""

    PRIORITIES = ("arrival", "remaining_steps", "remaining_work")

    def __init__(self, budget_bytes: float = 150e9, chunk: int = 500, max_chunk: int = 4000,
                 graph_steps: int = 32, max_active_nodes: int | None = 8_000_000, priority: str = "arrival",
                 plan: int = L.LBM_PLAN_BALANCED, row_overhead: float | None = 4.0,
                 clock=time.perf_counter, sleep=time.sleep):
        """plan / row_overhead: the batch work plan (LBM_PLAN_*) and the planner's
        fixed cost of a strip row in busy warps.  The active sets are uneven (lattices
        of 64 to 256 rows whose last strips are often narrow): the balanced plan with a
        row cost of 4 busy warps ran 10-20 lattice batches 19 % (FP32) to 44 % (FP16)
        faster than the split plan."""
        if priority not in self.PRIORITIES:
            raise ValueError(f"priority must be one of {self.PRIORITIES}")
        self.priority = priority
        self.plan = int(plan)
        self.row_overhead = row_overhead
        self.admission = Admission(int(budget_bytes))
        self.max_active_nodes = None if max_active_nodes is None else int(max_active_nodes)
        self.chunk = int(chunk)            # shortest chunk (bounds the wait of a new arrival)
        self.max_chunk = int(max_chunk)
        self.graph_steps = int(graph_steps)   # steps per graph replay (0: direct launches only)
        self.clock = clock
        self.sleep = sleep

    def _chunk_len(self, active, waiting, now: float) -> int:
        """Run to the next completion, but no longer than max_chunk; only `chunk`
        steps while the next request has not arrived yet (it may join when it
        does).  A request that has arrived and still waits is held back by the
        budget or the active cap, which only a completion relieves."""
        left = min(r.spec.steps - s.t for s, r, _, _ in active.values())
        n = max(1, min(left, self.max_chunk))
        if waiting and min(q.arrival for q in waiting) > now:
            n = min(n, self.chunk)
        return n

    def _rank(self, entry, rid: int):
        """Sort key of a resident request for the active set: its arrival (oldest
        first), its remaining steps (most first: members of one batch advance in
        lockstep, so a request with many steps left finishes last), or its
        remaining work in node updates (least first)."""
        s, r = entry[0], entry[1]
        if self.priority == "remaining_steps":
            return (-(r.spec.steps - s.t), r.arrival, rid)
        if self.priority == "remaining_work":
            return ((r.spec.steps - s.t) * r.spec.nx * r.spec.ny, r.arrival, rid)
        return (r.arrival, rid)

    def run(self, trace: list[tuple[float, SimSpec]]) -> tuple[list[Result], dict]:
        reqs = [Request(i, a, sp) for i, (a, sp) in enumerate(trace)]
        waiting = deque(sorted(reqs, key=lambda r: r.arrival))
        resident: dict[int, tuple] = {}        # rid -> (sim, request, admitted_at, bytes)
        results: list[Result] = []
        batch = None
        members: tuple = ()
        t0 = self.clock()
        while waiting or resident:
            now = self.clock() - t0
            for r in self.admission.take(waiting, now, lambda q: state_bytes(q.spec)):
                s = start_simulation(r.spec)
                s.set_stop(r.spec.steps)
                resident[r.rid] = (s, r, now, state_bytes(r.spec))
            if not resident:
                self.sleep(max(0.0, min(q.arrival for q in waiting) - (self.clock() - t0)))
                continue
            order = sorted(resident, key=lambda k: self._rank(resident[k], k))
            key = tuple(sorted(active_set(order, lambda k: resident[k][1].spec.nx * resident[k][1].spec.ny,
                                          self.max_active_nodes)))
            if key != members:
                if batch is not None:
                    batch.close()
                batch = L.Batch([resident[k][0] for k in key], plan=self.plan, row_overhead=self.row_overhead)
                members = key
            active = {k: resident[k] for k in key}
            pending = list(waiting) + [resident[k][1] for k in resident if k not in active]
            n = self._chunk_len(active, deque(q for q in pending if q.arrival > now), self.clock() - t0)
            g = self.graph_steps
            if g > 0 and n >= g:
                # one graph of g steps per batch, replayed; the remainder launched directly
                for _ in range(n // g):
                    batch.step(g, use_graph=True)
                n %= g
            if n:
                batch.step(n, use_graph=False)
            active[key[0]][0].synchronize()     # the batch runs on its first member's stream
            done = self.clock() - t0
            retired = []
            for k in key:
                s, r, adm, nb = active[k]
                # every member's FP64 diagnostics: a finished request returns them,
                # and one whose state went non-finite is retired at once as failed
                d = s.diagnostics(allow_unstable=True)
                if s.t >= r.spec.steps or _failed(d):
                    results.append(Result(r.rid, r.arrival, adm, done, r.spec.nx * r.spec.ny, s.t, d, _failed(d)))
                    retired.append(k)
            if retired:
                batch.close()                   # no batch may refer to a freed simulation
                batch = None
                members = ()
                for k in retired:
                    s, r, adm, nb = resident.pop(k)
                    s.close()
                    self.admission.release(nb)
        if batch is not None:
            batch.close()
        makespan = self.clock() - t0
        results.sort(key=lambda r: r.rid)
        return results, _stats(results, makespan)


def run_sequential(trace: list[tuple[float, SimSpec]], storage: int | None = 0,
                   clock=time.perf_counter, sleep=time.sleep, check_every: int = 4000) -> tuple[list[Result], dict]:
    """Baseline: each request alone, in arrival order, through the single-simulation
    path (FP32 storage by default), its state checked for non-finite values every
    `check_every` steps (the server's longest chunk)."""
    reqs = sorted((Request(i, a, sp) for i, (a, sp) in enumerate(trace)), key=lambda r: r.arrival)
    results = []
    t0 = clock()
    for r in reqs:
        now = clock() - t0
        if now < r.arrival:
            sleep(r.arrival - now)
        adm = clock() - t0
        with start_simulation(r.spec, storage=storage) as s:
            # the same failure check as the server's, at the same granularity
            while True:
                s.step(min(check_every, r.spec.steps - s.t))
                d = s.diagnostics(allow_unstable=True)
                ran = s.t
                if ran >= r.spec.steps or _failed(d):
                    break
        results.append(Result(r.rid, r.arrival, adm, clock() - t0, r.spec.nx * r.spec.ny, ran, d, _failed(d)))
    makespan = clock() - t0
    results.sort(key=lambda r: r.rid)
    return results, _stats(results, makespan)
