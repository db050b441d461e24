"""Continuous-batching serving loop for colour-gradient LBM simulation requests.

A request is a simulation spec (lattice, physics, boundary conditions, storage
type, number of steps) with an arrival time.  The server:

  * keeps every admitted simulation resident in device memory until it is done;
  * admits waiting requests in arrival order while the sum of the resident state
    bytes stays within an HBM budget and the active lattice nodes stay within
    `max_active_nodes`, about what it takes to keep every SM busy in one launch
    (first come, first served: a request that does not fit blocks the ones
    behind it).  Running more at once would only share the GPU among them and
    delay every result;
  * advances all resident simulations together, one batched fused-kernel launch
    per time step and storage type, replaying a graph of `graph_steps` steps; each
    simulation carries its own stop step, so one that finishes inside a chunk
    simply stops there while the others go on;
  * between chunks retires the finished simulations (their diagnostics are read
    back), frees their memory and admits new arrivals, which therefore join work
    already on the device.

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
    steps: int
    diag: dict = field(default_factory=dict)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def state_bytes(spec: SimSpec) -> int:
    """Device bytes a simulation of this spec keeps resident (both state buffers)."""
    p = params_of(spec)
    return L.lbm_bytes_required(spec.nx, spec.ny, p)


class Admission:
    """First-come-first-served admission under a byte budget (host logic only)."""

    def __init__(self, budget_bytes: int, max_active_nodes: int | None = None):
        self.budget = int(budget_bytes)
        self.resident = 0
        self.max_nodes = None if max_active_nodes is None else int(max_active_nodes)
        self.active_nodes = 0

    def fits(self, nbytes: int, nodes: int = 0) -> bool:
        if self.resident + nbytes > self.budget:
            return False
        # the node cap never holds back a request when nothing is active
        return self.max_nodes is None or self.active_nodes == 0 or self.active_nodes + nodes <= self.max_nodes

    def take(self, waiting: deque, now: float, size_of, nodes_of=lambda r: 0) -> list:
        """Pop and return the requests that have arrived by `now` and fit, in
        arrival order, stopping at the first one that does not fit."""
        out = []
        while waiting and waiting[0].arrival <= now:
            nb = size_of(waiting[0])
            if nb > self.budget:
                raise ValueError(f"request {waiting[0].rid} needs {nb} bytes, more than the whole budget")
            nn = nodes_of(waiting[0])
            if not self.fits(nb, nn):
                break
            self.resident += nb
            self.active_nodes += nn
            out.append(waiting.popleft())
        return out

    def release(self, nbytes: int, nodes: int = 0):
        self.resident -= int(nbytes)
        self.active_nodes -= int(nodes)
        assert self.resident >= 0 and self.active_nodes >= 0


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
            "makespan_s": makespan, "mlups": work / makespan / 1e6, "updates": work}


class Server:
    """Continuous-batching server on the current CUDA device."""

    def __init__(self, budget_bytes: float = 150e9, chunk: int = 500, max_chunk: int = 4000,
                 graph_steps: int = 32, max_active_nodes: int | None = 8_000_000,
                 clock=time.perf_counter, sleep=time.sleep):
        self.admission = Admission(int(budget_bytes), max_active_nodes)
        self.chunk = int(chunk)            # shortest chunk (bounds the wait of a new arrival)
        self.max_chunk = int(max_chunk)
        self.graph_steps = int(graph_steps)   # steps per graph replay (0: direct launches only)
        self.clock = clock
        self.sleep = sleep

    def _chunk_len(self, active, waiting, now: float) -> int:
        """Run to the next completion, but no longer than max_chunk; only `chunk`
        steps while the next request has not arrived yet (it may fit when it
        does).  A request that has arrived and still waits is held back by the
        budget or the node cap, which only a completion relieves."""
        left = min(r.spec.steps - s.t for s, r, _, _ in active.values())
        n = max(1, min(left, self.max_chunk))
        if waiting and waiting[0].arrival > now:
            n = min(n, self.chunk)
        return n

    def run(self, trace: list[tuple[float, SimSpec]]) -> tuple[list[Result], dict]:
        reqs = [Request(i, a, sp) for i, (a, sp) in enumerate(trace)]
        waiting = deque(sorted(reqs, key=lambda r: r.arrival))
        active: dict[int, tuple] = {}          # rid -> (sim, request, admitted_at, bytes)
        results: list[Result] = []
        batch = None
        members: tuple = ()
        t0 = self.clock()
        while waiting or active:
            now = self.clock() - t0
            for r in self.admission.take(waiting, now, lambda q: state_bytes(q.spec),
                                         lambda q: q.spec.nx * q.spec.ny):
                s = start_simulation(r.spec)
                s.set_stop(r.spec.steps)
                active[r.rid] = (s, r, now, state_bytes(r.spec))
            if not active:
                self.sleep(max(0.0, waiting[0].arrival - (self.clock() - t0)))
                continue
            key = tuple(sorted(active))
            if key != members:
                if batch is not None:
                    batch.close()
                batch = L.Batch([active[k][0] for k in key])
                members = key
            n = self._chunk_len(active, waiting, self.clock() - t0)
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
                if s.t >= r.spec.steps:
                    d = s.diagnostics(allow_unstable=True)
                    results.append(Result(r.rid, r.arrival, adm, done, r.spec.nx * r.spec.ny, r.spec.steps, d))
                    retired.append(k)
            if retired:
                batch.close()                   # no batch may refer to a freed simulation
                batch = None
                members = ()
                for k in retired:
                    s, r, adm, nb = active.pop(k)
                    s.close()
                    self.admission.release(nb, r.spec.nx * r.spec.ny)
        if batch is not None:
            batch.close()
        makespan = self.clock() - t0
        results.sort(key=lambda r: r.rid)
        return results, _stats(results, makespan)


def run_sequential(trace: list[tuple[float, SimSpec]], storage: int | None = 0,
                   clock=time.perf_counter, sleep=time.sleep) -> tuple[list[Result], dict]:
    """Baseline: each request alone, in arrival order, through the single-simulation
    path (FP32 storage by default)."""
    reqs = sorted((Request(i, a, sp) for i, (a, sp) in enumerate(trace)), key=lambda r: r.arrival)
    results = []
    t0 = clock()
    for r in reqs:
        now = clock() - t0
        if now < r.arrival:
            sleep(r.arrival - now)
        adm = clock() - t0
        with start_simulation(r.spec, storage=storage) as s:
            s.step(r.spec.steps)
            d = s.diagnostics(allow_unstable=True)
        results.append(Result(r.rid, r.arrival, adm, clock() - t0, r.spec.nx * r.spec.ny, r.spec.steps, d))
    makespan = clock() - t0
    results.sort(key=lambda r: r.rid)
    return results, _stats(results, makespan)
