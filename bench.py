"""Benchmark of the colour-gradient LBM hot path on GB300.

Workload (default): the Laplace sweep -- 40 independent periodic 256 x 256
static-bubble simulations (radii {20..60} x density ratio {1,10} x viscosity
ratio {1,10} x sigma {0.001, 0.01}, beta 0.7), FP32 populations, advanced
together: one batched fused-kernel launch per time step, K steps captured in a
CUDA graph.  One bench "step" = one LBM time step of all 40 lattices.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  `value` is whole-job MLUPS (million lattice-node
updates per second, both colours of a node counting as one update) over the
device-timed region (inputs resident in HBM).  That region replays the K-step
graph R times back to back, R chosen so that it lasts at least 0.5 s (long
enough for the nvidia-smi clock samples taken during it); `steps` is K,
`timed_steps` R K.  `e2e` is the same metric through the public API with host
buffers: upload of the initial fields, K steps and download of the final
fields, all inside the timed region.  `per_dtype` repeats the device-timed sweep
with FP16 and BF16 deviation storage and gives each storage type's error against
the FP64 oracle on two sampled runs after 100 steps.  `--impl reference` times
the FP64 CPU oracle (all host cores) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic bytes per node update: 18 populations read and written, 4 bytes each in
# FP32 and 2 with 16-bit deviation storage (the hot path's stated figures).  The
# split form of 16-bit storage actually moves 5 FP32 node scalars (densities and the
# split-form scalars) + 16 16-bit residuals each way: STORED_BYTES.
BYTES_PER_UPDATE = {0: 144, 1: 72, 2: 72}
STORED_BYTES = {0: 144, 1: 104, 2: 104}
FALLBACK_HBM_GBS = 6800.0

# DRAM traffic of one k_step_fused launch on this workload from an ncu capture of
# `dram__bytes_read.sum + dram__bytes_write.sum`, valid only for the kernel
# sources with this hash; reported as null otherwise.
NCU_TRAFFIC = {"sources_sha": "60141a825c48cb2c",
               "bytes_per_launch": {0: 229121536 + 154410496, 1: 170580992 + 96698624, 2: 170623488 + 96513792}}


def kernel_sources_sha() -> str:
    h = hashlib.sha256()
    for f in ("lbm_device.cuh", "lbm_kernels.cuh", "lbm_inst.cuh"):
        with open(os.path.join(ROOT, "paper_1903_01168_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(storage: int):
    """DRAM bytes of one sweep launch of this storage type from the ncu capture,
    or None when the kernel sources changed since or no capture exists."""
    if NCU_TRAFFIC["sources_sha"] != kernel_sources_sha():
        return None
    return NCU_TRAFFIC["bytes_per_launch"].get(storage)


def pinned_copy(torch, a):
    """A float64 numpy view of page-locked host memory holding a copy of `a`."""
    import numpy as np
    t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
    v = t.numpy()
    v[...] = a
    return v


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi SM clock / throttle samples while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, dist=None, device: str = "cuda") -> float:
    """The largest value of x over all ranks (x itself without a process group):
    every rank's timed region is bracketed by barriers, so the job takes as long
    as its slowest rank."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(nodes_per_rank: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job MLUPS: every rank runs its own replica of the workload (weak
    scaling), so the job updates world x nodes x steps nodes in `seconds`."""
    return nodes_per_rank * steps * world / seconds / 1e6


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        for k in ("hbm_gbs", "hbm_GBs", "hbm"):
            if k in d and isinstance(d[k], (int, float)):
                return float(d[k]), "of measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "of fallback"


def workload():
    from paper_1903_01168_gb300 import workloads as W
    return W.laplace_sweep(256, steps=20000)


def ensemble_workload():
    from paper_1903_01168_gb300 import workloads as W
    return W.ensemble(seed=W.DEFAULT_SEED, n_sims=256)


def serving_trace_results(args) -> dict:
    """Serving trace: Poisson arrivals of open-channel slug requests (mixed lattice
    sizes, step counts and storage types) through the continuous-batching server,
    then the same trace one request at a time through the plain FP32 path."""
    from paper_1903_01168_gb300 import serving as S
    from paper_1903_01168_gb300 import workloads as W
    trace = W.serving_trace(seed=W.DEFAULT_SEED, n_requests=args.requests, rate_hz=args.rate)
    # warm up kernels and graphs of every storage type
    warm = [(0.0, W.SimSpec(**{**sp.as_dict(), "nx": 256, "ny": 64, "steps": 64})) for _, sp in trace[:3]]
    S.Server(budget_bytes=150e9, chunk=32).run(warm)
    S.run_sequential(warm)
    cap = None if args.active_nodes <= 0 else args.active_nodes
    res_b, st_b = S.Server(budget_bytes=150e9, chunk=args.chunk, max_active_nodes=cap,
                           priority=args.priority).run(trace)
    res_s, st_s = S.run_sequential(trace, storage=0)
    keys = ("requests", "p50_s", "p99_s", "mean_s", "makespan_s", "mlups", "failed")
    return {"workload": f"serving_{args.requests}_requests_poisson_{args.rate}hz",
            "trace": "open-channel slug requests, nx 512..8192, ny 64..256, 5k-50k steps, storage uniform over "
                     "f32 / f16-deviation / bf16-deviation",
            "budget_bytes": 150e9, "chunk_steps": args.chunk, "max_active_nodes": cap, "priority": args.priority,
            "batched": {k: st_b[k] for k in keys}, "sequential_f32": {k: st_s[k] for k in keys},
            "failed_note": "failed = requests whose state went non-finite (retired at the next check, steps "
                           "run counted); request 5 of this trace (864x224, gas inlet Re ~500) also blows up "
                           "in the FP64 oracle"}


def run_serving(args):
    import torch
    from paper_1903_01168_gb300 import lbm as L
    torch.cuda.set_device(0)
    L.load(build_if_missing=True)
    sv = serving_trace_results(args)
    line = {"metric": "MLUPS", "value": sv["batched"]["mlups"], "unit": "MLUPS", "n_gpus": 1, "steps": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "mixed", "data": "synthetic",
            "config": {"workload": sv["workload"], "budget_bytes": 150e9, "chunk_steps": args.chunk,
                       "max_active_nodes": sv["max_active_nodes"]},
            "serving": sv["batched"], "sequential_f32": sv["sequential_f32"]}
    print(json.dumps(line), flush=True)


def host_cores() -> int:
    """Host cores this process may run on (the oracle's OpenMP threads)."""
    n = os.environ.get("OMP_NUM_THREADS")
    if n and n.isdigit():
        return int(n)
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_mlups(specs, steps: int, seconds: float):
    """FP64 oracle on a bounded sample: one sweep run at a time, `steps` steps each,
    until `seconds` of wall time have been spent.  Returns (MLUPS, sample text)."""
    from oracle import oracle as O
    from paper_1903_01168_gb300 import workloads as W
    nodes = 0
    t_used = 0.0
    runs = 0
    for sp in specs:
        o = O.Oracle(O.OracleParams(nx=sp.nx, ny=sp.ny, gamma=sp.gamma, tau_r=sp.tau_r, tau_b=sp.tau_b,
                                    sigma=sp.sigma, beta=sp.beta))
        o.init_fields(*W.bubble_fields(sp.nx, sp.ny, *sp.bubble, sp.gamma))
        t0 = time.perf_counter()
        o.step(steps)
        t_used += time.perf_counter() - t0
        nodes += sp.nx * sp.ny * steps
        runs += 1
        if t_used >= seconds:
            break
    return nodes / t_used / 1e6, (f"{runs} of the 40 runs x {steps} steps on 256x256 (plain C, FP64, "
                                  f"rows split over {host_cores()} OpenMP threads)")


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle as it stands, on this host's cores."""
    if rank != 0:
        return
    specs = workload()
    from oracle import oracle as O
    from paper_1903_01168_gb300 import workloads as W
    sims = []
    for sp in specs[:4]:
        o = O.Oracle(O.OracleParams(nx=sp.nx, ny=sp.ny, gamma=sp.gamma, tau_r=sp.tau_r, tau_b=sp.tau_b,
                                    sigma=sp.sigma, beta=sp.beta))
        o.init_fields(*W.bubble_fields(sp.nx, sp.ny, *sp.bubble, sp.gamma))
        sims.append(o)
    for j in range(args.warmup):
        sims[j % len(sims)].step(1)
    t0 = time.perf_counter()
    for j in range(args.steps):
        sims[j % len(sims)].step(1)
    dt = time.perf_counter() - t0
    mlups = 256 * 256 * args.steps / dt / 1e6
    cores = host_cores()
    sample = (f"each step = 1 time step of one 256x256 sweep run (rotating over 4 runs), FP64 oracle, "
              f"{cores} OpenMP threads")
    line = {
        "impl": "reference", "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "laplace_sweep_40x256x256_f32", "sample": sample},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


STORAGE_NAMES = ["f32", "f16", "bf16"]


class Sweep:
    """The workload's lattices as one batch on `stream` (torch-owned memory),
    with the plan tuned on the batch itself unless autotune is False."""

    def __init__(self, L, specs, storage: int, stream, autotune: bool):
        import torch
        self.specs, self.storage, self.stream = specs, storage, stream
        self.sims = []
        with torch.cuda.stream(stream):
            for sp in specs:
                self.sims.append(L.Simulation(sp.nx, sp.ny, torch_memory=True, gamma=sp.gamma, tau_r=sp.tau_r,
                                              tau_b=sp.tau_b, sigma=sp.sigma, beta=sp.beta, storage=storage,
                                              gx=sp.gx, bc_y=sp.bc_y))
            self.init_all()
            self.tuned, self.tune_s = None, 0.0
            if autotune:
                from paper_1903_01168_gb300.autotune import Autotuner
                ta = time.perf_counter()
                self.tuned = Autotuner().tune_batch(self.sims)
                self.tune_s = time.perf_counter() - ta
                self.init_all()
                self.batch = L.Batch(self.sims, row_overhead=self.tuned["row_overhead"], plan=self.tuned["plan"],
                                     member_plan_rows=self.tuned["member_plan_rows"])
            else:
                self.batch = L.Batch(self.sims)
        self.nodes = sum(sp.nx * sp.ny for sp in specs)

    def init_all(self):
        for sp, s in zip(self.specs, self.sims):
            if sp.geometry == "bubble":
                s.init_bubble(*sp.bubble)
            else:
                s.init_slug(int(sp.slug[0]), sp.slug[1], sp.slug[2], True)

    def timed(self, steps: int, warmup: int, floor_s: float, dist, local: int):
        """Warm up, then time R back-to-back replays of the `steps`-step graph (R so
        that the region lasts at least floor_s), between barriers, with CUDA events
        on the launching stream and nvidia-smi clock samples.  Returns
        (ms of the region, max over ranks; R; clock summary)."""
        import torch
        with torch.cuda.stream(self.stream):
            self.batch.step(warmup, use_graph=True)
            self.batch.step(steps, use_graph=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(self.stream):
            e0.record(self.stream)
            self.batch.step(steps, use_graph=True)
            e1.record(self.stream)
        torch.cuda.synchronize()
        one = max_over_ranks(e0.elapsed_time(e1), dist)
        reps = max(1, int(-(-floor_s * 1e3 // max(one, 1e-3))))
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            torch.cuda.nvtx.range_push("timed")   # ncu --nvtx --nvtx-include timed/ lists these launches
            with torch.cuda.stream(self.stream):
                e0.record(self.stream)
                for _ in range(reps):
                    self.batch.step(steps, use_graph=True)
                e1.record(self.stream)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
        if dist is not None:
            dist.barrier()
        return max_over_ranks(e0.elapsed_time(e1), dist), reps, clk.summary()

    def close(self):
        self.batch.close()
        for s in self.sims:
            s.close()


_ORACLE_FIELDS = {}


def sampled_oracle_error(L, specs, storage: int, idx=(3, 38), steps: int = 100):
    """Relative L-inf error of rho and of u (against max(||u||_inf, sigma / nu)) of
    sampled sweep runs after `steps` steps, GPU storage type `storage` against the
    FP64 oracle, worst over the samples."""
    from oracle import oracle as O
    from paper_1903_01168_gb300 import workloads as W
    import numpy as np
    e_rho = e_u = 0.0
    for i in idx:
        sp = specs[i]
        kw = dict(gamma=sp.gamma, tau_r=sp.tau_r, tau_b=sp.tau_b, sigma=sp.sigma, beta=sp.beta)
        f = W.bubble_fields(sp.nx, sp.ny, *sp.bubble, sp.gamma)
        if (i, steps) not in _ORACLE_FIELDS:
            o = O.Oracle(O.OracleParams(nx=sp.nx, ny=sp.ny, **kw))
            o.init_fields(*f)
            o.step(steps)
            _ORACLE_FIELDS[(i, steps)] = o.fields()
        fo = _ORACLE_FIELDS[(i, steps)]
        with L.Simulation(sp.nx, sp.ny, storage=storage, **kw) as s:
            s.init_fields(*f)
            s.step(steps)
            fg = s.fields()
        ro = fo["rho_r"] + fo["rho_b"]
        e_rho = max(e_rho, float(np.max(np.abs(fg["rho_r"] + fg["rho_b"] - ro) / ro)))
        uref = max(np.abs(fo["ux"]).max(), np.abs(fo["uy"]).max(), sp.sigma / (min(sp.tau_r, sp.tau_b) / 3 - 1 / 6))
        e_u = max(e_u, float(max(np.abs(fg["ux"] - fo["ux"]).max(), np.abs(fg["uy"] - fo["uy"]).max()) / uref))
    return {"rho_rel_linf": e_rho, "u_rel_linf": e_u, "steps": steps,
            "sample": f"sweep runs {list(idx)}, 256x256, vs the FP64 oracle"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--floor-seconds", type=float, default=0.5,
                    help="shortest device-timed region: the K-step graph is replayed until it lasts this long")
    ap.add_argument("--workload", default="laplace_sweep", choices=["laplace_sweep", "ensemble", "serving"],
                    help="laplace_sweep: 40 x 256^2 (default); ensemble: 256 uneven lattices, FP16 "
                         "deviations; serving: Poisson-arrival open-channel requests")
    ap.add_argument("--storage", default="f32", choices=STORAGE_NAMES,
                    help="population storage: FP32, or FP16 / BF16 deviations (FP32 arithmetic)")
    ap.add_argument("--no-per-dtype", action="store_true", help="skip the FP16 / BF16 sweeps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the measured choice of plan_rows per size class (default plan)")
    ap.add_argument("--requests", type=int, default=24, help="serving: number of requests")
    ap.add_argument("--rate", type=float, default=1.5, help="serving: Poisson arrival rate (1/s)")
    ap.add_argument("--chunk", type=int, default=500, help="serving: steps per batched chunk")
    ap.add_argument("--active-nodes", type=int, default=8_000_000,
                    help="serving: lattice nodes the active batch may hold (<= 0: no cap)")
    ap.add_argument("--priority", default="arrival", choices=["arrival", "remaining_steps", "remaining_work"],
                    help="serving: order in which resident requests enter the active batch")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving trace in the default line")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local = dist_env()

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "serving":
        run_serving(args)
        return

    import numpy as np
    import torch
    from paper_1903_01168_gb300 import lbm as L

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    L.load(build_if_missing=(rank == 0 and world == 1))

    specs = workload() if args.workload == "laplace_sweep" else ensemble_workload()
    storage = STORAGE_NAMES.index(args.storage)
    if args.workload == "ensemble":
        storage = 1   # the ensemble is defined with FP16-deviation storage
    stream = torch.cuda.Stream()
    peak, peak_kind = measured_peak()

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---- device-timed region: R replays of the K-step graph, inputs resident in HBM
    sw = Sweep(L, specs, storage, stream, not args.no_autotune)
    nodes = sw.nodes
    ms, reps, clocks = sw.timed(args.steps, args.warmup, args.floor_seconds, dist, local)
    timed_steps = reps * args.steps
    mlups = job_mlups(nodes, timed_steps, world, ms * 1e-3)
    ms_per_step = ms / timed_steps

    # ---- end to end through the public API with host buffers
    host_fields = []
    from paper_1903_01168_gb300 import workloads as W
    for sp in specs:
        if sp.geometry == "bubble":
            f = W.bubble_fields(sp.nx, sp.ny, *sp.bubble, sp.gamma)
        else:
            f = W.slug_fields(sp.nx, sp.ny, sp.gamma, int(sp.slug[0]), sp.slug[1], sp.slug[2], g=sp.gx,
                              nu_l=sp.extra.get("nu_l", 0.1))
        host_fields.append([pinned_copy(torch, a) for a in f])
    host_out = [{k: pinned_copy(torch, np.empty((sp.ny, sp.nx))) for k in ("rho_r", "rho_b", "ux", "uy", "p")}
                for sp in specs]
    barrier()
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for s, f in zip(sw.sims, host_fields):
            s.init_fields(*f)
        sw.batch.step(args.steps, use_graph=True)
        outs = [s.fields(o) for s, o in zip(sw.sims, host_out)]
    torch.cuda.synchronize()
    te = max_over_ranks(time.perf_counter() - te0, dist)
    algo_bytes = BYTES_PER_UPDATE[storage] * nodes
    h2d = sum(4 * sp.nx * sp.ny * 8 for sp in specs)
    d2h = sum(5 * sp.nx * sp.ny * 8 for sp in specs)
    e2e = {"value": job_mlups(nodes, args.steps, world, te), "unit": "MLUPS",
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
           "note": "upload of initial fields from pinned host memory + K steps + download of final "
                   "fields into pinned host memory, per step"}
    assert all(np.isfinite(o["rho_r"]).all() for o in outs)
    tuned, tune_s, items = sw.tuned, sw.tune_s, sw.batch.items
    sw.close()

    achieved = algo_bytes / (ms_per_step * 1e-3) / 1e9
    traffic = ncu_traffic(storage)

    # ---- the same sweep with every storage type, and each one's error against the oracle
    per_dtype = None
    if args.workload == "laplace_sweep" and not args.no_per_dtype:
        per_dtype = {}
        for st, name in enumerate(STORAGE_NAMES):
            if st == storage:
                m, ach = mlups, achieved
            else:
                sw2 = Sweep(L, specs, st, stream, not args.no_autotune)
                ms2, reps2, _ = sw2.timed(args.steps, args.warmup, args.floor_seconds / 2, dist, local)
                sw2.close()
                m = job_mlups(nodes, reps2 * args.steps, world, ms2 * 1e-3)
                ach = BYTES_PER_UPDATE[st] * nodes / (ms2 / (reps2 * args.steps) * 1e-3) / 1e9
            per_dtype[name] = {"mlups": m, "bytes_per_update": BYTES_PER_UPDATE[st], "achieved_gbs": ach,
                               "frac": ach / peak, "stored_bytes_per_update": STORED_BYTES[st],
                               "frac_of_stored_bytes": ach / peak * STORED_BYTES[st] / BYTES_PER_UPDATE[st],
                               "traffic": ncu_traffic(st),
                               "vs_oracle": sampled_oracle_error(L, specs, st) if rank == 0 else None}

    line = {
        "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "timed_steps": timed_steps, "graph_replays": reps,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if storage == 0 else STORAGE_NAMES[storage] + "-deviation (f32 math)",
        "data": "synthetic",
        "config": {"workload": (f"laplace_sweep_40x256x256_{STORAGE_NAMES[storage]}"
                                if args.workload == "laplace_sweep" else "ensemble_256_uneven_f16dev"),
                   "lattices": len(specs), "nx": specs[0].nx if args.workload == "laplace_sweep" else "64..512",
                   "ny": specs[0].ny if args.workload == "laplace_sweep" else "64..1024",
                   "nodes_per_step": nodes, "storage": STORAGE_NAMES[storage],
                   "kernel": "k_step_fused (batched, graph)",
                   "work_items": items,
                   "autotune": (None if tuned is None else
                                {"seconds": round(tune_s, 2), "row_overhead": tuned["row_overhead"],
                                 "plan": {0: "auto", 1: "balanced", 2: "split"}[tuned["plan"]],
                                 "plan_rows": {k: v for k, v in tuned["classes"].items() if v != 8}}),
                   "l2": f"inputs larger than L2: {STORED_BYTES[storage] * nodes / 1e6:.0f} MB of state "
                         f"touched per step",
                   "parallelism":
                   "replicas only" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                     "algorithmic_bytes_per_launch": algo_bytes},
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": timed_steps + reps,
    }
    if per_dtype is not None:
        line["per_dtype"] = per_dtype
    if rank == 0 and world == 1 and args.workload == "laplace_sweep" and not args.no_serving:
        line["serving"] = serving_trace_results(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "laplace_sweep":
        v, sample = oracle_mlups(specs, 100, args.cpu_seconds)
        line["cpu_baseline"] = {"value": v, "unit": "MLUPS", "cores": host_cores(), "kind": "oracle",
                                "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
