"""Benchmark of the colour-gradient LBM hot path on GB300.

Workload (default): the Laplace sweep -- 40 independent periodic 256 x 256
static-bubble simulations (radii {20..60} x density ratio {1,10} x viscosity
ratio {1,10} x sigma {0.001, 0.01}, beta 0.7), FP32 populations, advanced
together: one batched fused-kernel launch per time step, K steps captured in a
CUDA graph.  One bench "step" = one LBM time step of all 40 lattices.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  `value` is whole-job MLUPS (million lattice-node
updates per second, both colours of a node counting as one update) over the
device-timed region (inputs resident in HBM).  `e2e` is the same metric through
the public API with host buffers: upload of the initial fields, K steps and
download of the final fields, all inside the timed region.  `--impl reference`
times the FP64 CPU oracle on a bounded sample of the same workload.
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

# per node update, read and written: 2 FP32 densities + 16 FP32 deviations, or 5 FP32
# node scalars (densities and the split-form scalars) + 16 16-bit deviation residuals
BYTES_PER_UPDATE = {0: 144, 1: 104, 2: 104}
FALLBACK_HBM_GBS = 6800.0

# DRAM traffic of one k_step_fused launch on this workload from an ncu capture
# (profiles/k_step_fused_laplace_sweep_40x256.md), valid only for the kernel
# sources with this hash; reported as null otherwise.
NCU_TRAFFIC = {"sources_sha": "53264e91f9e3623d", "bytes_per_launch": 222819328 + 155179520}


def kernel_sources_sha() -> str:
    h = hashlib.sha256()
    for f in ("lbm_device.cuh", "lbm_kernels.cuh"):
        with open(os.path.join(ROOT, "paper_1903_01168_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


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


def run_serving(args):
    """Serving trace: Poisson arrivals of open-channel slug requests (mixed lattice
    sizes, step counts and storage types) through the continuous-batching server,
    then the same trace one request at a time through the plain FP32 path."""
    import torch
    from paper_1903_01168_gb300 import lbm as L
    from paper_1903_01168_gb300 import serving as S
    from paper_1903_01168_gb300 import workloads as W
    torch.cuda.set_device(0)
    L.load(build_if_missing=True)
    trace = W.serving_trace(seed=W.DEFAULT_SEED, n_requests=args.requests, rate_hz=args.rate)
    # warm up kernels and graphs of every storage type
    warm = [(0.0, W.SimSpec(**{**sp.as_dict(), "nx": 256, "ny": 64, "steps": 64})) for _, sp in trace[:3]]
    S.Server(budget_bytes=150e9, chunk=32).run(warm)
    S.run_sequential(warm)
    res_b, st_b = S.Server(budget_bytes=150e9, chunk=args.chunk).run(trace)
    res_s, st_s = S.run_sequential(trace, storage=0)
    line = {"metric": "MLUPS", "value": st_b["mlups"], "unit": "MLUPS", "n_gpus": 1, "steps": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"serving_{args.requests}_requests_poisson_{args.rate}hz",
                       "budget_bytes": 150e9, "chunk_steps": args.chunk},
            "serving": {k: st_b[k] for k in ("requests", "p50_s", "p99_s", "mean_s", "makespan_s", "mlups")},
            "sequential_f32": {k: st_s[k] for k in ("requests", "p50_s", "p99_s", "mean_s", "makespan_s",
                                                     "mlups")}}
    print(json.dumps(line), flush=True)


def oracle_mlups(specs, steps: int, seconds: float):
    """FP64 oracle on a bounded sample: one sweep run at a time, `steps` steps each,
    until `seconds` of CPU work have been spent.  Returns (MLUPS, sample text)."""
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
    return nodes / t_used / 1e6, f"{runs} of the 40 runs x {steps} steps on 256x256 (single-threaded C, FP64)"


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
    sample = f"each step = 1 time step of one 256x256 sweep run (rotating over 4 runs), FP64 oracle"
    line = {
        "impl": "reference", "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "laplace_sweep_40x256x256_f32", "sample": sample},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--workload", default="laplace_sweep", choices=["laplace_sweep", "ensemble", "serving"],
                    help="laplace_sweep: 40 x 256^2 (default); ensemble: 256 uneven lattices, FP16 "
                         "deviations; serving: Poisson-arrival open-channel requests")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"],
                    help="population storage: FP32, or FP16 / BF16 deviations (FP32 arithmetic)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the measured choice of plan_rows per size class (default plan)")
    ap.add_argument("--requests", type=int, default=24, help="serving: number of requests")
    ap.add_argument("--rate", type=float, default=1.5, help="serving: Poisson arrival rate (1/s)")
    ap.add_argument("--chunk", type=int, default=500, help="serving: steps per batched chunk")
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
    storage = {"f32": 0, "f16": 1, "bf16": 2}[args.storage]
    if args.workload == "ensemble":
        storage = 1   # the ensemble is defined with FP16-deviation storage
    stream = torch.cuda.Stream()
    sim_params = [dict(gamma=sp.gamma, tau_r=sp.tau_r, tau_b=sp.tau_b, sigma=sp.sigma, beta=sp.beta,
                       storage=storage, gx=sp.gx, bc_y=sp.bc_y) for sp in specs]
    sims = []
    with torch.cuda.stream(stream):
        for sp, kw in zip(specs, sim_params):
            sims.append(L.Simulation(sp.nx, sp.ny, torch_memory=True, **kw))

    def init_all():
        for sp, s in zip(specs, sims):
            if sp.geometry == "bubble":
                s.init_bubble(*sp.bubble)
            else:
                s.init_slug(int(sp.slug[0]), sp.slug[1], sp.slug[2], True)

    tuned = None
    with torch.cuda.stream(stream):
        init_all()
        if not args.no_autotune:
            # per size class plan_rows and plan options, timed on this batch, then a fresh start
            from paper_1903_01168_gb300.autotune import Autotuner
            ta = time.perf_counter()
            tuned = Autotuner().tune_batch(sims)
            tune_s = time.perf_counter() - ta
            init_all()
            batch = L.Batch(sims, row_overhead=tuned["row_overhead"], plan=tuned["plan"],
                            member_plan_rows=tuned["member_plan_rows"])
        else:
            batch = L.Batch(sims)
    nodes = sum(sp.nx * sp.ny for sp in specs)

    def barrier():
        if dist is not None:
            dist.barrier()

    # warm-up (also captures the graphs of both lengths used below)
    with torch.cuda.stream(stream):
        batch.step(args.warmup, use_graph=True)
        batch.step(args.steps, use_graph=True)
    torch.cuda.synchronize()

    # ---- device-timed region: K steps, inputs resident in HBM
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            ev0.record(stream)
            batch.step(args.steps, use_graph=True)
            ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    t_max = max_over_ranks(ms, dist)
    mlups = job_mlups(nodes, args.steps, world, t_max * 1e-3)
    ms_per_step = t_max / args.steps

    # ---- end to end through the public API with host buffers
    host_fields = []
    from paper_1903_01168_gb300 import workloads as W
    for sp in specs:
        if sp.geometry == "bubble":
            f = W.bubble_fields(sp.nx, sp.ny, *sp.bubble, sp.gamma)
        else:
            f = W.slug_fields(sp.nx, sp.ny, sp.gamma, int(sp.slug[0]), sp.slug[1], sp.slug[2], g=sp.gx,
                              nu_l=sp.extra.get("nu_l", 0.1))
        host_fields.append([np.ascontiguousarray(a) for a in f])
    barrier()
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for s, f in zip(sims, host_fields):
            s.init_fields(*f)
        batch.step(args.steps, use_graph=True)
        outs = [s.fields() for s in sims]
    torch.cuda.synchronize()
    te = max_over_ranks(time.perf_counter() - te0, dist)
    algo_bytes = BYTES_PER_UPDATE[storage] * nodes
    h2d = sum(4 * sp.nx * sp.ny * 8 for sp in specs)
    d2h = sum(5 * sp.nx * sp.ny * 8 for sp in specs)
    e2e = {"value": job_mlups(nodes, args.steps, world, te), "unit": "MLUPS",
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
           "note": "upload of initial fields + K steps + download of final fields, per step"}
    assert all(np.isfinite(o["rho_r"]).all() for o in outs)

    peak, peak_kind = measured_peak()
    achieved = algo_bytes / (ms_per_step * 1e-3) / 1e9
    traffic = (NCU_TRAFFIC["bytes_per_launch"]
               if NCU_TRAFFIC["sources_sha"] == kernel_sources_sha() and storage == 0 else None)
    line = {
        "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": (f"laplace_sweep_40x256x256_{args.storage}" if args.workload == "laplace_sweep"
                                else "ensemble_256_uneven_f16dev"),
                   "lattices": len(specs), "nx": specs[0].nx if args.workload == "laplace_sweep" else "64..512",
                   "ny": specs[0].ny if args.workload == "laplace_sweep" else "64..1024",
                   "nodes_per_step": nodes, "storage": ["f32", "f16", "bf16"][storage],
                   "kernel": "k_step_fused (batched, graph)",
                   "work_items": batch.items,
                   "autotune": (None if tuned is None else
                                {"seconds": round(tune_s, 2), "row_overhead": tuned["row_overhead"],
                                 "plan": {0: "auto", 1: "balanced", 2: "split"}[tuned["plan"]],
                                 "plan_rows": {k: v for k, v in tuned["classes"].items() if v != 8}}),
                   "l2": f"inputs larger than L2: {2 * algo_bytes / 2e6:.0f} MB of state touched per step",
                   "parallelism":
                   "replicas only" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                     "algorithmic_bytes_per_launch": algo_bytes},
        "clocks": clk.summary(),
        "e2e": e2e,
        "gpu_launches": args.steps + 1,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "laplace_sweep":
        v, sample = oracle_mlups(specs, 100, args.cpu_seconds)
        line["cpu_baseline"] = {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    batch.close()
    for s in sims:
        s.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
