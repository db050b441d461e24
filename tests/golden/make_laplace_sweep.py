"""Write laplace_sweep_20000.json: the oracle's results for the 40-run Laplace
sweep (256 x 256 periodic static bubbles, radii {20..60} x density ratio {1, 10}
x viscosity ratio {1, 10} x sigma {0.001, 0.01}, beta 0.7) after 20 000 steps.
Calls only the oracle and the seeded workload recipes.

    OMP_NUM_THREADS=1 python tests/golden/make_laplace_sweep.py [--procs 8] [--steps 20000]

Per run: the Laplace jump dp and R_eff at the last step (mean p inside
r < R_eff/2 minus mean p outside r > R_eff + 8, R_eff from the light-phase
area), the jump averaged over the second half of the run (sampled every 100
steps: at density ratio 10 the bubble's pressure carries acoustic oscillations
with a period near 1150 steps and an amplitude of several Laplace jumps, so the
last step alone samples a phase), the largest spurious speed max |u|, and the
colour masses at t = 0 and at the end.

"runs" come from the FP64 oracle; "runs_fp32" from the same oracle source
compiled with an FP32 arithmetic type (oracle.fp32_library): what FP32 rounding
alone does to each result."""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
SAMPLE_EVERY = 100

_FP32_LIB = None


def run_one(args):
    idx, steps, fp32 = args
    sys.path.insert(0, ROOT)
    import tempfile
    import numpy as np
    from oracle import oracle as O
    from paper_1903_01168_gb300 import workloads as W
    global _FP32_LIB
    library = None
    if fp32:
        if _FP32_LIB is None:
            _FP32_LIB = O.fp32_library(tempfile.mkdtemp(prefix="orc32_"))
        library = _FP32_LIB
    sp = W.laplace_sweep(256, steps=steps)[idx]
    o = O.Oracle(O.OracleParams(nx=sp.nx, ny=sp.ny, gamma=sp.gamma, tau_r=sp.tau_r, tau_b=sp.tau_b,
                                sigma=sp.sigma, beta=sp.beta), library=library)
    o.init_fields(*W.bubble_fields(sp.nx, sp.ny, *sp.bubble, sp.gamma))
    f0 = o.fields()
    cx, cy, _ = sp.bubble
    t0 = time.time()
    half = steps // 2
    o.step(half)
    samples = []
    for t in range(half, steps + 1, SAMPLE_EVERY):
        if t > half:
            o.step(SAMPLE_EVERY)
        f = o.fields()
        samples.append(float(W.laplace_pressure_jump(f["p"], f["psi"], cx, cy)[0]))
    dp, reff = W.laplace_pressure_jump(f["p"], f["psi"], cx, cy)
    umax = float(np.sqrt(f["ux"] ** 2 + f["uy"] ** 2).max())
    return idx, {"gamma": sp.gamma, "tau_r": sp.tau_r, "tau_b": sp.tau_b, "sigma": sp.sigma, "R": sp.bubble[2],
                 "dp": float(dp), "r_eff": float(reff), "max_u": umax,
                 "dp_avg": float(np.mean(samples)), "dp_samples": len(samples),
                 "mass_r0": float(f0["rho_r"].sum()), "mass_b0": float(f0["rho_b"].sum()),
                 "mass_r": float(f["rho_r"].sum()), "mass_b": float(f["rho_b"].sum()),
                 "finite": bool(np.isfinite(f["rho_r"]).all()), "seconds": time.time() - t0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--out", default=os.path.join(HERE, "laplace_sweep_20000.json"))
    a = ap.parse_args()
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    ctx = mp.get_context("spawn")
    out = {"source": "FP64 oracle (oracle/lbm_oracle.c), tests/golden/make_laplace_sweep.py",
           "source_fp32": "the same oracle source compiled with ORC_REAL=float (oracle.fp32_library)",
           "steps": a.steps, "lattice": [256, 256], "beta": 0.7,
           "dp_avg_window": [a.steps // 2, a.steps, SAMPLE_EVERY]}
    for key, fp32 in (("runs", False), ("runs_fp32", True)):
        with ctx.Pool(a.procs) as pool:
            res = dict(pool.map(run_one, [(i, a.steps, fp32) for i in range(40)], chunksize=1))
        out[key] = [res[i] for i in range(40)]
        print("done", key, flush=True)
    with open(a.out, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", a.out)


if __name__ == "__main__":
    main()
