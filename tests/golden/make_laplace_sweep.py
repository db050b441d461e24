"""Write laplace_sweep_20000.json: the FP64 oracle's results for the 40-run Laplace
sweep (256 x 256 periodic static bubbles, radii {20..60} x density ratio {1, 10}
x viscosity ratio {1, 10} x sigma {0.001, 0.01}, beta 0.7) after 20 000 steps.
Calls only the oracle and the seeded workload recipes.

    OMP_NUM_THREADS=1 python tests/golden/make_laplace_sweep.py [--procs 8] [--steps 20000]

Per run: the Laplace jump dp and R_eff (mean p inside r < R_eff/2 minus mean p
outside r > R_eff + 8, R_eff from the light-phase area), the largest spurious
speed max |u|, and the colour masses at t = 0 and at the end."""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))


def run_one(args):
    idx, steps = args
    sys.path.insert(0, ROOT)
    import numpy as np
    from oracle import oracle as O
    from paper_1903_01168_gb300 import workloads as W
    sp = W.laplace_sweep(256, steps=steps)[idx]
    o = O.Oracle(O.OracleParams(nx=sp.nx, ny=sp.ny, gamma=sp.gamma, tau_r=sp.tau_r, tau_b=sp.tau_b,
                                sigma=sp.sigma, beta=sp.beta))
    o.init_fields(*W.bubble_fields(sp.nx, sp.ny, *sp.bubble, sp.gamma))
    f0 = o.fields()
    t0 = time.time()
    o.step(steps)
    f = o.fields()
    cx, cy, _ = sp.bubble
    dp, reff = W.laplace_pressure_jump(f["p"], f["psi"], cx, cy)
    umax = float(np.sqrt(f["ux"] ** 2 + f["uy"] ** 2).max())
    return idx, {"gamma": sp.gamma, "tau_r": sp.tau_r, "tau_b": sp.tau_b, "sigma": sp.sigma, "R": sp.bubble[2],
                 "dp": float(dp), "r_eff": float(reff), "max_u": umax,
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
    with ctx.Pool(a.procs) as pool:
        res = dict(pool.map(run_one, [(i, a.steps) for i in range(40)], chunksize=1))
    out = {"source": "FP64 oracle (oracle/lbm_oracle.c), tests/golden/make_laplace_sweep.py",
           "steps": a.steps, "lattice": [256, 256], "beta": 0.7, "runs": [res[i] for i in range(40)]}
    with open(a.out, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", a.out)


if __name__ == "__main__":
    main()
