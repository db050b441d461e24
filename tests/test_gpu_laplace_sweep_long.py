"""The 40-run Laplace sweep at its full length on the GPU (FP32, 256 x 256 periodic
static bubbles, radii {20..60} x density ratio {1, 10} x viscosity ratio {1, 10} x
sigma {0.001, 0.01}, beta 0.7, 20 000 steps), all runs in one batched launch per
step, against the FP64 oracle's results for the same runs
(tests/golden/laplace_sweep_20000.json, written by make_laplace_sweep.py, which
calls only the oracle).

Per run, with the bar of each quantity:
  dp_avg : the Laplace jump averaged over the second half of the run (sampled
           every 100 steps), within 1 % of the oracle's (the spec bar);
  R_eff  : the bubble's effective radius at the last step, within 1 %;
  max|u| : the largest spurious speed at the last step, within 5 % (a velocity
           at the 1e-5 level, set by the interface's discretisation);
  mass   : each colour's mass conserved to 1e-6 relative over the run.
Each bar is raised to twice the distance between the FP32-compiled oracle
("runs_fp32") and the FP64 oracle where that distance, the method's own FP32
floor, exceeds half of it.  For max|u| the floor is the largest over the runs that
share the density ratio and sigma: at sigma = 0.001 the last-step max|u| is one
sample of a velocity field at the 1e-6 level that also carries the bubble's
acoustic oscillation, and one run's FP32 realisation estimates its FP32 spread
poorly (the per-run floors of one class scatter from 0.2 % to 20 %).  The jump at
the last step alone is printed with its floor but not held to a bar: at density
ratio 10 the bubble's pressure carries acoustic oscillations with a period near
1150 steps and an amplitude of several Laplace jumps, and FP32 rounding alone moves
the oracle's last-step jump by up to a factor 3."""
import json
import os

import numpy as np
import pytest

from paper_1903_01168_gb300 import lbm as L
from paper_1903_01168_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "laplace_sweep_20000.json")


@pytest.fixture(scope="module", autouse=True)
def _native():
    L.load(build_if_missing=True)


def _jump(f, sp):
    a = f["rho_r"] / sp.gamma
    psi = (a - f["rho_b"]) / (a + f["rho_b"])
    return W.laplace_pressure_jump(f["p"], psi, *sp.bubble[:2])


def _rel(a, b):
    return abs(a / b - 1.0)


def _mass_drift(r):
    return max(_rel(r["mass_r"], r["mass_r0"]), _rel(r["mass_b"], r["mass_b0"]))


def test_full_sweep_20000_steps_against_the_oracle():
    with open(GOLDEN) as f:
        gold = json.load(f)
    steps = gold["steps"]
    t_from, t_to, every = gold["dp_avg_window"]
    assert t_to == steps
    specs = W.laplace_sweep(256, steps=steps)
    sims = []
    for sp in specs:
        s = L.Simulation(sp.nx, sp.ny, gamma=sp.gamma, tau_r=sp.tau_r, tau_b=sp.tau_b, sigma=sp.sigma,
                         beta=sp.beta)
        s.init_bubble(*sp.bubble)
        sims.append(s)
    m0 = [(s.diagnostics()["mass_r"], s.diagnostics()["mass_b"]) for s in sims]
    b = L.Batch(sims)
    b.step(t_from, use_graph=True)
    samples = [[] for _ in sims]
    for t in range(t_from, t_to + 1, every):
        if t > t_from:
            b.step(every, use_graph=True)
        for i, (sp, s) in enumerate(zip(specs, sims)):
            samples[i].append(_jump(s.fields(), sp)[0])
    b.close()
    class_floor_u = {}
    for g, h in zip(gold["runs"], gold["runs_fp32"]):
        c = (g["gamma"], g["sigma"])
        class_floor_u[c] = max(class_floor_u.get(c, 0.0), _rel(h["max_u"], g["max_u"]))
    worst = {"dp_avg": 0.0, "r_eff": 0.0, "max_u": 0.0, "mass": 0.0}
    failures = []
    for i, (sp, s, g, h) in enumerate(zip(specs, sims, gold["runs"], gold["runs_fp32"])):
        assert g["finite"] and abs(g["gamma"] - sp.gamma) < 1e-12 and abs(g["sigma"] - sp.sigma) < 1e-15
        assert g["dp_samples"] == len(samples[i])
        f = s.fields()
        s.close()
        assert np.isfinite(f["rho_r"]).all(), i
        dp, reff = _jump(f, sp)
        umax = float(np.sqrt(f["ux"] ** 2 + f["uy"] ** 2).max())
        dp_avg = float(np.mean(samples[i]))
        err = {"dp_avg": _rel(dp_avg, g["dp_avg"]), "r_eff": _rel(reff, g["r_eff"]),
               "max_u": _rel(umax, g["max_u"]),
               "mass": max(_rel(f["rho_r"].sum(), m0[i][0]), _rel(f["rho_b"].sum(), m0[i][1]))}
        floor = {"dp_avg": _rel(h["dp_avg"], g["dp_avg"]), "r_eff": _rel(h["r_eff"], g["r_eff"]),
                 "max_u": class_floor_u[(g["gamma"], g["sigma"])], "mass": _mass_drift(h)}
        bar = {q: max(v, 2.0 * floor[q]) for q, v in {"dp_avg": 0.01, "r_eff": 0.01, "max_u": 0.05,
                                                         "mass": 1e-6}.items()}
        print(f"run {i:2d} gamma {sp.gamma:g} tau {sp.tau_r:.2f}/{sp.tau_b:.2f} sigma {sp.sigma:g} "
              f"R {sp.bubble[2]:g} (Laplace {sp.sigma / sp.bubble[2]:.4e}): "
              f"dp_avg {dp_avg:.5e}/{g['dp_avg']:.5e} ({err['dp_avg']:.1e}, bar {bar['dp_avg']:.1e})  "
              f"last-step dp {dp:.4e}/{g['dp']:.4e} (FP32 floor {_rel(h['dp'], g['dp']):.1e})  "
              f"R_eff {err['r_eff']:.1e}  max|u| {err['max_u']:.1e} (bar {bar['max_u']:.1e})  "
              f"mass {err['mass']:.1e} (bar {bar['mass']:.1e})")
        for q in worst:
            worst[q] = max(worst[q], err[q])
            if err[q] > bar[q]:
                failures.append((i, q, err[q], bar[q]))
    print("worst", worst)
    assert not failures, failures
