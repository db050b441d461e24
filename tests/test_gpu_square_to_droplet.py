"""Square-to-droplet resolution study on the GPU (the paper's Sec. 4): 60, 100 and
200 nodes a side for the density / viscosity ratio pairs (1, 1), (5, 2),
(1000, 1000) and (1, 100), each run for 10 t_sigma (1.7 million steps at 200 for
(1000, 1000), whose heavy phase sets t_sigma).  At 60 x 60 the GPU's error equals
the oracle's; every pressure inside a drop is within 10 % of Laplace's jump, and
for every pair the error at 200 is below the one at 60.  The measured orders of
convergence are printed beside the paper's LBM "bubble only" orders (0.718 for
(1, 1), 1.577 for (5, 2), 0.438 for (1000, 1000), 1.604 for (1, 100)), not pinned:
the paper gives no viscosities, steady-state time or exact norm."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_01168_gb300 import lbm as L
from paper_1903_01168_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [(1, 1), (5, 2), (1000, 1000), (1, 100)]
SIZES = [60, 100, 200]


def _kw(sp):
    return dict(gamma=sp.gamma, tau_r=sp.tau_r, tau_b=sp.tau_b, sigma=sp.sigma, beta=sp.beta)


def test_resolution_study():
    runs = {}
    for r in CASES:
        for n in SIZES:
            sp = W.square_to_droplet(n, r)
            s = L.Simulation(n, n, **_kw(sp))
            s.init_fields(*W.square_fields(n, sp.extra["a"], sp.gamma))
            s.step(sp.steps)                  # each on its own stream: all run concurrently
            runs[(r, n)] = (s, sp)
    err = {}
    for (r, n), (s, sp) in runs.items():
        s.synchronize()
        err[(r, n)] = W.centreline_laplace_error(s.fields()["p"], n, sp.extra["a"], sp.sigma)
        s.close()
    for r in CASES:
        e = np.array([err[(r, n)] for n in SIZES])
        order = -np.polyfit(np.log(SIZES), np.log(e), 1)[0]
        print(f"ratios {r}: errors {np.round(e, 5)} order {order:.3f}")
    for r in CASES:
        e = np.array([err[(r, n)] for n in SIZES])
        assert np.isfinite(e).all() and (e < 0.10).all(), (r, e)
    for r in CASES:
        e = np.array([err[(r, n)] for n in SIZES])
        assert e[-1] < e[0], (r, e)

    # the 60 x 60 (1, 1) case against the oracle
    sp = W.square_to_droplet(60)
    o = O.Oracle(O.OracleParams(nx=60, ny=60, **_kw(sp)))
    o.init_fields(*W.square_fields(60, sp.extra["a"], sp.gamma))
    o.step(sp.steps)
    eo = W.centreline_laplace_error(o.fields()["p"], 60, sp.extra["a"], sp.sigma)
    assert abs(err[((1, 1), 60)] - eo) < 0.05 * eo, (err[((1, 1), 60)], eo)   # FP32 vs FP64 after 8810 steps
