"""Square-to-droplet resolution study (the paper's Sec. 4): workload recipe, the
centreline Laplace error measure, and the oracle at 60 x 60.  The paper gives no
viscosities, no steady-state time and no exact error norm, so its printed
convergence orders are reported beside the measured ones rather than pinned."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_01168_gb300 import workloads as W


def test_recipe_follows_the_printed_setup():
    for n in (60, 100, 200):
        sp = W.square_to_droplet(n)
        assert sp.nx == sp.ny == n and sp.sigma == 0.01
        assert sp.extra["a"] == round(0.33 * n)
        rr, rb, _, _ = W.square_fields(n, sp.extra["a"], sp.gamma)
        assert rb.sum() == sp.extra["a"] ** 2                                  # exactly a x a nodes
        assert abs(sp.beta - 0.99 * (60 / n) ** 0.625) < 1e-12
    sp = W.square_to_droplet(100, (5, 2))
    nu_h, nu_l = (sp.tau_r - 0.5) / 3, (sp.tau_b - 0.5) / 3
    assert sp.gamma == 5 and abs(sp.gamma * nu_h / nu_l - 2.0) < 1e-12       # mu ratio 2


def test_error_measure_is_zero_for_the_exact_jump():
    n, a, sigma = 100, 33.0, 0.01
    R = a / math.sqrt(math.pi)
    c = np.arange(n) + 0.5
    r = np.hypot(c[None, :] - n / 2, c[:, None] - n / 2)
    p = np.where(r < R, 0.4 + sigma / R, 0.4)
    assert W.centreline_laplace_error(p, n, a, sigma) < 1e-12
    assert abs(W.centreline_laplace_error(p * 0 + 0.4, n, a, sigma) - 1.0) < 1e-12


@pytest.mark.slow
def test_oracle_60_reaches_laplace():
    sp = W.square_to_droplet(60)
    o = O.Oracle(O.OracleParams(nx=60, ny=60, gamma=sp.gamma, tau_r=sp.tau_r, tau_b=sp.tau_b,
                                sigma=sp.sigma, beta=sp.beta))
    o.init_fields(*W.square_fields(60, sp.extra["a"], sp.gamma))
    o.step(sp.steps)
    e = W.centreline_laplace_error(o.fields()["p"], 60, sp.extra["a"], sp.sigma)
    assert e < 0.05, e
