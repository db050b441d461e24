"""Rayleigh-Taylor workload (the paper's two-phase instability case): the seeded
geometry and parameters, and the oracle's behaviour on a reduced box -- exact
per-colour mass, mirror symmetry about the axis of the imposed sine mode, and
the heavy spike falling / light bubble rising where the interface starts
lowest / highest.  The paper compares its result with interfaces it does not
print, so no quantitative interface position is pinned."""
import math

import numpy as np

from oracle import oracle as O
from paper_1903_01168_gb300 import workloads as W


def test_workload_matches_the_printed_setup():
    sp = W.rayleigh_taylor()
    assert sp.ny == 2 * sp.nx and abs(sp.nx * sp.ny - 40000) < 1000
    assert sp.gamma == 1.8 and sp.tau_r == sp.tau_b and sp.sigma == 0.0
    assert sp.gy == -1e-4 and sp.gx == 0.0 and sp.bc_y == 1
    nu = (sp.tau_r - 0.5) / 3.0
    assert abs(math.sqrt((sp.ny / 2) ** 3 * 1e-4) / nu - 420.0) < 1e-9
    rr, rb, ux, uy = W.rayleigh_taylor_fields(sp.nx, sp.ny, sp.gamma, sp.extra["amp"])
    assert ((rr > 0) ^ (rb > 0)).all()                         # sharp interface
    assert rr[-1].all() and rb[0].all()                        # heavy on top
    idx = (sp.nx // 2 - 1 - np.arange(sp.nx)) % sp.nx          # mirror axis of the mode
    assert np.array_equal(rr, rr[:, idx])
    assert rr.sum() / sp.gamma == rb.sum()                     # equal volumes


def _column_heights(f):
    return ((1.0 - f["psi"]) / 2.0).sum(axis=0)                # light-phase height per column


def test_oracle_spike_falls_and_bubble_rises_symmetrically():
    L, H = 40, 80
    g = 1e-4
    nu = math.sqrt((H / 2) ** 3 * g) / 100.0                   # Re 100 on the reduced box
    tau = W.tau_of_nu(nu)
    o = O.Oracle(O.OracleParams(nx=L, ny=H, gamma=1.8, tau_r=tau, tau_b=tau, sigma=0.0, beta=0.7,
                                gy=-g, bc_y=1))
    o.init_fields(*W.rayleigh_taylor_fields(L, H, 1.8, 0.15))
    f0 = o.fields()
    h0 = _column_heights(f0)
    m0 = (f0["rho_r"].sum(), f0["rho_b"].sum())
    o.step(int(math.sqrt(H / g)))                              # one t_g
    f1 = o.fields()
    h1 = _column_heights(f1)
    assert abs(f1["rho_r"].sum() - m0[0]) <= 1e-12 * m0[0]
    assert abs(f1["rho_b"].sum() - m0[1]) <= 1e-12 * m0[1]
    spike, bubble = L // 4 - 1, 3 * L // 4 - 1                 # lowest / highest start of the interface
    assert h0[spike] < h0[bubble]
    assert h1[spike] < h0[spike] - 0.5 and h1[bubble] > h0[bubble] + 0.5
    idx = (L // 2 - 1 - np.arange(L)) % L
    assert np.abs(f1["psi"] - f1["psi"][:, idx]).max() < 1e-9
    assert np.abs(f1["ux"] + f1["ux"][:, idx]).max() < 1e-12 + 1e-9 * np.abs(f1["ux"]).max()
