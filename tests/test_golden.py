"""Fixtures transcribed from the paper's printed tables (tests/golden/), each with
its citation in the file header, checked against the oracle and the workload
recipes."""
import os

import numpy as np

from oracle import oracle as O
from paper_1903_01168_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as f:
        return [l.split() for l in f if l.strip() and not l.startswith("#")]


def test_mrt_matrices_match_printed_appendix():
    """Appendix 'Transformation matrices': the oracle's M and M^-1 are the printed ones."""
    rows = np.array(_rows("mrt_matrices.txt"), dtype=np.float64)
    M_print, Minv36_print = rows[:9], rows[9:]
    M, Mi = O.mrt_matrices()
    assert np.array_equal(M, M_print)
    assert np.array_equal(np.round(Mi * 36), Minv36_print)
    assert np.abs(Mi * 36 - Minv36_print).max() < 1e-13


def test_slug_table_tau_from_reynolds():
    """Sec. 5.1 tables: with g = 5e-7, H = 91, Re = g H^3 / (8 nu_l^2) and
    tau = 3 nu + 1/2, Re = 10 gives the printed tau_l = 0.706 and mu_l = rho_l nu_l
    = 3.43e-1 (the rule slug_channel() uses to set g from Re)."""
    for Re, mu_l, tau_l in np.array(_rows("slug_viscosity_table.txt"), dtype=np.float64):
        nu_l = np.sqrt(5e-7 * 91 ** 3 / (8 * Re))
        assert abs(W.tau_of_nu(nu_l) - tau_l) < 6e-4
        assert abs(5.0 * nu_l - mu_l) / mu_l < 2e-3
