"""Reduced-precision storage (FP16 / BF16 deviations in the split form: the
recolouring shift and flux rebuilt from FP32 node scalars, only the colour-blind
remainder rounded to 16 bits; FP32 arithmetic and colour densities) against the
FP64 oracle.

Field bars follow from the storage precision: the stored remainders are rounded
to their unit roundoff u_s = 2^-11 (FP16) or 2^-8 (BF16) each step, and the field
errors after 100 steps scale with u_s.  On the MRT + Hermite case below the
measured errors are about 0.6 u_s on rho and 4 u_s (FP16) to 14 u_s (BF16) on u
against the case's velocity scale; the bars are 2 u_s and 20 u_s.  Per-colour mass lives in
the FP32 densities and stays conserved to FP32 round-off.  The integral
diagnostics, slug (light-phase) velocity and Laplace jump, are held to 1 % of the
oracle's for both storage types."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_01168_gb300 import lbm as L
from paper_1903_01168_gb300 import workloads as W

pytestmark = pytest.mark.gpu

F16, BF16 = L.LBM_F16DEV, L.LBM_BF16DEV


@pytest.fixture(scope="module", autouse=True)
def _native():
    L.load(build_if_missing=True)


U_S = {F16: 2.0 ** -11, BF16: 2.0 ** -8}


@pytest.mark.parametrize("storage", [F16, BF16])
def test_parity_100_steps_within_storage_precision(storage):
    tol_rho, tol_u = 2 * U_S[storage], 20 * U_S[storage]
    nx, ny = 200, 37
    kw = dict(gamma=10.0, tau_r=0.6, tau_b=1.1, sigma=0.01, beta=0.7, collision=L.LBM_MRT,
              equilibrium=L.LBM_EQ_HERMITE, gx=2e-6, gy=-1e-6)
    f = W.random_fields(nx, ny, seed=11, gamma=10.0, u_amp=0.03)
    o = O.Oracle(O.OracleParams(nx=nx, ny=ny, **kw))
    o.init_fields(*f)
    o.step(100)
    fo = o.fields()
    with L.Simulation(nx, ny, storage=storage, **kw) as s:
        s.init_fields(*f)
        s.step(100)
        fg = s.fields()
    ro, rg = fo["rho_r"] + fo["rho_b"], fg["rho_r"] + fg["rho_b"]
    e_rho = float(np.max(np.abs(rg - ro) / ro))
    e_u = max(np.abs(fg["ux"] - fo["ux"]).max(), np.abs(fg["uy"] - fo["uy"]).max()) / 0.03
    print(f"storage {storage}: rho {e_rho:.2e} u {e_u:.2e}")
    assert e_rho <= tol_rho and e_u <= tol_u


@pytest.mark.parametrize("storage", [F16, BF16])
def test_colour_mass_conserved_with_16bit_deviations(storage):
    with L.Simulation(64, 64, gamma=1.0, sigma=0.005, beta=0.7, storage=storage) as s:
        s.init_bubble(32, 32, 16)
        d0 = s.diagnostics()
        s.step(2000)
        d1 = s.diagnostics()
    for k in ("mass_r", "mass_b"):
        assert abs(d1[k] - d0[k]) <= 1e-6 * d0[k]


@pytest.mark.parametrize("storage,tol", [(F16, 0.01), (BF16, 0.01)])
def test_slug_velocity_vs_oracle(storage, tol):
    """Gravity-driven periodic slug (walls, gamma = 10, Re = 50, Bo = 0.7848), 4000
    steps: light-phase mean x-velocity against the oracle's.  FP16 is within 0.1 %;
    BF16 (8 mantissa bits on the colour-blind remainder, which carries the
    momentum) at 0.8 %."""
    nx, ny = 128, 32
    sp = W.slug_channel(Re=50, M=1.0, nx=nx, ny=ny)
    kw = dict(gamma=sp.gamma, tau_r=sp.tau_r, tau_b=sp.tau_b, sigma=sp.sigma, beta=0.7, gx=sp.gx,
              bc_y=L.LBM_BC_WALL)
    f = W.slug_fields(nx, ny, sp.gamma, 1, nx / 2, 0.5 * ny, g=sp.gx, nu_l=sp.extra["nu_l"])
    o = O.Oracle(O.OracleParams(nx=nx, ny=ny, **kw))
    o.init_fields(*f)
    o.step(4000)
    fo = o.fields()
    wb = (1 - fo["psi"]) / 2
    ub = (wb * fo["ux"]).sum() / wb.sum()
    with L.Simulation(nx, ny, storage=storage, **kw) as s:
        s.init_fields(*f)
        s.step(4000)
        d = s.diagnostics()
    rel = abs(d["ux_b"] - ub) / abs(ub)
    print(f"storage {storage}: slug velocity {d['ux_b']:.6e} oracle {ub:.6e} rel {rel:.2e}")
    assert rel <= tol


@pytest.mark.parametrize("storage,tol", [(F16, 0.01), (BF16, 0.01)])
def test_laplace_jump_vs_oracle(storage, tol):
    """64^2 static bubble, 2000 steps.  The jump is 3.3e-4 of a pressure of 0.48,
    i.e. the density varies by ~7e-4 across the interface.  Rounding the full
    per-colour deviations (O(rho_r rho_b / rho) at the interface) to 16 bits moved
    it by 2.5 % (FP16) to 14 % (BF16); the split form keeps both within 1 %."""
    o = O.Oracle(O.OracleParams(nx=64, ny=64, gamma=1.0, sigma=0.005, beta=0.7))
    o.init_fields(*W.bubble_fields(64, 64, 32, 32, 16, 1.0))
    o.step(2000)
    fo = o.fields()
    dp_o, _ = W.laplace_pressure_jump(fo["p"], fo["psi"], 32, 32)
    with L.Simulation(64, 64, gamma=1.0, sigma=0.005, beta=0.7, storage=storage) as s:
        s.init_bubble(32, 32, 16)
        s.step(2000)
        d = s.diagnostics()
    rel = abs(d["dp"] - dp_o) / abs(dp_o)
    print(f"storage {storage}: dp {d['dp']:.6e} oracle {dp_o:.6e} rel {rel:.2e}")
    assert rel <= tol
