"""GPU parity: the CUDA path (called through the C ABI) against the FP64 oracle on the
same seeded inputs, plus bit-level consistency of the GPU paths among themselves.

The parity bar is a relative L-infinity of 1e-5 on rho and u after 100 FP32 steps:
  rho   : max_x |rho_gpu - rho_ora| / rho_ora                      <= 1e-5
  u     : max_x |u_gpu - u_ora| / max(||u_ora||_inf, U_ref)        <= 1e-5
  u_inf : max_x |u_gpu - u_ora| / ||u_ora||_inf                    <= max(1e-5, 2 F)
  colour: max_x |rho_r,gpu - rho_r,ora| / rho_ora                  <= max(1e-5, 2 F)
U_ref is the case's velocity scale (the imposed speed for flows; the capillary
velocity sigma / (rho nu) for static bubbles).  F is the same error of the oracle
compiled with an FP32 arithmetic type against the FP64 oracle on the same case: the
method's own FP32 floor.  Where the flow is a static bubble, ||u_ora||_inf is the
spurious current (1e-4 of U_ref), and F relative to it reaches 1e-4; the test prints
every figure and holds each to the larger of 1e-5 and twice the floor.  Where the
floor on rho or on the U_ref-floored u itself exceeds 1e-5 (the alternating inlet,
whose abrupt phase switches amplify rounding), those bars become max(1e-5, 2 F) as
well, and the test says so."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_01168_gb300 import lbm as L
from paper_1903_01168_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _native():
    L.load(build_if_missing=True)


def _oracle_params(nx, ny, kw):
    ok = {k: v for k, v in kw.items() if k in O.OracleParams.__dataclass_fields__}
    return O.OracleParams(nx=nx, ny=ny, **ok)


def _gpu_params(kw):
    return {k: v for k, v in kw.items() if k in L.PARAM_NAMES}


def run_pair(nx, ny, fields, steps, kernel=L.LBM_KERNEL_FUSED, **kw):
    o = O.Oracle(_oracle_params(nx, ny, kw))
    o.init_fields(*fields)
    o.step(steps)
    fo = o.fields()
    with L.Simulation(nx, ny, kernel=kernel, **_gpu_params(kw)) as s:
        s.init_fields(*fields)
        s.step(steps)
        fg = s.fields()
    return fo, fg


def errors(fo, fg, u_ref):
    """(rho, u against max(||u||_inf, U_ref), colour split) errors of fg against fo."""
    rho_o = fo["rho_r"] + fo["rho_b"]
    rho_g = fg["rho_r"] + fg["rho_b"]
    e_rho = np.max(np.abs(rho_g - rho_o) / rho_o)
    umax = max(np.abs(fo["ux"]).max(), np.abs(fo["uy"]).max(), u_ref)
    e_u = max(np.abs(fg["ux"] - fo["ux"]).max(), np.abs(fg["uy"] - fo["uy"]).max()) / umax
    # colour split, relative to the local total density
    e_col = np.max(np.abs(fg["rho_r"] - fo["rho_r"]) / rho_o)
    return e_rho, e_u, e_col


def u_inf_error(fo, fg):
    """u error relative to ||u_oracle||_inf alone (no velocity-scale floor)."""
    umax = max(np.abs(fo["ux"]).max(), np.abs(fo["uy"]).max())
    return max(np.abs(fg["ux"] - fo["ux"]).max(), np.abs(fg["uy"] - fo["uy"]).max()) / umax


@pytest.fixture(scope="module")
def fp32_oracle(tmp_path_factory):
    """The oracle source compiled with an FP32 arithmetic type."""
    return O.fp32_library(str(tmp_path_factory.mktemp("oracle_fp32")))


def oracle_fields(nx, ny, fields, steps, kw, library=None):
    o = O.Oracle(_oracle_params(nx, ny, kw), library)
    o.init_fields(*fields)
    o.step(steps)
    return o.fields()


CASES = {
    # name: (nx, ny, params, field recipe, u_ref)
    "bubble64_bgk": (64, 64, dict(gamma=1.0, tau_r=1.0, tau_b=1.0, sigma=0.005, beta=0.7),
                     lambda: W.bubble_fields(64, 64, 32, 32, 16, 1.0), 0.005 / (1.0 / 6.0)),
    "random_ragged_mrt_hermite": (200, 37, dict(gamma=10.0, tau_r=0.6, tau_b=1.1, sigma=0.01, beta=0.7,
                                                collision=L.LBM_MRT, equilibrium=L.LBM_EQ_HERMITE,
                                                gx=2e-6, gy=-1e-6),
                                  lambda: W.random_fields(200, 37, seed=11, gamma=10.0, u_amp=0.03), 0.03),
    "walls_bgk_gravity": (136, 24, dict(gamma=5.0, tau_r=0.7, tau_b=0.9, sigma=0.005, beta=0.99,
                                        bc_y=L.LBM_BC_WALL, gx=1e-5),
                          lambda: W.random_fields(136, 24, seed=12, gamma=5.0, u_amp=0.02, walls_y=True), 0.02),
    "walls_mrt_hermite": (96, 33, dict(gamma=10.0, tau_r=0.55, tau_b=1.0, sigma=0.01, beta=0.7,
                                       collision=L.LBM_MRT, equilibrium=L.LBM_EQ_HERMITE,
                                       bc_y=L.LBM_BC_WALL, gx=5e-6),
                          lambda: W.random_fields(96, 33, seed=13, gamma=10.0, u_amp=0.02, walls_y=True), 0.02),
    "inout_alternating": (160, 32, dict(gamma=5.0, tau_r=0.6, tau_b=0.6, sigma=1e-3, beta=0.7,
                                        bc_x=L.LBM_BC_INOUT, bc_y=L.LBM_BC_WALL, u_in_r=0.0125,
                                        u_in_b=0.075, p_out=0.48, inlet_period_r=30, inlet_period_b=20),
                          lambda: W.slug_fields(160, 32, 5.0, 1, 40.0, 16.0), 0.075),
    "inout_layered_hermite": (144, 20, dict(gamma=3.0, tau_r=0.7, tau_b=0.8, sigma=2e-3, beta=0.7,
                                            collision=L.LBM_MRT, equilibrium=L.LBM_EQ_HERMITE,
                                            bc_x=L.LBM_BC_INOUT, bc_y=L.LBM_BC_WALL, u_in_r=0.01,
                                            u_in_b=0.06, p_out=0.5, inlet_mode=L.LBM_INLET_LAYERED,
                                            inlet_layer=10),
                              lambda: W.random_fields(144, 20, seed=14, gamma=3.0, u_amp=0.01, walls_y=True), 0.06),
    "tiny_8x4": (8, 4, dict(gamma=2.0, tau_r=0.8, tau_b=0.8, sigma=0.01, beta=0.7),
                 lambda: W.random_fields(8, 4, seed=15, gamma=2.0, n_bubbles=1, rmin=1.0, rmax=2.0, u_amp=0.02),
                 0.02),
    "odd_37x17_walls": (37, 17, dict(gamma=1.0, tau_r=0.9, tau_b=0.6, sigma=0.005, beta=0.7,
                                     bc_y=L.LBM_BC_WALL, gy=-2e-6),
                        lambda: W.random_fields(37, 17, seed=16, gamma=1.0, u_amp=0.02, walls_y=True), 0.02),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("kernel", [L.LBM_KERNEL_FUSED, L.LBM_KERNEL_TWOPASS])
def test_parity_100_steps(name, kernel, fp32_oracle):
    nx, ny, kw, make, u_ref = CASES[name]
    f = make()
    fo, fg = run_pair(nx, ny, f, 100, kernel=kernel, **kw)
    f32 = oracle_fields(nx, ny, f, 100, kw, fp32_oracle)
    e_rho, e_u, e_col = errors(fo, fg, u_ref)
    e_ui = u_inf_error(fo, fg)
    F_rho, F_u, F_col = errors(fo, f32, u_ref)
    F_ui = u_inf_error(fo, f32)
    bar = lambda F: max(RTOL, 2.0 * F)
    print(f"{name} kernel={kernel}: rho {e_rho:.2e} (floor {F_rho:.2e})  u {e_u:.2e} (floor {F_u:.2e})  "
          f"u/|u|inf {e_ui:.2e} (floor {F_ui:.2e}, |u|inf {max(np.abs(fo['ux']).max(), np.abs(fo['uy']).max()):.2e}, "
          f"U_ref {u_ref:.2e})  colour {e_col:.2e} (floor {F_col:.2e})")
    assert np.all(np.isfinite(fg["rho_r"]))
    assert e_rho <= bar(F_rho) and e_u <= bar(F_u)
    assert e_ui <= bar(F_ui) and e_col <= bar(F_col)


def _state_after(nx, ny, fields, steps, **kw):
    with L.Simulation(nx, ny, **kw) as s:
        s.init_fields(*fields)
        s.step(steps)
        s.synchronize()
        return s.save_state()


@pytest.mark.parametrize("name", ["random_ragged_mrt_hermite", "walls_mrt_hermite", "inout_alternating"])
def test_fused_and_twopass_agree(name):
    """The fused single-pass kernel and the two-pass kernel pair run the same node
    code; they differ only by the compiler's floating-point contraction (FMA)
    choices, which the interface dynamics amplify, so after 37 steps they agree
    within half the oracle tolerance."""
    nx, ny, kw, make, u_ref = CASES[name]
    f = make()
    out = []
    for kernel in (L.LBM_KERNEL_FUSED, L.LBM_KERNEL_TWOPASS):
        with L.Simulation(nx, ny, kernel=kernel, **_gpu_params(kw)) as s:
            s.init_fields(*f)
            s.step(37)
            out.append(s.fields())
    e_rho, e_u, e_col = errors(out[1], out[0], u_ref)
    print(f"fused vs two-pass {name}: rho {e_rho:.2e} u {e_u:.2e} colour {e_col:.2e}")
    assert e_rho <= RTOL / 2 and e_u <= RTOL / 2 and e_col <= RTOL / 2


def test_graph_and_direct_stepping_agree_and_resume_is_exact():
    nx, ny, kw, make, _ = CASES["walls_bgk_gravity"]
    f = make()
    with L.Simulation(nx, ny, **_gpu_params(kw)) as s:
        s.init_fields(*f)
        s.step(70)                     # two graph chunks + direct remainder
        ref = s.save_state()
    with L.Simulation(nx, ny, **_gpu_params(kw)) as s:
        s.init_fields(*f)
        for _ in range(7):
            s.step(10)                 # direct launches only
        assert s.save_state() == ref
    with L.Simulation(nx, ny, **_gpu_params(kw)) as s:
        s.init_fields(*f)
        s.step(33)
        mid = s.save_state()
    with L.Simulation(nx, ny, **_gpu_params(kw)) as s2:
        s2.load_state(mid)
        assert s2.t == 33
        s2.step(37)
        assert s2.save_state() == ref


def test_batch_equals_alone():
    """Simulations of different sizes and parameters advanced in one batched launch
    per step give bit-identical states to the same simulations advanced alone."""
    names = ["random_ragged_mrt_hermite", "walls_bgk_gravity", "inout_alternating", "tiny_8x4"]
    alone = []
    for nm in names:
        nx, ny, kw, make, _ = CASES[nm]
        alone.append(_state_after(nx, ny, make(), 45, **_gpu_params(kw)))
    sims = []
    for nm in names:
        nx, ny, kw, make, _ = CASES[nm]
        s = L.Simulation(nx, ny, **_gpu_params(kw))
        s.init_fields(*make())
        sims.append(s)
    b = L.Batch(sims, rows_per_item=8)
    b.step(20, use_graph=True)
    b.step(20, use_graph=True)
    b.step(5, use_graph=False)
    for s, ref in zip(sims, alone):
        assert s.t == 45
        assert s.save_state() == ref
    b.close()
    for s in sims:
        s.close()


def test_stop_times_in_a_batch():
    """Members of one batch stopped at different times end exactly where the same
    simulations stepped alone to those times end, bit for bit, and stay there."""
    names = ["random_ragged_mrt_hermite", "walls_bgk_gravity", "tiny_8x4"]
    stops = [13, 40, 27]
    alone = []
    for nm, te in zip(names, stops):
        nx, ny, kw, make, _ = CASES[nm]
        alone.append(_state_after(nx, ny, make(), te, **_gpu_params(kw)))
    sims = []
    for nm, te in zip(names, stops):
        nx, ny, kw, make, _ = CASES[nm]
        s = L.Simulation(nx, ny, **_gpu_params(kw))
        s.init_fields(*make())
        s.set_stop(te)
        sims.append(s)
    b = L.Batch(sims)
    b.step(32, use_graph=True)
    b.step(32, use_graph=True)
    for s, te, ref in zip(sims, stops, alone):
        assert s.t == te
        assert s.save_state() == ref
    b.close()
    for s in sims:
        s.close()


def test_stop_times_changed_after_the_batch_was_built():
    """A stop time set on a member between two batch steps takes effect in the
    batch (its device descriptor follows the member): the member ends at the new
    stop, bit for bit where it ends alone, while the others run on; lifting the
    stop lets it continue."""
    names = ["random_ragged_mrt_hermite", "walls_bgk_gravity"]
    sims = []
    for nm in names:
        nx, ny, kw, make, _ = CASES[nm]
        s = L.Simulation(nx, ny, **_gpu_params(kw))
        s.init_fields(*make())
        sims.append(s)
    b = L.Batch(sims)
    b.step(16, use_graph=True)
    sims[0].set_stop(16 + 5)
    b.step(16, use_graph=True)
    assert sims[0].t == 21 and sims[1].t == 32
    nx, ny, kw, make, _ = CASES[names[0]]
    assert sims[0].save_state() == _state_after(nx, ny, make(), 21, **_gpu_params(kw))
    sims[0].set_stop(-1)
    b.step(11, use_graph=False)
    assert sims[0].t == 32 and sims[1].t == 43
    assert sims[0].save_state() == _state_after(nx, ny, make(), 32, **_gpu_params(kw))
    nx, ny, kw, make, _ = CASES[names[1]]
    assert sims[1].save_state() == _state_after(nx, ny, make(), 43, **_gpu_params(kw))
    b.close()
    for s in sims:
        s.close()


def test_diagnostics_match_oracle_sums():
    nx, ny, kw, make, _ = CASES["walls_mrt_hermite"]
    f = make()
    o = O.Oracle(_oracle_params(nx, ny, kw))
    o.init_fields(*f)
    o.step(60)
    fo = o.fields()
    with L.Simulation(nx, ny, **_gpu_params(kw)) as s:
        s.init_fields(*f)
        s.step(60)
        d = s.diagnostics()
    rho = fo["rho_r"] + fo["rho_b"]
    assert d["t"] == 60
    assert abs(d["mass_r"] - fo["rho_r"].sum()) <= 1e-5 * fo["rho_r"].sum()
    assert abs(d["mass_b"] - fo["rho_b"].sum()) <= 1e-5 * fo["rho_b"].sum()
    umax = np.hypot(fo["ux"], fo["uy"]).max()
    assert abs(d["max_u"] - umax) <= 1e-5 * umax
    mx = (rho * fo["ux"]).sum()
    assert abs(d["mom_x"] - mx) <= 1e-5 * np.abs(rho * fo["ux"]).sum()
    area = ((1 - fo["psi"]) / 2).sum()
    assert abs(d["area_b"] - area) <= 1e-4 * area
    assert d["nonfinite"] == 0


def test_gpu_colour_mass_conservation_2000_steps():
    """Per-colour mass is conserved by every operator; in FP32 the drift after
    2000 steps stays at round-off level."""
    with L.Simulation(64, 64, gamma=1.0, sigma=0.005, beta=0.7) as s:
        s.init_bubble(32, 32, 16)
        d0 = s.diagnostics()
        s.step(2000)
        d1 = s.diagnostics()
    assert abs(d1["mass_r"] - d0["mass_r"]) <= 2e-5 * d0["mass_r"]
    assert abs(d1["mass_b"] - d0["mass_b"]) <= 2e-5 * d0["mass_b"]


def test_laplace_pressure_gpu_vs_oracle():
    """64^2 static bubble, 2000 steps: the GPU Laplace jump matches the oracle's
    within 1% and the Laplace law sigma / R_eff within 6%."""
    o = _bubble_oracle()
    fo = o.fields()
    dp_o, R_o = W.laplace_pressure_jump(fo["p"], fo["psi"], 32, 32)
    with L.Simulation(64, 64, gamma=1.0, tau_r=1.0, tau_b=1.0, sigma=0.005, beta=0.7) as s:
        s.init_bubble(32, 32, 16)
        s.step(2000)
        d = s.diagnostics()
    assert abs(d["dp"] - dp_o) <= 0.01 * abs(dp_o)
    assert abs(d["r_eff"] - R_o) <= 0.01 * R_o
    assert abs(d["dp"] * d["r_eff"] / 0.005 - 1.0) <= 0.06


def _bubble_oracle():
    o = O.Oracle(O.OracleParams(nx=64, ny=64, gamma=1.0, tau_r=1.0, tau_b=1.0, sigma=0.005, beta=0.7))
    o.init_fields(*W.bubble_fields(64, 64, 32, 32, 16, 1.0))
    o.step(2000)
    return o


def test_full_size_laplace_batch_sampled_parity(fp32_oracle):
    """The launch configuration the benchmark times (the 40-run 256^2 Laplace sweep
    as one batch, one launch per step, graph-captured): after 100 steps two
    sampled runs match the oracle run alone at full size (bars as in
    test_parity_100_steps, the FP32 floor from the FP32-compiled oracle)."""
    specs = W.laplace_sweep(256, steps=100)
    sims = []
    for sp in specs:
        s = L.Simulation(sp.nx, sp.ny, gamma=sp.gamma, tau_r=sp.tau_r, tau_b=sp.tau_b, sigma=sp.sigma,
                         beta=sp.beta)
        s.init_bubble(*sp.bubble)
        sims.append(s)
    b = L.Batch(sims)
    b.step(100, use_graph=True)
    for idx in (3, 38):
        sp = specs[idx]
        kw = dict(gamma=sp.gamma, tau_r=sp.tau_r, tau_b=sp.tau_b, sigma=sp.sigma, beta=sp.beta)
        f = W.bubble_fields(256, 256, *sp.bubble, sp.gamma)
        fo = oracle_fields(256, 256, f, 100, kw)
        f32 = oracle_fields(256, 256, f, 100, kw, fp32_oracle)
        fg = sims[idx].fields()
        nu = min(sp.tau_r, sp.tau_b) / 3 - 1 / 6
        e_rho, e_u, _ = errors(fo, fg, sp.sigma / nu)
        F_rho, F_u, _ = errors(fo, f32, sp.sigma / nu)
        e_ui, F_ui = u_inf_error(fo, fg), u_inf_error(fo, f32)
        print(f"sweep[{idx}] rho {e_rho:.2e} (floor {F_rho:.2e}) u {e_u:.2e} (floor {F_u:.2e}) "
              f"u/|u|inf {e_ui:.2e} (floor {F_ui:.2e})")
        assert e_rho <= max(RTOL, 2 * F_rho) and e_u <= max(RTOL, 2 * F_u)
        assert e_ui <= max(RTOL, 2 * F_ui)
    b.close()
    for s in sims:
        s.close()


def test_invalid_arguments_rejected():
    with pytest.raises(L.LBMError) as e:
        L.Simulation(4, 4)
    assert e.value.status == L.LBM_EINVAL
    with pytest.raises(L.LBMError):
        L.Simulation(64, 64, tau_r=0.5)
    with L.Simulation(16, 8) as s:
        with pytest.raises(L.LBMError):
            s.step(-1)
        with pytest.raises(L.LBMError):
            s.load_state(b"\0" * 8)
