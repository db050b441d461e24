"""Serving loop on the GPU: requests of different sizes, boundary conditions and
storage types arrive while others run, are admitted into the running batch, and
each result equals the same request run alone (the batched launch runs the same
kernel code per simulation, so equality is exact up to the FP64 reduction order of
the diagnostics, which is deterministic)."""
import pytest

from paper_1903_01168_gb300 import lbm as L
from paper_1903_01168_gb300 import serving as S
from paper_1903_01168_gb300.workloads import SimSpec

pytestmark = pytest.mark.gpu


def _trace():
    inout = dict(gamma=5.0, tau_r=0.6, tau_b=0.6, sigma=1e-3, beta=0.7, bc_x=2, bc_y=1, geometry="inout",
                 u_in_r=0.0125, u_in_b=0.075, p_out=0.48, inlet_period_r=60, inlet_period_b=40)
    return [
        (0.00, SimSpec(nx=256, ny=32, steps=400, storage=0, **inout)),
        (0.00, SimSpec(nx=160, ny=64, steps=250, storage=1, **inout)),
        (0.05, SimSpec(nx=96, ny=48, gamma=10.0, tau_r=0.8, tau_b=0.8, sigma=0.01, beta=0.7,
                       geometry="bubble", bubble=(48.0, 24.0, 12.0), steps=300, storage=0)),
        (0.10, SimSpec(nx=384, ny=32, steps=150, storage=2, **inout)),
        (0.15, SimSpec(nx=128, ny=64, gamma=10.0, tau_r=0.55, tau_b=0.7, sigma=2e-4, beta=0.7, gx=2e-6, bc_y=1,
                       geometry="slug", slug=(1, 64.0, 32.0), steps=333, storage=0)),
    ]


@pytest.mark.parametrize("max_active_nodes", [4_000_000, 20_000])
def test_each_result_is_the_same_alone_and_in_the_mix(max_active_nodes):
    """Every request's diagnostics equal those of the same simulation run alone,
    whether all requests share the GPU or the node cap admits them a few at a time."""
    L.load(build_if_missing=True)
    trace = _trace()
    results, stats = S.Server(budget_bytes=2e9, chunk=64, max_active_nodes=max_active_nodes).run(trace)
    assert stats["requests"] == len(trace)
    for r, (_, spec) in zip(results, trace):
        with S.start_simulation(spec) as s:
            s.step(spec.steps)
            d = s.diagnostics(allow_unstable=True)
        assert r.diag["t"] == spec.steps == d["t"]
        for k in ("mass_r", "mass_b", "mom_x", "mom_y", "max_u", "area_b", "ux_b"):
            assert r.diag[k] == d[k], (r.rid, k, r.diag[k], d[k])
        assert r.diag["nonfinite"] == 0


def test_budget_limits_residency():
    """With a budget that holds only the largest request at a time, requests run one
    after another but still complete with the same results."""
    L.load(build_if_missing=True)
    trace = _trace()[:2]
    need = max(S.state_bytes(sp) for _, sp in trace)
    results, stats = S.Server(budget_bytes=need, chunk=64).run(trace)
    assert stats["requests"] == 2
    assert results[1].admitted >= results[0].finished - 1e-9 or results[0].admitted >= results[1].finished - 1e-9


def test_a_request_that_goes_non_finite_is_retired_as_failed():
    """A physically unstable request (tau = 0.51 with the inlet at 0.1: the flow
    blows up within a few hundred steps, in the method itself, without any fault)
    is retired at the first check after its state goes non-finite, with the steps
    it ran; the requests beside it finish with the results they have alone."""
    L.load(build_if_missing=True)
    good = _trace()[:2]
    (_, sp0), (_, sp1) = good
    bad = SimSpec(**{**sp0.as_dict(), "nx": 256, "ny": 64, "tau_r": 0.51, "tau_b": 0.51, "u_in_r": 0.1,
                     "u_in_b": 0.1, "steps": 3000})
    trace = [(0.0, sp0), (0.0, bad), (0.0, sp1)]
    results, stats = S.Server(budget_bytes=2e9, chunk=64, max_chunk=500).run(trace)
    by = {r.rid: r for r in results}
    assert stats["failed"] == 1 and by[1].failed
    assert 0 < by[1].steps < bad.steps and by[1].diag["nonfinite"] > 0
    for rid, spec in ((0, sp0), (2, sp1)):
        r = by[rid]
        assert not r.failed and r.steps == spec.steps
        with S.start_simulation(spec) as s:
            s.step(spec.steps)
            d = s.diagnostics()
        for k in ("mass_r", "mass_b", "mom_x", "mom_y", "max_u", "area_b", "ux_b"):
            assert r.diag[k] == d[k], (rid, k, r.diag[k], d[k])
    # the sequential baseline applies the same check
    seq, st = S.run_sequential(trace, check_every=500)
    assert st["failed"] == 1 and seq[1].failed and seq[1].steps < bad.steps
