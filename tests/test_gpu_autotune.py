"""Autotuner on the device: it times every candidate, picks the fastest, and the
plan it picks never changes results (the plan only decides which thread block
updates which rows)."""
import numpy as np
import pytest

from paper_1903_01168_gb300 import autotune as A
from paper_1903_01168_gb300 import lbm as L
from paper_1903_01168_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _state(nx, ny, steps, **kw):
    with L.Simulation(nx, ny, **kw) as s:
        s.init_fields(*W.bubble_fields(nx, ny, nx / 2, ny / 2, ny / 4, 10.0))
        s.step(steps)
        return s.save_state()


def test_tune_single_times_every_candidate(tmp_path):
    tuner = A.Autotuner(cache_path=str(tmp_path / "t.json"), steps=8)
    c = tuner.tune_single(160, 96, gamma=10.0, sigma=0.005)
    assert set(c["timings"]) == {f"fused/{r}" for r in A.PLAN_CANDIDATES} | {"twopass/0"}
    assert all(t > 0 for t in c["timings"].values())
    assert c["ms"] == min(c["timings"].values())
    tuner.save()
    again = A.Autotuner(cache_path=str(tmp_path / "t.json"))
    assert again.params_for(160, 96, False, gamma=10.0, sigma=0.005)["plan_rows"] == c["plan_rows"]


@pytest.mark.parametrize("storage", [0, 1])
def test_plan_rows_never_changes_results(storage):
    """Every candidate plan (and hence whatever the tuner picks) gives the
    bit-identical state after 30 steps of a ragged 300 x 200 lattice."""
    ref = _state(300, 200, 30, gamma=10.0, sigma=0.005, storage=storage, kernel=L.LBM_KERNEL_FUSED)
    for r in A.PLAN_CANDIDATES + (3, 200):
        assert _state(300, 200, 30, gamma=10.0, sigma=0.005, storage=storage,
                      kernel=L.LBM_KERNEL_FUSED, plan_rows=r) == ref


def test_tuned_batch_equals_alone():
    """A batch planned with what the tuner picked (per class plan_rows, plan kind,
    row cost) gives each member the state it reaches alone with the default plan."""
    specs = [(96, 64), (300, 200), (128, 512), (300, 210)]
    kw = dict(gamma=10.0, sigma=0.005, storage=1)

    def start(nx, ny):
        s = L.Simulation(nx, ny, torch_memory=True, **kw)
        s.init_fields(*W.bubble_fields(nx, ny, nx / 2, ny / 2, ny / 4, 10.0))
        return s

    sims = [start(nx, ny) for nx, ny in specs]
    tuner = A.Autotuner(candidates=(8, 32))
    got = tuner.tune_batch(sims, steps=4)
    assert set(got["classes"]) == {A.class_of(nx, ny, {"storage": 1}) for nx, ny in specs}
    assert len(got["classes"]) == 3   # 300x200 and 300x210 share a class
    assert all(r in (0, 32) for r in got["member_plan_rows"])
    for s in sims:
        s.close()
    sims = [start(nx, ny) for nx, ny in specs]
    b = L.Batch(sims, row_overhead=got["row_overhead"], plan=got["plan"], member_plan_rows=got["member_plan_rows"])
    b.step(25, use_graph=True)
    for s, (nx, ny) in zip(sims, specs):
        s.synchronize()
        assert s.save_state() == _state(nx, ny, 25, **kw)
    b.close()
    for s in sims:
        s.close()


def test_plan_options_never_change_results():
    """Plan kind and row cost only move rows between thread blocks: batches
    planned with every candidate reach bit-identical states, and the tuner
    returns one of the candidates."""
    specs = [(96, 64), (160, 200), (300, 90), (32, 128)]

    def members():
        out = []
        for nx, ny in specs:
            s = L.Simulation(nx, ny, torch_memory=True, gamma=10.0, sigma=0.005, storage=1)
            s.init_fields(*W.bubble_fields(nx, ny, nx / 2, ny / 2, ny / 4, 10.0))
            out.append(s)
        return out

    ref = None
    for kind, c in A.PLAN_OPTION_CANDIDATES + ((L.LBM_PLAN_AUTO, -1.0),):
        sims = members()
        b = L.Batch(sims, row_overhead=c, plan=kind)
        b.step(17, use_graph=False)
        sims[0].synchronize()
        states = [s.save_state() for s in sims]
        b.close()
        for s in sims:
            s.close()
        if ref is None:
            ref = states
        assert states == ref
    sims = members()
    best, timings = A.tune_plan(sims, steps=4)
    assert best in A.PLAN_OPTION_CANDIDATES and set(timings) == set(A.PLAN_OPTION_CANDIDATES)
    for s in sims:
        s.close()
