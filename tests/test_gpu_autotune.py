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
    """A batch whose members carry the tuned plan_rows of their size classes gives
    each member the state it reaches alone with the default plan."""
    specs = [(96, 64), (300, 200), (128, 512), (300, 210)]
    members = [(nx, ny, dict(gamma=10.0, sigma=0.005, storage=1)) for nx, ny in specs]
    tuner = A.Autotuner(steps=6, candidates=(8, 32))
    table = tuner.tune_batch(members)
    assert len(table) == 3   # 300x200 and 300x210 share a class
    sims = []
    for nx, ny, kw in members:
        s = L.Simulation(nx, ny, **tuner.params_for(nx, ny, True, **kw))
        s.init_fields(*W.bubble_fields(nx, ny, nx / 2, ny / 2, ny / 4, 10.0))
        sims.append(s)
    b = L.Batch(sims)
    b.step(25, use_graph=True)
    for s, (nx, ny, kw) in zip(sims, members):
        s.synchronize()
        assert s.save_state() == _state(nx, ny, 25, **kw)
    b.close()
    for s in sims:
        s.close()


def test_row_overhead_never_changes_results():
    """The planner's row cost only moves rows between thread blocks: batches
    planned with every candidate cost reach bit-identical states, and the tuner
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
    for c in A.ROW_OVERHEAD_CANDIDATES:
        sims = members()
        b = L.Batch(sims, row_overhead=c)
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
    best, timings = A.tune_row_overhead(sims, steps=4)
    assert best in A.ROW_OVERHEAD_CANDIDATES and set(timings) == set(A.ROW_OVERHEAD_CANDIDATES)
    for s in sims:
        s.close()
