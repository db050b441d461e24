"""Host-side pieces of the autotuner: size classes and the cached table."""
import json

from paper_1903_01168_gb300 import autotune as A


def test_size_class_rounds_up_to_powers_of_two():
    assert A.size_class(300, 200) == "s0-c0-e0-x512-y256"
    assert A.size_class(256, 256, storage=1) == "s1-c0-e0-x256-y256"
    assert A.size_class(257, 64, collision=1, equilibrium=1) == "s0-c1-e1-x512-y64"
    assert A.class_of(96, 64, {"storage": 2}) == "s2-c0-e0-x128-y64"


def test_params_for_uses_the_table(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({"single-s0-c0-e0-x512-y256": {"kernel": 2, "plan_rows": 0, "ms": 1.0},
                                "batch-s0-c0-e0-x512-y256": {"kernel": 1, "plan_rows": 32, "ms": 1.0}}))
    t = A.Autotuner(cache_path=str(path))
    assert t.params_for(300, 200, False, gamma=10.0) == {"gamma": 10.0, "kernel": 2, "plan_rows": 0}
    assert t.params_for(300, 200, True, gamma=10.0) == {"gamma": 10.0, "plan_rows": 32}
    # an untuned class is left alone
    assert t.params_for(64, 64, True, gamma=1.0) == {"gamma": 1.0}
    t.save()
    assert json.loads(path.read_text()) == t.table
