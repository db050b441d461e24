"""Failure detection without a GPU fault: the failure is made on the host (a NaN
written into one simulation's state and copied to the device), detected by the
FP64 diagnostics (LBM_EUNSTABLE), and a failed member of a batch is evicted while
every other member goes on exactly as if nothing had happened."""
import numpy as np
import pytest

from paper_1903_01168_gb300 import lbm as L
from paper_1903_01168_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GHOST = 8   # ghost columns on each side of a stored row


@pytest.fixture(scope="module", autouse=True)
def _native():
    L.load(build_if_missing=True)


def _with_nan(state: bytes, nx: int, ny: int, t: int) -> bytes:
    """The saved state with both colour densities of every node of row ny/2 of the
    buffer that step t reads set to NaN.  Raw state: an 8-byte time stamp, then the
    FP32 density planes laid out [buffer][row][colour][pitch] with the ghost columns
    in front (pitch = nx + 2 ghosts rounded up to 4 floats)."""
    pitch = (nx + 2 * GHOST + 3) // 4 * 4
    raw = bytearray(state)
    dens = np.frombuffer(raw, dtype=np.float32, count=2 * ny * 2 * pitch, offset=8).reshape(2, ny, 2, pitch)
    dens = dens.copy()
    dens[t & 1, ny // 2, :, GHOST:GHOST + nx] = np.nan
    raw[8:8 + dens.nbytes] = dens.tobytes()
    return bytes(raw)


def test_nan_written_from_the_host_is_reported_unstable():
    nx, ny = 64, 32
    with L.Simulation(nx, ny, gamma=1.0, sigma=0.005, beta=0.7) as s:
        s.init_bubble(32, 16, 8)
        s.step(10)
        assert s.diagnostics()["nonfinite"] == 0
        s.load_state(_with_nan(s.save_state(), nx, ny, s.t))
        with pytest.raises(L.LBMError) as e:
            s.diagnostics()
        assert e.value.status == L.LBM_EUNSTABLE
        assert "non-finite" in L.lbm_last_error(s.h)
        s.step(5)                      # stepping a broken state is allowed and stays broken
        d = s.diagnostics(allow_unstable=True)
        assert d["status"] == L.LBM_EUNSTABLE and d["nonfinite"] > 0


def _members():
    specs = [(96, 48, dict(gamma=10.0, tau_r=0.8, tau_b=0.8, sigma=0.01, beta=0.7), (48.0, 24.0, 12.0)),
             (64, 32, dict(gamma=1.0, tau_r=1.0, tau_b=1.0, sigma=0.005, beta=0.7), (32.0, 16.0, 8.0)),
             (160, 64, dict(gamma=5.0, tau_r=0.7, tau_b=0.9, sigma=0.005, beta=0.99), (80.0, 32.0, 16.0)),
             (128, 40, dict(gamma=2.0, tau_r=0.8, tau_b=0.8, sigma=0.01, beta=0.7, storage=L.LBM_F16DEV),
              (64.0, 20.0, 10.0))]
    sims = []
    for nx, ny, kw, bub in specs:
        s = L.Simulation(nx, ny, **kw)
        s.init_bubble(*bub)
        sims.append(s)
    return specs, sims


def test_failed_batch_member_is_evicted_and_the_others_are_untouched():
    # reference: the same four simulations, never injected, 30 steps in one batch
    _, ref = _members()
    b = L.Batch(ref)
    b.step(30, use_graph=True)
    b.close()
    want = [s.save_state() for s in ref]
    for s in ref:
        s.close()

    specs, sims = _members()
    b = L.Batch(sims)
    b.step(10, use_graph=True)
    b.close()
    bad = 2
    nx, ny = specs[bad][0], specs[bad][1]
    sims[bad].load_state(_with_nan(sims[bad].save_state(), nx, ny, sims[bad].t))
    b = L.Batch(sims)
    b.step(10, use_graph=True)
    b.close()
    status = [s.diagnostics(allow_unstable=True)["status"] for s in sims]
    assert status == [L.LBM_OK, L.LBM_OK, L.LBM_EUNSTABLE, L.LBM_OK]
    # evict the failed member; the others go on in a new batch
    keep = [s for i, s in enumerate(sims) if status[i] == L.LBM_OK]
    b = L.Batch(keep)
    b.step(10, use_graph=True)
    b.close()
    for i, s in enumerate(sims):
        if i == bad:
            continue
        assert s.t == 30
        assert s.save_state() == want[i], i
    for s in sims:
        s.close()
