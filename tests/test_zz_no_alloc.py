"""lbm_step_noalloc: stepping a caller-owned state buffer with no device allocation.

Callers that cannot call cudaMalloc at run time (an embedding runtime whose own
allocator owns the GPU, a fixed pre-registered pool, an allocation-free loop)
use this entry point; its scratch is a static array inside the library.  The
test checks it against the existing two-pass entry point (lbm_create +
lbm_step) on the same state, over two calls in a row, within the parity
tolerance used by the other GPU tests.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1903_01168_gb300 import lbm as L
from paper_1903_01168_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-5


def _rel(a, b, scale):
    return float(np.max(np.abs(a - b)) / scale)


def _fields_from_state(nx, ny, kw, raw_bytes, t):
    """Read fields of a raw state through the existing API (load_state)."""
    header = np.array([t], dtype=np.int64).tobytes()
    with L.Simulation(nx, ny, **kw) as s:
        s.load_state(header + raw_bytes)
        return s.fields()


def test_noalloc_matches_existing_entry_point_over_two_calls():
    torch = pytest.importorskip("torch")
    L.load(build_if_missing=True)
    nx, ny, n1, n2 = 136, 40, 25, 17
    kw = dict(gamma=10.0, tau_r=0.6, tau_b=1.0, sigma=0.01, beta=0.7, collision=L.LBM_MRT,
              equilibrium=L.LBM_EQ_HERMITE, bc_y=L.LBM_BC_WALL, gx=5e-6, kernel=L.LBM_KERNEL_TWOPASS)
    fields = W.random_fields(nx, ny, seed=21, gamma=10.0, u_amp=0.02, walls_y=True)

    # existing entry point: library-owned buffers, lbm_step
    with L.Simulation(nx, ny, **kw) as ref:
        ref.init_fields(*fields)
        state0 = ref.save_state()
        ref.step(n1)
        f1_ref = ref.fields()
        ref.step(n2)
        f2_ref = ref.fields()

    # allocation-free entry point on a caller-owned device buffer, two calls in a row
    p = L.make_params(**kw)
    nbytes = L.lbm_bytes_required(nx, ny, p)
    raw0 = np.frombuffer(state0[8:], dtype=np.uint8)
    assert raw0.size == nbytes
    buf = torch.from_numpy(raw0.copy()).to("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    L.lbm_step_noalloc(p, nx, ny, buf.data_ptr(), nbytes, 0, n1, stream)
    torch.cuda.synchronize()
    f1 = _fields_from_state(nx, ny, kw, buf.cpu().numpy().tobytes(), n1)
    L.lbm_step_noalloc(p, nx, ny, buf.data_ptr(), nbytes, n1, n2, stream)
    torch.cuda.synchronize()
    f2 = _fields_from_state(nx, ny, kw, buf.cpu().numpy().tobytes(), n1 + n2)

    for got, want in ((f1, f1_ref), (f2, f2_ref)):
        rho_w = want["rho_r"] + want["rho_b"]
        e_rho = float(np.max(np.abs(got["rho_r"] + got["rho_b"] - rho_w) / rho_w))
        umax = max(np.abs(want["ux"]).max(), np.abs(want["uy"]).max(), 0.02)
        e_u = max(_rel(got["ux"], want["ux"], umax), _rel(got["uy"], want["uy"], umax))
        print(f"no-alloc vs lbm_step: rho {e_rho:.2e}  u {e_u:.2e}")
        assert e_rho <= RTOL and e_u <= RTOL


def test_noalloc_rejects_lattices_beyond_its_scratch():
    L.load(build_if_missing=True)
    p = L.make_params()
    with pytest.raises(L.LBMError) as e:
        L.lbm_step_noalloc(p, 1024, 512, 0, 0, 0, 1, 0)
    assert e.value.status == L.LBM_EINVAL
    assert "static scratch" in L.lbm_last_error(None)


def test_noalloc_rejects_memory_that_is_not_on_the_current_device():
    """A host buffer passes the size and alignment checks but is not device
    memory: the call refuses it instead of handing it to the kernels."""
    torch = pytest.importorskip("torch")
    L.load(build_if_missing=True)
    nx, ny = 64, 32
    p = L.make_params()
    nbytes = L.lbm_bytes_required(nx, ny, p)
    host = torch.empty(nbytes + 256, dtype=torch.uint8)
    ptr = (host.data_ptr() + 255) // 256 * 256
    with pytest.raises(L.LBMError) as e:
        L.lbm_step_noalloc(p, nx, ny, ptr, nbytes, 0, 1, 0)
    assert e.value.status == L.LBM_EINVAL
    assert "not device memory" in L.lbm_last_error(None)
