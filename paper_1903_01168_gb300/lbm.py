"""Python binding of the C ABI in include/lbm.h (argument marshalling only).

Every function named ``lbm_*`` here calls the C function of the same name in
``_native/liblbm_gb300.so``; all lattice work runs in that library's CUDA
kernels.  There is no CPU fallback: importing this module on a machine without
the built library raises, and the library reports an error when no CUDA device
is present.

``Simulation`` and ``Batch`` are thin conveniences over those calls.  With
``torch_memory=True`` the population buffers are a torch tensor on the current
device and the library runs on torch's current stream (``lbm_create_ex``).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, fields

import numpy as np

from . import build as _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_EBUDGET = 0, -1, -2, -3, -4, -5, -6
LBM_BGK, LBM_MRT = 0, 1
LBM_EQ_STD, LBM_EQ_HERMITE = 0, 1
LBM_F32, LBM_F16DEV, LBM_BF16DEV = 0, 1, 2
LBM_BC_PERIODIC, LBM_BC_WALL, LBM_BC_INOUT = 0, 1, 2
LBM_INLET_ALTERNATE, LBM_INLET_LAYERED = 0, 1
LBM_KERNEL_AUTO, LBM_KERNEL_FUSED, LBM_KERNEL_TWOPASS = 0, 1, 2

_STATUS = {0: "LBM_OK", -1: "LBM_EINVAL", -2: "LBM_ENOMEM", -3: "LBM_ECUDA", -4: "LBM_EUNSTABLE",
           -5: "LBM_ETIMEOUT", -6: "LBM_EBUDGET"}

# The C functions every build exports (declared in include/lbm.h).
ABI_SYMBOLS = (
    "lbm_default_params", "lbm_bytes_required", "lbm_create", "lbm_create_ex", "lbm_init_bubble",
    "lbm_init_slug", "lbm_init_fields", "lbm_init_populations", "lbm_step", "lbm_set_stop",
    "lbm_synchronize", "lbm_time", "lbm_read_fields", "lbm_read_populations",
    "lbm_diagnostics", "lbm_state_bytes", "lbm_save_state", "lbm_load_state", "lbm_last_error",
    "lbm_destroy", "lbm_batch_create", "lbm_batch_create_ex", "lbm_plan_preview", "lbm_batch_step",
    "lbm_batch_items",
    "lbm_batch_destroy",
    "lbm_step_noalloc", "lbm_slug_geometry",
)


LBM_PLAN_AUTO, LBM_PLAN_BALANCED, LBM_PLAN_SPLIT = 0, 1, 2


class lbm_batch_opts(ctypes.Structure):
    _fields_ = [("rows_per_item", ctypes.c_int), ("row_overhead", ctypes.c_float), ("plan", ctypes.c_int),
                ("member_plan_rows", ctypes.POINTER(ctypes.c_int))]


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("gamma", ctypes.c_double), ("alpha_b", ctypes.c_double),
        ("tau_r", ctypes.c_double), ("tau_b", ctypes.c_double),
        ("delta", ctypes.c_double), ("sigma", ctypes.c_double), ("beta", ctypes.c_double),
        ("gx", ctypes.c_double), ("gy", ctypes.c_double),
        ("collision", ctypes.c_int), ("equilibrium", ctypes.c_int),
        ("mrt_lambda", ctypes.c_double), ("c7_sign", ctypes.c_double),
        ("c7_factor", ctypes.c_double), ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int), ("storage", ctypes.c_int),
        ("u_in_r", ctypes.c_double), ("u_in_b", ctypes.c_double), ("p_out", ctypes.c_double),
        ("inlet_mode", ctypes.c_int), ("inlet_period_r", ctypes.c_int),
        ("inlet_period_b", ctypes.c_int), ("inlet_layer", ctypes.c_int),
        ("kernel", ctypes.c_int), ("plan_rows", ctypes.c_int), ("plan", ctypes.c_int),
        ("wall_slip", ctypes.c_int), ("contact_angle", ctypes.c_double),
    ]


class lbm_diag(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_longlong),
        ("mass_r", ctypes.c_double), ("mass_b", ctypes.c_double),
        ("mom_x", ctypes.c_double), ("mom_y", ctypes.c_double), ("max_u", ctypes.c_double),
        ("area_b", ctypes.c_double), ("cx_b", ctypes.c_double), ("cy_b", ctypes.c_double),
        ("ux_b", ctypes.c_double), ("ux_r", ctypes.c_double), ("r_eff", ctypes.c_double),
        ("p_in", ctypes.c_double), ("p_out", ctypes.c_double), ("dp", ctypes.c_double),
        ("nonfinite", ctypes.c_longlong),
    ]

    def as_dict(self) -> dict:
        return {f[0]: getattr(self, f[0]) for f in self._fields_}


LBM_SLUG_MAX = 16


class lbm_slug(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_longlong), ("n_bubbles", ctypes.c_int), ("n_slugs", ctypes.c_int),
        ("bubble_len", ctypes.c_double), ("slug_len", ctypes.c_double), ("film", ctypes.c_double),
        ("x_tail", ctypes.c_double * LBM_SLUG_MAX), ("x_nose", ctypes.c_double * LBM_SLUG_MAX),
    ]

    def as_dict(self) -> dict:
        n = min(self.n_bubbles, LBM_SLUG_MAX)
        return {"t": self.t, "n_bubbles": self.n_bubbles, "n_slugs": self.n_slugs,
                "bubble_len": self.bubble_len, "slug_len": self.slug_len, "film": self.film,
                "x_tail": list(self.x_tail[:n]), "x_nose": list(self.x_nose[:n])}


class LBMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load the native library (optionally building it first)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and _build.stale():
        _build.build()
    if not os.path.exists(path):
        raise ImportError(f"native library {path} is not built; run "
                          "`python -m paper_1903_01168_gb300.build` (no CPU fallback exists)")
    L = ctypes.CDLL(path)
    vp, dp, i, l, st = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_long, ctypes.c_size_t
    pp = ctypes.POINTER(lbm_params)
    L.lbm_default_params.argtypes = [pp]
    L.lbm_bytes_required.argtypes = [i, i, pp]
    L.lbm_bytes_required.restype = st
    L.lbm_create.argtypes = [i, i, pp, ctypes.POINTER(vp)]
    L.lbm_create_ex.argtypes = [i, i, pp, vp, st, vp, ctypes.POINTER(vp)]
    L.lbm_init_bubble.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    L.lbm_init_slug.argtypes = [vp, i, ctypes.c_double, ctypes.c_double, i]
    L.lbm_init_fields.argtypes = [vp, dp, dp, dp, dp]
    L.lbm_init_populations.argtypes = [vp, dp]
    L.lbm_step.argtypes = [vp, l]
    L.lbm_set_stop.argtypes = [vp, ctypes.c_longlong]
    L.lbm_synchronize.argtypes = [vp]
    L.lbm_time.argtypes = [vp]
    L.lbm_time.restype = ctypes.c_longlong
    L.lbm_read_fields.argtypes = [vp, dp, dp, dp, dp, dp]
    L.lbm_read_populations.argtypes = [vp, dp]
    L.lbm_diagnostics.argtypes = [vp, ctypes.POINTER(lbm_diag)]
    L.lbm_slug_geometry.argtypes = [vp, ctypes.POINTER(lbm_slug), dp]
    L.lbm_state_bytes.argtypes = [vp]
    L.lbm_state_bytes.restype = st
    L.lbm_save_state.argtypes = [vp, vp, st]
    L.lbm_load_state.argtypes = [vp, vp, st]
    L.lbm_last_error.argtypes = [vp]
    L.lbm_last_error.restype = ctypes.c_char_p
    L.lbm_destroy.argtypes = [vp]
    L.lbm_destroy.restype = None
    L.lbm_step_noalloc.argtypes = [pp, i, i, vp, st, ctypes.c_longlong, l, vp]
    L.lbm_batch_create.argtypes = [ctypes.POINTER(vp), i, i, ctypes.POINTER(vp)]
    L.lbm_batch_create_ex.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(lbm_batch_opts), ctypes.POINTER(vp)]
    L.lbm_plan_preview.argtypes = [ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), i,
                                   ctypes.POINTER(lbm_batch_opts), i, ctypes.POINTER(i), ctypes.POINTER(i),
                                   ctypes.POINTER(i), i]
    L.lbm_batch_step.argtypes = [vp, l, i]
    L.lbm_batch_items.argtypes = [vp]
    L.lbm_batch_destroy.argtypes = [vp]
    L.lbm_batch_destroy.restype = None
    _lib = L
    return L


def _check(status: int, sim=None):
    if status != LBM_OK:
        msg = load().lbm_last_error(sim).decode(errors="replace")
        raise LBMError(status, msg)


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ------------------------------------------------------------- C ABI wrappers

def lbm_default_params() -> lbm_params:
    p = lbm_params()
    _check(load().lbm_default_params(ctypes.byref(p)))
    return p


def lbm_bytes_required(nx: int, ny: int, p: lbm_params) -> int:
    return load().lbm_bytes_required(nx, ny, ctypes.byref(p))


def lbm_create(nx: int, ny: int, p: lbm_params) -> int:
    h = ctypes.c_void_p()
    _check(load().lbm_create(nx, ny, ctypes.byref(p), ctypes.byref(h)))
    return h.value


def lbm_create_ex(nx: int, ny: int, p: lbm_params, dev_ptr: int, nbytes: int, stream: int) -> int:
    h = ctypes.c_void_p()
    _check(load().lbm_create_ex(nx, ny, ctypes.byref(p), ctypes.c_void_p(dev_ptr), nbytes,
                                ctypes.c_void_p(stream), ctypes.byref(h)))
    return h.value


def lbm_init_bubble(sim: int, cx: float, cy: float, R: float):
    _check(load().lbm_init_bubble(sim, cx, cy, R), sim)


def lbm_init_slug(sim: int, n_bubbles: int, length: float, height: float, poiseuille: bool):
    _check(load().lbm_init_slug(sim, n_bubbles, length, height, int(poiseuille)), sim)


def lbm_init_fields(sim: int, rho_r, rho_b, ux, uy):
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (rho_r, rho_b, ux, uy)]
    _check(load().lbm_init_fields(sim, *[_dptr(v) for v in a]), sim)


def lbm_init_populations(sim: int, pops):
    a = np.ascontiguousarray(pops, dtype=np.float64)
    _check(load().lbm_init_populations(sim, _dptr(a)), sim)


def lbm_step(sim: int, n: int):
    _check(load().lbm_step(sim, int(n)), sim)


def lbm_set_stop(sim: int, t_end: int):
    _check(load().lbm_set_stop(sim, int(t_end)), sim)


def lbm_synchronize(sim: int):
    _check(load().lbm_synchronize(sim), sim)


def lbm_time(sim: int) -> int:
    return load().lbm_time(sim)


def lbm_read_fields(sim: int, nx: int, ny: int, out: dict | None = None) -> dict:
    """Fields into `out` (C-contiguous float64 arrays (ny, nx) keyed rho_r, rho_b, ux,
    uy, p, e.g. views of pinned host memory) or into new arrays."""
    names = ("rho_r", "rho_b", "ux", "uy", "p")
    if out is None:
        out = {k: np.empty((ny, nx)) for k in names}
    for k in names:
        a = out[k]
        if a.dtype != np.float64 or a.shape != (ny, nx) or not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"out[{k!r}] must be a C-contiguous float64 array of shape {(ny, nx)}")
    _check(load().lbm_read_fields(sim, *[_dptr(out[k]) for k in ("rho_r", "rho_b", "ux", "uy", "p")]), sim)
    return out


def lbm_read_populations(sim: int, nx: int, ny: int) -> np.ndarray:
    out = np.empty((2, 9, ny, nx))
    _check(load().lbm_read_populations(sim, _dptr(out)), sim)
    return out


def lbm_diagnostics(sim: int, allow_unstable: bool = False) -> dict:
    d = lbm_diag()
    st = load().lbm_diagnostics(sim, ctypes.byref(d))
    if not (allow_unstable and st == LBM_EUNSTABLE):
        _check(st, sim)
    out = d.as_dict()
    out["status"] = st
    return out


def lbm_slug_geometry(sim: int, nx: int) -> tuple[dict, np.ndarray]:
    """Slug-train geometry (lbm_slug as a dict) and the column light thickness g(x)."""
    o = lbm_slug()
    gas = np.empty(nx)
    _check(load().lbm_slug_geometry(sim, ctypes.byref(o), _dptr(gas)), sim)
    return o.as_dict(), gas


def lbm_state_bytes(sim: int) -> int:
    return load().lbm_state_bytes(sim)


def lbm_save_state(sim: int) -> bytes:
    n = lbm_state_bytes(sim)
    buf = ctypes.create_string_buffer(n)
    _check(load().lbm_save_state(sim, buf, n), sim)
    return buf.raw


def lbm_load_state(sim: int, state: bytes):
    buf = ctypes.create_string_buffer(state, len(state))
    _check(load().lbm_load_state(sim, buf, len(state)), sim)


def lbm_last_error(sim) -> str:
    return load().lbm_last_error(sim).decode(errors="replace")


def lbm_destroy(sim: int):
    if sim:
        load().lbm_destroy(sim)


def lbm_step_noalloc(p: lbm_params, nx: int, ny: int, state_ptr: int, nbytes: int, t: int, n: int,
                     stream: int = 0):
    """Advance a caller-owned device state buffer by n steps without any device
    allocation (see include/lbm.h)."""
    _check(load().lbm_step_noalloc(ctypes.byref(p), nx, ny, ctypes.c_void_p(state_ptr), nbytes, int(t), int(n),
                                   ctypes.c_void_p(stream)))


def lbm_batch_create(sims, rows_per_item: int = 0, row_overhead: float | None = None,
                     plan: int = LBM_PLAN_AUTO, member_plan_rows=None) -> int:
    arr = (ctypes.c_void_p * len(sims))(*sims)
    h = ctypes.c_void_p()
    if row_overhead is None and plan == LBM_PLAN_AUTO and member_plan_rows is None:
        _check(load().lbm_batch_create(arr, len(sims), rows_per_item, ctypes.byref(h)))
    else:
        rows = None
        if member_plan_rows is not None:
            if len(member_plan_rows) != len(sims):
                raise ValueError("member_plan_rows needs one value per member")
            rows = (ctypes.c_int * len(sims))(*[int(r) for r in member_plan_rows])
        opts = lbm_batch_opts(rows_per_item=rows_per_item,
                              row_overhead=-1.0 if row_overhead is None else row_overhead, plan=plan,
                              member_plan_rows=rows)
        _check(load().lbm_batch_create_ex(arr, len(sims), ctypes.byref(opts), ctypes.byref(h)))
    return h.value


def lbm_plan_preview(sizes, max_blocks: int, plan: int = LBM_PLAN_AUTO, row_overhead: float | None = None,
                     rows_per_item: int = 0, plan_rows=None) -> tuple[int, np.ndarray]:
    """Host-only preview of a batch's work plan: (blocks, items) with items an
    (n_items, 6) int array of member, x0, width, first row, end row, block."""
    n = len(sizes)
    nx = (ctypes.c_int * n)(*[int(a) for a, _ in sizes])
    ny = (ctypes.c_int * n)(*[int(b) for _, b in sizes])
    pr = None if plan_rows is None else (ctypes.c_int * n)(*[int(r) for r in plan_rows])
    opts = lbm_batch_opts(rows_per_item=rows_per_item, row_overhead=-1.0 if row_overhead is None else row_overhead,
                          plan=plan)
    ni, nb = ctypes.c_int(), ctypes.c_int()
    lib = load()
    _check(lib.lbm_plan_preview(nx, ny, pr, n, ctypes.byref(opts), max_blocks, ctypes.byref(ni), ctypes.byref(nb),
                                None, 0))
    buf = (ctypes.c_int * (6 * ni.value))()
    _check(lib.lbm_plan_preview(nx, ny, pr, n, ctypes.byref(opts), max_blocks, ctypes.byref(ni), ctypes.byref(nb),
                                buf, ni.value))
    return nb.value, np.array(buf, dtype=np.int64).reshape(ni.value, 6)


def lbm_batch_step(batch: int, n: int, use_graph: bool = True, sim_for_errors=None):
    _check(load().lbm_batch_step(batch, int(n), int(use_graph)), sim_for_errors)


def lbm_batch_items(batch: int) -> int:
    return load().lbm_batch_items(batch)


def lbm_batch_destroy(batch: int):
    if batch:
        load().lbm_batch_destroy(batch)


# --------------------------------------------------------------- convenience

PARAM_NAMES = [f[0] for f in lbm_params._fields_]


def make_params(**kw) -> lbm_params:
    """Defaults of lbm_default_params() overridden by keyword arguments."""
    p = lbm_default_params()
    for k, v in kw.items():
        if k not in PARAM_NAMES:
            raise KeyError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


class Simulation:
    """One lattice on the current CUDA device."""

    def __init__(self, nx: int, ny: int, torch_memory: bool = False, **params):
        self.nx, self.ny = nx, ny
        self.params = make_params(**params)
        self._buf = None
        if torch_memory:
            import torch
            nbytes = lbm_bytes_required(nx, ny, self.params)
            if nbytes == 0:
                raise LBMError(LBM_EINVAL, "invalid parameters")
            self._buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            stream = torch.cuda.current_stream().cuda_stream
            self.h = lbm_create_ex(nx, ny, self.params, self._buf.data_ptr(), nbytes, stream)
        else:
            self.h = lbm_create(nx, ny, self.params)

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def t(self) -> int:
        return lbm_time(self.h)

    def init_bubble(self, cx, cy, R):
        lbm_init_bubble(self.h, cx, cy, R)

    def init_slug(self, n_bubbles, length, height, poiseuille=True):
        lbm_init_slug(self.h, n_bubbles, length, height, poiseuille)

    def init_fields(self, rho_r, rho_b, ux, uy):
        lbm_init_fields(self.h, rho_r, rho_b, ux, uy)

    def init_populations(self, pops):
        """pops: array (2, 9, ny, nx) of pre-collision populations."""
        lbm_init_populations(self.h, pops)

    def step(self, n: int = 1):
        lbm_step(self.h, n)

    def set_stop(self, t_end: int):
        """Steps at or after t_end leave the state unchanged (t_end < 0: no stop)."""
        lbm_set_stop(self.h, t_end)

    def synchronize(self):
        lbm_synchronize(self.h)

    def fields(self, out: dict | None = None) -> dict:
        """rho_r, rho_b, ux, uy, p as float64 (ny, nx) arrays; `out` gives the arrays
        to fill (pinned host memory makes the device-to-host copies direct)."""
        return lbm_read_fields(self.h, self.nx, self.ny, out)

    def populations(self) -> np.ndarray:
        """Pre-collision populations, array (2, 9, ny, nx)."""
        return lbm_read_populations(self.h, self.nx, self.ny)

    def diagnostics(self, allow_unstable: bool = False) -> dict:
        return lbm_diagnostics(self.h, allow_unstable)

    def slug_geometry(self) -> tuple[dict, np.ndarray]:
        """(bubble / slug / film geometry, column light thickness g(x))."""
        return lbm_slug_geometry(self.h, self.nx)

    def save_state(self) -> bytes:
        return lbm_save_state(self.h)

    def load_state(self, state: bytes):
        lbm_load_state(self.h, state)


class Batch:
    """Several simulations advanced together, one launch per step."""

    def __init__(self, sims, rows_per_item: int = 0, row_overhead: float | None = None,
                 plan: int = LBM_PLAN_AUTO, member_plan_rows=None):
        """rows_per_item > 0: fixed plan; otherwise `plan` (LBM_PLAN_*) with
        row_overhead, the planner's fixed cost of a strip row in busy warps
        (None: library default), and optionally one plan_rows per member in
        place of the members' own."""
        self.sims = list(sims)
        self.h = lbm_batch_create([s.h for s in self.sims], rows_per_item, row_overhead, plan, member_plan_rows)

    @property
    def items(self) -> int:
        return lbm_batch_items(self.h)

    def step(self, n: int = 1, use_graph: bool = True):
        lbm_batch_step(self.h, n, use_graph, self.sims[0].h)

    def close(self):
        if getattr(self, "h", None):
            lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
