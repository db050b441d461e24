"""FP64 CPU oracle of the two-phase colour-gradient LBM step (arXiv 1903.01168, Sec. 2).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module.  The product path (the CUDA library and its
binding) never does.

This file only marshals arguments to the plain C oracle in ``lbm_oracle.c`` (built with
gcc on first use) and converts its flat arrays to numpy.  All arithmetic is in the C file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_HDR = os.path.join(_HERE, "lbm_oracle.h")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")

BGK, MRT = 0, 1
EQ_STD, EQ_HERMITE = 0, 1
PERIODIC, WALL, INOUT = 0, 1, 2
INLET_ALTERNATE, INLET_LAYERED = 0, 1
PERTURB_PER_COLOUR, PERTURB_ONCE = 0, 1


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("gamma", ctypes.c_double), ("alpha_b", ctypes.c_double),
        ("tau_r", ctypes.c_double), ("tau_b", ctypes.c_double),
        ("delta", ctypes.c_double), ("sigma", ctypes.c_double),
        ("beta", ctypes.c_double), ("gx", ctypes.c_double), ("gy", ctypes.c_double),
        ("collision", ctypes.c_int), ("equilibrium", ctypes.c_int),
        ("mrt_lambda", ctypes.c_double), ("c7_sign", ctypes.c_double),
        ("c7_factor", ctypes.c_double), ("perturb_mode", ctypes.c_int),
        ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
        ("u_in_r", ctypes.c_double), ("u_in_b", ctypes.c_double), ("p_out", ctypes.c_double),
        ("inlet_mode", ctypes.c_int), ("inlet_period_r", ctypes.c_int),
        ("inlet_period_b", ctypes.c_int), ("inlet_layer", ctypes.c_int),
        ("wall_slip", ctypes.c_int), ("contact_angle", ctypes.c_double),
    ]


@dataclass
class OracleParams:
    """Parameters of one simulation; defaults are the paper's constants
    (alpha_b = 0.2, delta = 0.1, beta = 0.99, MRT lambda = 4/5)."""
    nx: int = 64
    ny: int = 64
    gamma: float = 1.0
    alpha_b: float = 0.2
    tau_r: float = 1.0
    tau_b: float = 1.0
    delta: float = 0.1
    sigma: float = 0.005
    beta: float = 0.99
    gx: float = 0.0
    gy: float = 0.0
    collision: int = BGK
    equilibrium: int = EQ_STD
    mrt_lambda: float = 0.8
    c7_sign: float = -1.0
    c7_factor: float = 1.0
    perturb_mode: int = PERTURB_PER_COLOUR
    bc_x: int = PERIODIC
    bc_y: int = PERIODIC
    u_in_r: float = 0.0
    u_in_b: float = 0.0
    p_out: float = 0.0
    inlet_mode: int = INLET_ALTERNATE
    inlet_period_r: int = 0
    inlet_period_b: int = 0
    inlet_layer: int = 0
    wall_slip: int = 0
    contact_angle: float = 0.0

    def to_c(self) -> _Params:
        return _Params(**{f.name: getattr(self, f.name) for f in fields(self)})


def build(force: bool = False) -> str:
    """Compile the C oracle into a shared library next to its source."""
    stale = (not os.path.exists(_LIB)
             or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def bind(path: str, real=ctypes.c_double) -> ctypes.CDLL:
    """Load an oracle shared library and declare its C signatures.  `real` is the
    library's arithmetic type (ctypes.c_double, or ctypes.c_float for a build
    with ORC_REAL=float); arrays passed to it use the matching numpy dtype."""
    L = ctypes.CDLL(path)
    L.real_dtype = np.float64 if real is ctypes.c_double else np.float32
    dp = ctypes.POINTER(real)
    pp = ctypes.POINTER(_Params)
    L.orc_create.restype = ctypes.c_void_p
    L.orc_create.argtypes = [pp]
    L.orc_destroy.argtypes = [ctypes.c_void_p]
    L.orc_time.restype = ctypes.c_long
    L.orc_time.argtypes = [ctypes.c_void_p]
    L.orc_set_pops.argtypes = [ctypes.c_void_p, dp]
    L.orc_get_pops.argtypes = [ctypes.c_void_p, dp]
    L.orc_init_fields.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
    L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
    L.orc_fields.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, dp, dp]
    L.orc_gradient_fields.argtypes = [ctypes.c_void_p, dp, dp, dp]
    L.orc_derived.argtypes = [pp] + [dp] * 8
    L.orc_equilibrium.argtypes = [pp, ctypes.c_int, real, real, real, dp]
    L.orc_omega_eff.restype = real
    L.orc_omega_eff.argtypes = [pp, real]
    L.orc_perturbation.argtypes = [pp, real, real, real, dp]
    L.orc_recolour.argtypes = [pp, real, real, real, real, dp, dp, dp]
    L.orc_mrt_matrices.argtypes = [dp, dp]
    L.orc_collide_node.argtypes = [pp, dp, real, real] + [real] * 4 + [dp]
    L.orc_zouhe_inlet.argtypes = [pp, real, dp, dp]
    L.orc_zouhe_outlet.argtypes = [pp, dp, dp]
    return L


def compile_variant(source_text: str, out_dir: str, flags=()) -> str:
    """Compile a copy of the oracle source, possibly modified (the tests plant
    mistakes in it to show that the pins catch them), with extra gcc flags into
    out_dir; returns the library path."""
    src = os.path.join(out_dir, "lbm_oracle_variant.c")
    with open(src, "w") as f:
        f.write(source_text)
    so = os.path.join(out_dir, "liblbm_oracle_variant.so")
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-shared", "-fPIC", *flags, "-I", _HERE, "-o",
                           so, src, "-lm"])
    return so


def fp32_library(out_dir: str) -> ctypes.CDLL:
    """The oracle source built with an FP32 arithmetic type and single-precision
    constants (parameters are still given in double): what FP32 rounding alone
    does to a case, with no other difference from the FP64 oracle."""
    src = open(_SRC).read()
    return bind(compile_variant(src, out_dir, ("-DORC_REAL=float", "-fsingle-precision-constant")),
                real=ctypes.c_float)


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = bind(build())
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype in (np.float64, np.float32) and a.flags["C_CONTIGUOUS"]
    ct = ctypes.c_double if a.dtype == np.float64 else ctypes.c_float
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """One FP64 simulation.  State = pre-collision populations N^k_i(x, t),
    array shape (2, 9, ny, nx), k = 0 red (heavy), 1 blue (light)."""

    def __init__(self, params: OracleParams, library=None):
        """library: a bound oracle library (default: the FP64 oracle)."""
        self.params = params
        self._cp = params.to_c()
        self._L = library if library is not None else lib()
        self._dt = self._L.real_dtype
        self._h = self._L.orc_create(ctypes.byref(self._cp))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.orc_destroy(h)
            self._h = None

    @property
    def shape(self):
        return (self.params.ny, self.params.nx)

    @property
    def t(self) -> int:
        return self._L.orc_time(self._h)

    def init_fields(self, rho_r, rho_b, ux, uy):
        a = [np.ascontiguousarray(v, dtype=self._dt).reshape(self.shape) for v in (rho_r, rho_b, ux, uy)]
        self._L.orc_init_fields(self._h, *[_ptr(v) for v in a])

    def set_pops(self, pops):
        a = np.ascontiguousarray(pops, dtype=self._dt).reshape((2, 9) + self.shape)
        self._L.orc_set_pops(self._h, _ptr(a))

    def get_pops(self) -> np.ndarray:
        out = np.empty((2, 9) + self.shape, dtype=self._dt)
        self._L.orc_get_pops(self._h, _ptr(out))
        return out.astype(np.float64)

    def step(self, n: int = 1):
        self._L.orc_step(self._h, int(n))

    def fields(self) -> dict:
        names = ("rho_r", "rho_b", "ux", "uy", "p", "psi")
        out = {k: np.empty(self.shape, dtype=self._dt) for k in names}
        self._L.orc_fields(self._h, *[_ptr(out[k]) for k in names])
        return {k: v.astype(np.float64) for k, v in out.items()}


# ---- single operators (for pins) ----

def derived(params: OracleParams) -> dict:
    vals = [ctypes.c_double() for _ in range(8)]
    cp = params.to_c()
    lib().orc_derived(ctypes.byref(cp), *[ctypes.byref(v) for v in vals])
    names = ("alpha_r", "omega_r", "omega_b", "chi", "eta", "kappa", "lam", "nu")
    return {k: v.value for k, v in zip(names, vals)}


def equilibrium(params: OracleParams, k: int, rho_k: float, ux: float, uy: float) -> np.ndarray:
    out = np.empty(9)
    cp = params.to_c()
    lib().orc_equilibrium(ctypes.byref(cp), k, rho_k, ux, uy, _ptr(out))
    return out


def omega_eff(params: OracleParams, psi: float) -> float:
    cp = params.to_c()
    return lib().orc_omega_eff(ctypes.byref(cp), psi)


def perturbation(params: OracleParams, A: float, Fx: float, Fy: float) -> np.ndarray:
    out = np.empty(9)
    cp = params.to_c()
    lib().orc_perturbation(ctypes.byref(cp), A, Fx, Fy, _ptr(out))
    return out


def recolour(params: OracleParams, rho_r, rho_b, Fx, Fy, N):
    N = _f64(N)
    Nr, Nb = np.empty(9), np.empty(9)
    cp = params.to_c()
    lib().orc_recolour(ctypes.byref(cp), rho_r, rho_b, Fx, Fy, _ptr(N), _ptr(Nr), _ptr(Nb))
    return Nr, Nb


def mrt_matrices():
    M, Mi = np.empty(81), np.empty(81)
    lib().orc_mrt_matrices(_ptr(M), _ptr(Mi))
    return M.reshape(9, 9), Mi.reshape(9, 9)


def collide_node(params: OracleParams, Nk, Fx=0.0, Fy=0.0, divQ=(0.0, 0.0, 0.0, 0.0)):
    Nk = _f64(Nk).reshape(18)
    out = np.empty(18)
    cp = params.to_c()
    lib().orc_collide_node(ctypes.byref(cp), _ptr(Nk), Fx, Fy, *divQ, _ptr(out))
    return out.reshape(2, 9)


def zouhe_inlet(params: OracleParams, f_r: float, Nr, Nb):
    Nr, Nb = _f64(Nr).copy(), _f64(Nb).copy()
    cp = params.to_c()
    lib().orc_zouhe_inlet(ctypes.byref(cp), f_r, _ptr(Nr), _ptr(Nb))
    return Nr, Nb


def zouhe_outlet(params: OracleParams, Nr, Nb):
    Nr, Nb = _f64(Nr).copy(), _f64(Nb).copy()
    cp = params.to_c()
    lib().orc_zouhe_outlet(ctypes.byref(cp), _ptr(Nr), _ptr(Nb))
    return Nr, Nb


def gradient_fields(o: Oracle):
    """Colour gradient F and the S2I4 derivatives of Q^k for every node."""
    ny, nx = o.shape
    Fx, Fy, dQ = (np.empty(o.shape, dtype=o._dt), np.empty(o.shape, dtype=o._dt),
                  np.empty((4, ny, nx), dtype=o._dt))
    o._L.orc_gradient_fields(o._h, _ptr(Fx), _ptr(Fy), _ptr(dQ))
    return Fx, Fy, dQ
