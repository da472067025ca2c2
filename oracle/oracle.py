"""ctypes binding of the FP64 CPU oracle in ``lbm_oracle.c``.

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, plain statement of the
coupled central-moment lattice Boltzmann step of arXiv 2408.00146 against which
the CUDA path is checked.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the product package
never does.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
HDR = os.path.join(HERE, "lbm_oracle.h")
LIB = os.path.join(HERE, "_build", "liboracle.so")

# Field order of the orc_params struct (must match lbm_oracle.h).
PARAM_FIELDS = [
    ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("walls", ctypes.c_int32),
    ("R", ctypes.c_double), ("xb", ctypes.c_double), ("yb", ctypes.c_double),
    ("W", ctypes.c_double), ("M_phi", ctypes.c_double),
    ("rho_A", ctypes.c_double), ("rho_ratio", ctypes.c_double),
    ("mu_ratio", ctypes.c_double), ("alpha_ratio", ctypes.c_double),
    ("Re", ctypes.c_double), ("Ma", ctypes.c_double),
    ("sigma0", ctypes.c_double), ("sigma_T", ctypes.c_double),
    ("sigma_TT", ctypes.c_double), ("T_ref", ctypes.c_double),
    ("T_H", ctypes.c_double), ("T_C", ctypes.c_double),
    ("beta", ctypes.c_double), ("Pi", ctypes.c_double), ("Ex", ctypes.c_double),
    ("M_psi", ctypes.c_double), ("psi0", ctypes.c_double),
    ("Fext_x", ctypes.c_double), ("Fext_y", ctypes.c_double),
    ("gravity", ctypes.c_double), ("nu_A", ctypes.c_double),
    ("alpha_A", ctypes.c_double),
    ("psi_L", ctypes.c_double), ("psi_R", ctypes.c_double), ("psi_bc", ctypes.c_int32),
]
# parameters added after the first release: absent from a dict means 0
OPTIONAL = ("psi_L", "psi_R", "psi_bc")

DERIVED_FIELDS = [
    "dT", "M1", "M2", "L", "U_o", "rho_A", "rho_B", "mu_A", "mu_B", "nu_A",
    "nu_B", "alpha_A", "alpha_B", "omega_phi", "omega_psi", "lambda", "s", "w",
    "m_psi", "D_psi",
]


class OrcParams(ctypes.Structure):
    _fields_ = PARAM_FIELDS


class OrcDerived(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in DERIVED_FIELDS]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, FP64,
    OpenMP, no FMA contraction so x86 and Arm round alike)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    stale = force or not os.path.exists(LIB) or any(
        os.path.getmtime(p) > os.path.getmtime(LIB) for p in (SRC, HDR))
    if stale:
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-std=c11", "-Wall", "-o", tmp, SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


def _bind(L):
    """Argument and result types of every exported oracle function."""
    P, I64, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
    dp = ctypes.POINTER(ctypes.c_double)
    L.orc_derive.argtypes = [ctypes.POINTER(OrcParams), ctypes.POINTER(OrcDerived)]
    L.orc_create.argtypes = [ctypes.POINTER(OrcParams), ctypes.POINTER(P)]
    L.orc_destroy.argtypes = [P]
    L.orc_destroy.restype = None
    L.orc_set_threads.argtypes = [ctypes.c_int]
    L.orc_init_fields.argtypes = [P, dp]
    L.orc_set_populations.argtypes = [P, dp]
    L.orc_get_populations.argtypes = [P, dp]
    L.orc_step.argtypes = [P, I64]
    L.orc_time.argtypes = [P]
    L.orc_time.restype = I64
    L.orc_fields.argtypes = [P, dp]
    L.orc_observe.argtypes = [P, dp]
    L.orc_matrix_P.argtypes = [dp]
    L.orc_matrix_P.restype = None
    L.orc_matrix_Pinv.argtypes = [dp]
    L.orc_matrix_Pinv.restype = None
    L.orc_matrix_F.argtypes = [D, D, dp]
    L.orc_matrix_F.restype = None
    L.orc_weights.argtypes = [dp]
    L.orc_weights.restype = None
    L.orc_velocities.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.orc_velocities.restype = None
    L.orc_sigma_eos.argtypes = [ctypes.POINTER(OrcParams), D, D]
    L.orc_sigma_eos.restype = D
    L.orc_G.argtypes = [ctypes.POINTER(OrcDerived), D, D]
    L.orc_G.restype = D
    L.orc_dG.argtypes = [ctypes.POINTER(OrcDerived), D, D]
    L.orc_dG.restype = D
    L.orc_cm_collide.argtypes = [dp, D, D, dp, dp, dp, ctypes.c_int, D, D, dp]
    L.orc_cm_collide.restype = None
    L.orc_gradient_periodic.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(LIB))
    return _lib


_variants: dict = {}


def variant(tag: str, edits: list[tuple[str, str]]):
    """The oracle with a planted mistake, for tests that show a pin fails on
    it: a copy of lbm_oracle.c with each (old, new) text replaced (old must
    occur exactly once), compiled like the oracle into its own library under
    _build/variants/ and loaded beside it.  The oracle's source is untouched."""
    with _lock:
        if tag in _variants:
            return _variants[tag]
        with open(SRC) as fh:
            src = fh.read()
        for old, new in edits:
            if src.count(old) != 1:
                raise ValueError(f"variant {tag}: {old!r} occurs {src.count(old)} times")
            src = src.replace(old, new)
        vdir = os.path.join(HERE, "_build", "variants")
        os.makedirs(vdir, exist_ok=True)
        csrc = os.path.join(vdir, f"lbm_oracle_{tag}.c")
        so = os.path.join(vdir, f"liboracle_{tag}.so")
        with open(csrc, "w") as fh:
            fh.write(src)
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC",
                               "-shared", "-std=c11", "-Wall", "-I", HERE, "-o", so, csrc,
                               "-lm"])
        L = _bind(ctypes.CDLL(so))
        L.orc_set_threads(os.cpu_count() or 1)
        _variants[tag] = L
        return L


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_params(d: dict) -> OrcParams:
    p = OrcParams()
    for name, _ in PARAM_FIELDS:
        setattr(p, name, d.get(name, 0) if name in OPTIONAL else d[name])
    return p


def set_threads(n: int) -> int:
    return lib().orc_set_threads(int(n))


def derive(d: dict) -> dict:
    p = make_params(d)
    out = OrcDerived()
    rc = lib().orc_derive(ctypes.byref(p), ctypes.byref(out))
    if rc != 0:
        raise ValueError(f"orc_derive rejected the parameters (code {rc})")
    return {n: getattr(out, n) for n in DERIVED_FIELDS}


def matrix_P() -> np.ndarray:
    a = np.zeros(81)
    lib().orc_matrix_P(_dp(a))
    return a.reshape(9, 9)


def matrix_Pinv() -> np.ndarray:
    a = np.zeros(81)
    lib().orc_matrix_Pinv(_dp(a))
    return a.reshape(9, 9)


def matrix_F(ux: float, uy: float) -> np.ndarray:
    a = np.zeros(81)
    lib().orc_matrix_F(float(ux), float(uy), _dp(a))
    return a.reshape(9, 9)


def weights() -> np.ndarray:
    a = np.zeros(9)
    lib().orc_weights(_dp(a))
    return a


def velocities():
    ex = (ctypes.c_int * 9)()
    ey = (ctypes.c_int * 9)()
    lib().orc_velocities(ex, ey)
    return np.array(list(ex)), np.array(list(ey))


def sigma_eos(d: dict, T: float, psi: float) -> float:
    p = make_params(d)
    return lib().orc_sigma_eos(ctypes.byref(p), float(T), float(psi))


def _derived_struct(d: dict) -> OrcDerived:
    p = make_params(d)
    out = OrcDerived()
    if lib().orc_derive(ctypes.byref(p), ctypes.byref(out)) != 0:
        raise ValueError("orc_derive rejected the parameters")
    return out


def G(d: dict, phi: float) -> float:
    return lib().orc_G(ctypes.byref(_derived_struct(d)), float(d["W"]), float(phi))


def dG(d: dict, phi: float) -> float:
    return lib().orc_dG(ctypes.byref(_derived_struct(d)), float(d["W"]), float(phi))


def cm_collide(pop, ux, uy, eq, om, src=None, split=False, om2s=1.0, om2d=1.0):
    pop = np.ascontiguousarray(pop, dtype=np.float64)
    eq = np.ascontiguousarray(eq, dtype=np.float64)
    om = np.ascontiguousarray(om, dtype=np.float64)
    out = np.zeros(9)
    src_p = None
    if src is not None:
        src = np.ascontiguousarray(src, dtype=np.float64)
        src_p = _dp(src)
    lib().orc_cm_collide(_dp(pop), float(ux), float(uy), _dp(eq), _dp(om), src_p,
                         int(bool(split)), float(om2s), float(om2d), _dp(out))
    return out


def gradient_periodic(a: np.ndarray):
    a = np.ascontiguousarray(a, dtype=np.float64)
    ny, nx = a.shape
    gx = np.zeros_like(a)
    gy = np.zeros_like(a)
    lib().orc_gradient_periodic(nx, ny, _dp(a), _dp(gx), _dp(gy))
    return gx, gy


class Oracle:
    """One FP64 simulation held by the oracle library."""

    def __init__(self, params: dict, library=None):
        self.params = dict(params)
        self._L = library if library is not None else lib()
        self._p = make_params(params)
        h = ctypes.c_void_p()
        rc = self._L.orc_create(ctypes.byref(self._p), ctypes.byref(h))
        if rc != 0:
            raise ValueError(f"orc_create rejected the parameters (code {rc})")
        self._h = h
        self.nx, self.ny = int(params["nx"]), int(params["ny"])

    def close(self):
        if self._h:
            self._L.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_fields(self, fields: np.ndarray):
        f = np.ascontiguousarray(fields, dtype=np.float64)
        assert f.shape == (6, self.ny, self.nx)
        self._L.orc_init_fields(self._h, _dp(f))

    def set_populations(self, pops: np.ndarray):
        f = np.ascontiguousarray(pops, dtype=np.float64)
        assert f.shape == (4, 9, self.ny, self.nx)
        self._L.orc_set_populations(self._h, _dp(f))

    def populations(self) -> np.ndarray:
        out = np.zeros((4, 9, self.ny, self.nx))
        self._L.orc_get_populations(self._h, _dp(out))
        return out

    def step(self, n: int = 1):
        rc = self._L.orc_step(self._h, int(n))
        if rc != 0:
            raise RuntimeError(f"orc_step failed ({rc})")

    @property
    def t(self) -> int:
        return int(self._L.orc_time(self._h))

    def fields(self) -> np.ndarray:
        out = np.zeros((6, self.ny, self.nx))
        self._L.orc_fields(self._h, _dp(out))
        return out

    def observe(self) -> dict:
        out = np.zeros(9)
        self._L.orc_observe(self._h, _dp(out))
        keys = ["t", "mass_phi", "mass_psi", "xc", "yc", "ux_bub", "uy_bub", "U_o", "t_star"]
        return dict(zip(keys, out.tolist()))
