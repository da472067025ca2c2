"""Python binding of the C ABI in ``include/lbm.h`` (ctypes).

The functions keep the C names (``lbm_create``, ``lbm_init``, ``lbm_step``,
``lbm_observe``, ``lbm_destroy`` ...) and only marshal arguments: every step
of the computation runs in the CUDA kernels of ``_build/liblbm.so``.  There is
no fallback: if the library cannot be built or loaded, ``load()`` raises.

PyTorch is optional plumbing: ``Sim(..., workspace="torch")`` takes the
device workspace from PyTorch's caching allocator and ``stream=`` accepts a
``torch.cuda.Stream`` (or a raw ``cudaStream_t`` integer).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

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
    ("alpha_A", ctypes.c_double), ("precision", ctypes.c_int32),
    ("psi_L", ctypes.c_double), ("psi_R", ctypes.c_double), ("psi_bc", ctypes.c_int32),
]
# fields a parameter dict may leave out (0 if absent)
OPTIONAL = ("precision", "psi_L", "psi_R", "psi_bc")

OBS_FIELDS = ["t", "mass_phi", "mass_psi", "xc", "yc", "ux_bub", "uy_bub", "U_o", "t_star"]

DERIVED_NAMES = [
    "dT", "M1", "M2", "L", "U_o", "rho_A", "rho_B", "mu_A", "mu_B", "nu_A", "nu_B",
    "alpha_A", "alpha_B", "omega_phi", "omega_psi", "lambda", "s", "w", "m_psi", "D_psi",
]

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_ESTATE = (
    0, -1, -2, -3, -4, -5, -6)
# Population storage precision (lbm_params.precision).
LBM_FP32, LBM_FP16, LBM_BF16 = 0, 1, 2
PRECISIONS = {"fp32": LBM_FP32, "fp16": LBM_FP16, "bf16": LBM_BF16}
STATUS_NAMES = {0: "LBM_OK", -1: "LBM_EINVAL", -2: "LBM_ENOMEM", -3: "LBM_ECUDA",
                -4: "LBM_EUNSTABLE", -5: "LBM_ETIMEOUT", -6: "LBM_ESTATE"}

# Symbols include/lbm.h declares.
EXPORTS = [
    "lbm_derive", "lbm_workspace_bytes", "lbm_create", "lbm_create_ex", "lbm_init", "lbm_step",
    "lbm_step_batch", "lbm_batch_plan", "lbm_batch_tiles", "lbm_pin_batch_plan", "lbm_tune_batch",
    "lbm_observe", "lbm_observe_enqueue", "lbm_observe_collect",
    "lbm_get_populations", "lbm_get_derived", "lbm_launch_count",
    "lbm_destroy", "lbm_last_error", "lbm_reduce_observables_noalloc", "lbm_probe_bounded_wait",
]


class LbmParams(ctypes.Structure):
    _fields_ = PARAM_FIELDS


class LbmObs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in OBS_FIELDS] + [("nan_flag", ctypes.c_int32)]


class LbmError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def load() -> ctypes.CDLL:
    """Builds (if stale) and loads ``liblbm.so``; raises if that fails."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} missing after build")
            L = ctypes.CDLL(path)
            vp, sz = ctypes.c_void_p, ctypes.c_size_t
            PP = ctypes.POINTER(LbmParams)
            dp = ctypes.POINTER(ctypes.c_double)
            fp = ctypes.POINTER(ctypes.c_float)
            L.lbm_derive.argtypes = [PP, dp]
            L.lbm_workspace_bytes.argtypes = [PP, ctypes.POINTER(sz)]
            L.lbm_create.argtypes = [PP, vp, ctypes.POINTER(vp)]
            L.lbm_create_ex.argtypes = [PP, vp, vp, sz, ctypes.POINTER(vp)]
            L.lbm_init.argtypes = [vp, dp, fp]
            L.lbm_step.argtypes = [vp, ctypes.c_int64]
            L.lbm_step_batch.argtypes = [ctypes.POINTER(vp), ctypes.c_int32, ctypes.c_int64]
            L.lbm_batch_plan.argtypes = [ctypes.POINTER(vp), ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_int32)]
            i32p = ctypes.POINTER(ctypes.c_int32)
            L.lbm_batch_tiles.argtypes = [ctypes.POINTER(vp), ctypes.c_int32, i32p, i32p]
            L.lbm_pin_batch_plan.argtypes = [ctypes.POINTER(vp), ctypes.c_int32, i32p, i32p]
            L.lbm_tune_batch.argtypes = [ctypes.POINTER(vp), ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_int64)]
            L.lbm_observe.argtypes = [vp, ctypes.POINTER(LbmObs), dp]
            L.lbm_observe_enqueue.argtypes = [ctypes.POINTER(vp), ctypes.c_int32]
            L.lbm_observe_collect.argtypes = [ctypes.POINTER(vp), ctypes.c_int32,
                                              ctypes.POINTER(LbmObs),
                                              ctypes.POINTER(ctypes.c_int32)]
            L.lbm_get_populations.argtypes = [vp, fp]
            L.lbm_get_derived.argtypes = [vp, dp]
            L.lbm_launch_count.argtypes = [vp]
            L.lbm_launch_count.restype = ctypes.c_int64
            L.lbm_destroy.argtypes = [vp]
            L.lbm_destroy.restype = None
            L.lbm_reduce_observables_noalloc.argtypes = [vp, ctypes.c_int32, ctypes.c_int32,
                                                         ctypes.c_int32, vp, vp]
            L.lbm_probe_bounded_wait.argtypes = [ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)]
            L.lbm_last_error.argtypes = []
            L.lbm_last_error.restype = ctypes.c_char_p
            for name in EXPORTS:
                if name not in ("lbm_destroy", "lbm_last_error", "lbm_launch_count"):
                    getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def _check(status: int, where: str):
    if status != LBM_OK:
        raise LbmError(status, where, load().lbm_last_error().decode())


def make_params(d: dict) -> LbmParams:
    p = LbmParams()
    for name, _ in PARAM_FIELDS:
        setattr(p, name, d.get(name, 0) if name in OPTIONAL else d[name])
    return p


def _stream_handle(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


# ---- thin wrappers with the C names -------------------------------------------------

def lbm_derive(params: dict) -> dict:
    p = make_params(params)
    a = (ctypes.c_double * len(DERIVED_NAMES))()
    _check(load().lbm_derive(ctypes.byref(p), a), "lbm_derive")
    return dict(zip(DERIVED_NAMES, list(a)))


def lbm_workspace_bytes(params: dict) -> int:
    p = make_params(params)
    n = ctypes.c_size_t()
    _check(load().lbm_workspace_bytes(ctypes.byref(p), ctypes.byref(n)), "lbm_workspace_bytes")
    return int(n.value)


def lbm_create(params: dict, stream=None) -> ctypes.c_void_p:
    p = make_params(params)
    h = ctypes.c_void_p()
    _check(load().lbm_create(ctypes.byref(p), ctypes.c_void_p(_stream_handle(stream)),
                             ctypes.byref(h)), "lbm_create")
    return h


def lbm_create_ex(params: dict, stream, workspace_ptr: int, workspace_bytes: int):
    p = make_params(params)
    h = ctypes.c_void_p()
    _check(load().lbm_create_ex(ctypes.byref(p), ctypes.c_void_p(_stream_handle(stream)),
                                ctypes.c_void_p(workspace_ptr), workspace_bytes,
                                ctypes.byref(h)), "lbm_create_ex")
    return h


def lbm_init(sim, fields: np.ndarray | None = None, populations: np.ndarray | None = None):
    fptr = pptr = None
    if fields is not None:
        fields = np.ascontiguousarray(fields, dtype=np.float64)
        fptr = fields.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    if populations is not None:
        populations = np.ascontiguousarray(populations, dtype=np.float32)
        pptr = populations.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    _check(load().lbm_init(sim, fptr, pptr), "lbm_init")


def lbm_step(sim, nsteps: int):
    _check(load().lbm_step(sim, int(nsteps)), "lbm_step")


def _handles(sims):
    hs = [s.handle if isinstance(s, Sim) else s for s in sims]
    return (ctypes.c_void_p * len(hs))(*[h.value if isinstance(h, ctypes.c_void_p) else h
                                         for h in hs]), len(hs)


def lbm_step_batch(sims, nsteps: int):
    """One launch per step over every simulation in `sims` (handles or Sim)."""
    arr, n = _handles(sims)
    _check(load().lbm_step_batch(arr, n, int(nsteps)), "lbm_step_batch")


def lbm_batch_plan(sims) -> list[int]:
    """Strip length (in chunks of the tile shape's rows) lbm_step_batch uses
    for each sim; 0 for sims stepped by the tile kernel."""
    arr, n = _handles(sims)
    out = (ctypes.c_int32 * n)()
    _check(load().lbm_batch_plan(arr, n, out), "lbm_batch_plan")
    return list(out)


def lbm_batch_tiles(sims) -> list[tuple[int, int]]:
    """(column width, chunk rows) of the streaming tile shape each sim is
    stepped in; (0, 0) for sims stepped by the tile kernel."""
    arr, n = _handles(sims)
    w, h = (ctypes.c_int32 * n)(), (ctypes.c_int32 * n)()
    _check(load().lbm_batch_tiles(arr, n, w, h), "lbm_batch_tiles")
    return list(zip(list(w), list(h)))


def lbm_pin_batch_plan(sims, tile_w, strip_chunks):
    """Sets the batch's plan: tile width (32 or 64) and strip length of every
    streaming sim (entries of the others are ignored)."""
    arr, n = _handles(sims)
    w = (ctypes.c_int32 * n)(*[int(x) for x in tile_w])
    c = (ctypes.c_int32 * n)(*[int(x) for x in strip_chunks])
    _check(load().lbm_pin_batch_plan(arr, n, w, c), "lbm_pin_batch_plan")


def lbm_tune_batch(sims, trial_steps: int) -> int:
    """Times every candidate strip plan on the batch for trial_steps steps and
    keeps the fastest; returns the number of steps every sim advanced."""
    arr, n = _handles(sims)
    taken = ctypes.c_int64(0)
    _check(load().lbm_tune_batch(arr, n, int(trial_steps), ctypes.byref(taken)), "lbm_tune_batch")
    return int(taken.value)


def lbm_observe(sim, host_fields: np.ndarray | None = None, check: bool = True) -> dict:
    ob = LbmObs()
    fptr = None
    if host_fields is not None:
        assert host_fields.dtype == np.float64 and host_fields.flags["C_CONTIGUOUS"]
        fptr = host_fields.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = load().lbm_observe(sim, ctypes.byref(ob), fptr)
    if check:
        _check(st, "lbm_observe")
    out = {n: getattr(ob, n) for n in OBS_FIELDS}
    out["nan_flag"] = ob.nan_flag
    out["status"] = st
    return out


def lbm_observe_enqueue(sims):
    """Enqueues the observables of every sim (one stream) without waiting."""
    arr, n = _handles(sims)
    _check(load().lbm_observe_enqueue(arr, n), "lbm_observe_enqueue")


def lbm_observe_collect(sims) -> list[dict]:
    """Waits for the observables lbm_observe_enqueue enqueued and returns one
    dict per sim (with its 'status')."""
    arr, n = _handles(sims)
    obs = (LbmObs * n)()
    st = (ctypes.c_int32 * n)()
    _check(load().lbm_observe_collect(arr, n, obs, st), "lbm_observe_collect")
    out = []
    for i in range(n):
        d = {k: getattr(obs[i], k) for k in OBS_FIELDS}
        d["nan_flag"] = obs[i].nan_flag
        d["status"] = int(st[i])
        out.append(d)
    return out


def lbm_get_populations(sim, out: np.ndarray):
    assert out.dtype == np.float32 and out.flags["C_CONTIGUOUS"]
    _check(load().lbm_get_populations(sim, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
           "lbm_get_populations")


def lbm_get_derived(sim) -> dict:
    a = (ctypes.c_double * len(DERIVED_NAMES))()
    _check(load().lbm_get_derived(sim, a), "lbm_get_derived")
    return dict(zip(DERIVED_NAMES, list(a)))


def lbm_launch_count(sim) -> int:
    return int(load().lbm_launch_count(sim))


def lbm_destroy(sim):
    load().lbm_destroy(sim)


def lbm_probe_bounded_wait(limit_ns: int) -> bool:
    """True if a block waiting on a barrier that never completes gave up after
    limit_ns nanoseconds (the kernels' bounded wait; see include/lbm.h)."""
    flag = ctypes.c_int32(0)
    _check(load().lbm_probe_bounded_wait(int(limit_ns), ctypes.byref(flag)),
           "lbm_probe_bounded_wait")
    return bool(flag.value)


def lbm_reduce_observables_noalloc(d_fields_ptr: int, nx: int, ny: int, walls: int,
                                   d_sums_ptr: int, stream=None):
    """Observable sums of a device field array into a device array of 8
    doubles, without any device allocation (see include/lbm.h)."""
    _check(load().lbm_reduce_observables_noalloc(
        ctypes.c_void_p(d_fields_ptr), int(nx), int(ny), int(walls),
        ctypes.c_void_p(d_sums_ptr), ctypes.c_void_p(_stream_handle(stream))),
        "lbm_reduce_observables_noalloc")


# ---- convenience object ---------------------------------------------------------------

class Sim:
    """One simulation on the current CUDA device.

    ``workspace="library"`` lets the library cudaMalloc its workspace;
    ``workspace="torch"`` takes it from PyTorch's allocator.
    """

    def __init__(self, params: dict, stream=None, workspace: str = "library"):
        self.params = dict(params)
        self.nx, self.ny = int(params["nx"]), int(params["ny"])
        self._ws = None
        if workspace == "torch":
            import torch
            nbytes = lbm_workspace_bytes(params)
            self._ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            self._h = lbm_create_ex(params, stream, self._ws.data_ptr(), nbytes)
        elif workspace == "library":
            self._h = lbm_create(params, stream)
        else:
            raise ValueError(workspace)

    def close(self):
        if getattr(self, "_h", None):
            lbm_destroy(self._h)
            self._h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    def init(self, fields=None, populations=None):
        lbm_init(self._h, fields, populations)

    def step(self, n: int = 1):
        lbm_step(self._h, n)

    def observe(self, check: bool = True) -> dict:
        return lbm_observe(self._h, None, check=check)

    def fields(self) -> np.ndarray:
        out = np.zeros((6, self.ny, self.nx))
        lbm_observe(self._h, out)
        return out

    def populations(self) -> np.ndarray:
        out = np.zeros((4, 9, self.ny, self.nx), dtype=np.float32)
        lbm_get_populations(self._h, out)
        return out

    def derived(self) -> dict:
        return lbm_get_derived(self._h)

    def launches(self) -> int:
        return lbm_launch_count(self._h)
