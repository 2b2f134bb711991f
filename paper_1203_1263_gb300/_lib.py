"""ctypes binding of libnlse.so (include/nlse.h): argument marshalling only.

The library is built in-tree on first use when it is missing or stale.  There
is no CPU fallback: if the CUDA library cannot be built or loaded, every call
raises.
"""
from __future__ import annotations

import ctypes
import threading

from . import build as _build

NLSE_OK = 0
NLSE_EINVAL = -1
NLSE_ENOMEM = -2
NLSE_ECUDA = -3
NLSE_EUNSTABLE = -4
NLSE_ENONFINITE = -5
NLSE_ETIMEOUT = -6
NLSE_ESTATE = -7

BC_DIRICHLET = 0
BC_MSD = 1
BC_L0 = 2
BC_PERIODIC = 3
C128 = 0
C64 = 1
C64_ACC64 = 2
DEBUG_SPIN_LIMIT = 1
DEBUG_EXTRA_TX = 2
DEBUG_FIX_OFFSET = 3

STATUS_NAMES = {0: "NLSE_OK", -1: "NLSE_EINVAL", -2: "NLSE_ENOMEM", -3: "NLSE_ECUDA", -4: "NLSE_EUNSTABLE",
                -5: "NLSE_ENONFINITE", -6: "NLSE_ETIMEOUT", -7: "NLSE_ESTATE"}

# name -> (restype, argtypes); the exported entry points of include/nlse.h
_I64P = ctypes.POINTER(ctypes.c_int64)
_VP = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
SIGNATURES = {
    "nlse_workspace_bytes": (ctypes.c_size_t, [_I, _I64P, _I]),
    "nlse_create": (_I, [ctypes.POINTER(_VP), _I, _I64P, _D, _D, _D, _VP, _I, _I, _I, _VP, _VP, ctypes.c_size_t,
                         _VP]),
    "nlse_step": (_I, [_VP, ctypes.c_int64, _D]),
    "nlse_refresh_potential": (_I, [_VP]),
    "nlse_mass": (_I, [_VP, ctypes.POINTER(_D)]),
    "nlse_energy": (_I, [_VP, ctypes.POINTER(_D)]),
    "nlse_rhs": (_I, [_VP, _VP, _VP]),
    "nlse_max_dt": (_D, [_I, _D, _D, _I, _D, _D]),
    "nlse_sync": (_I, [_VP]),
    "nlse_destroy": (_I, [_VP]),
    "nlse_last_error": (ctypes.c_char_p, []),
    "nlse_set_kernel": (_I, [_VP, _I, _I]),
    "nlse_kernel_in_use": (_I, [_VP]),
    "nlse_debug_set": (_I, [_VP, _I, ctypes.c_longlong]),
    "nlse_autotune": (_I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_float)]),
    "nlse_mass_noalloc": (_I, [_I, _I64P, _D, _I, _VP, _VP, _VP]),
    "nlse_batch_workspace_bytes": (ctypes.c_size_t, [_I, _VP]),
    "nlse_batch_create": (_I, [ctypes.POINTER(_VP), _I, _VP, _VP, ctypes.c_size_t, _VP]),
    "nlse_batch_step": (_I, [_VP, ctypes.c_int64]),
    "nlse_batch_set_tile": (_I, [_VP, _I]),
    "nlse_batch_autotune": (_I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_float)]),
    "nlse_batch_sync": (_I, [_VP]),
    "nlse_batch_destroy": (_I, [_VP]),
    "nlse_sur_param_count": (ctypes.c_size_t, [_I, _I]),
    "nlse_sur_workspace_bytes": (ctypes.c_size_t, [_I, _I, _I, _I, _I]),
    "nlse_sur_create": (_I, [ctypes.POINTER(_VP), _I, _I, _I, _I, ctypes.POINTER(_I), _I, _VP, _VP, ctypes.c_size_t,
                             _VP]),
    "nlse_sur_init": (_I, [_VP, ctypes.c_uint64]),
    "nlse_sur_sync_params": (_I, [_VP]),
    "nlse_sur_forward": (_I, [_VP, _I, _VP, _VP, _I, _VP]),
    "nlse_sur_set_mass_weight": (_I, [_VP, _D]),
    "nlse_sur_compare": (_I, [_VP, _I, _VP, _VP, ctypes.POINTER(_D)]),
    "nlse_sur_gradients": (_I, [_VP, _I, _VP, _VP, _VP, ctypes.POINTER(_D)]),
    "nlse_sur_train_step": (_I, [_VP, _I, _VP, _VP, ctypes.c_float, ctypes.c_float, ctypes.POINTER(_D)]),
    "nlse_sur_set_kernel": (_I, [_VP, _I]),
    "nlse_sur_sync": (_I, [_VP]),
    "nlse_sur_destroy": (_I, [_VP]),
}


class RunDesc(ctypes.Structure):
    """nlse_run_desc of include/nlse.h."""
    _fields_ = [("n", ctypes.c_int64 * 2), ("h", ctypes.c_double), ("a", ctypes.c_double), ("s", ctypes.c_double),
                ("dt", ctypes.c_double), ("bc", ctypes.c_int), ("order", ctypes.c_int), ("psi", ctypes.c_void_p),
                ("V", ctypes.c_void_p)]


class NLSEError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def lib(build_if_needed: bool = True):
    """The loaded CUDA library (raises if it cannot be built or loaded)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_needed else _build.LIB
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(rc: int) -> None:
    if rc != NLSE_OK:
        raise NLSEError(rc, lib().nlse_last_error().decode(errors="replace"))


def int64_array(vals):
    return (ctypes.c_int64 * len(vals))(*[int(v) for v in vals])
