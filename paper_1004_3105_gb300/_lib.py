"""Loads libnrng.so (built in-tree by paper_1004_3105_gb300.build) and declares
the ctypes signatures of every entry point of include/nrng.h.

There is no fallback: if the library is missing or fails to load, every call
raises.  Nothing here computes; it only marshals arguments.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

STATUS = {
    0: "NRNG_OK", 1: "NRNG_ERR_INVALID_VALUE", 2: "NRNG_ERR_MISALIGNED", 3: "NRNG_ERR_WORKSPACE",
    4: "NRNG_ERR_COUNTER_OVERFLOW", 5: "NRNG_ERR_CUDA", 6: "NRNG_ERR_TIMEOUT",
    7: "NRNG_ERR_EXHAUSTED", 8: "NRNG_ERR_NOT_SUPPORTED",
}
OK, ERR_INVALID_VALUE, ERR_MISALIGNED, ERR_WORKSPACE, ERR_COUNTER_OVERFLOW, ERR_CUDA, \
    ERR_TIMEOUT, ERR_EXHAUSTED, ERR_NOT_SUPPORTED = range(9)


class NrngError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        msg = load().nrng_status_string(int(status)).decode()
        super().__init__(f"{where}: {msg}" if where else msg)


_P = ctypes.c_void_p
_I32, _I64, _U64, _F32, _SZ = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_float, ctypes.c_size_t
_PSZ = ctypes.POINTER(ctypes.c_size_t)
_PU64 = ctypes.POINTER(ctypes.c_uint64)
_PI32 = ctypes.POINTER(ctypes.c_int32)
_PF32 = ctypes.POINTER(ctypes.c_float)

SIGNATURES = {
    "nrng_status_string": (ctypes.c_char_p, [_I32]),
    "nrng_abi_version": (_I32, []),
    "nrng_uniform": (_I32, [_P, _I64, _U64, _U64, _P]),
    "nrng_philox_ceiling": (_I32, [_P, _I64, _U64, _U64, _P]),
    "nrng_boxmuller": (_I32, [_P, _I64, _F32, _F32, _U64, _U64, _I32, _I32, _P]),
    "nrng_polar_workspace_size": (_I32, [_I64, _PSZ]),
    "nrng_polar_max_blocks": (_I32, [_I64, _PU64]),
    "nrng_polar": (_I32, [_P, _I64, _F32, _F32, _U64, _U64, _I32, _I32, _P, _SZ, _P, _P, _P]),
    "nrng_polar_noalloc": (_I32, [_P, _I64, _F32, _F32, _U64, _U64, _I32, _I32, _P, _P, _P, _P]),
    "nrng_polar_twopass_workspace_size": (_I32, [_I64, _PSZ]),
    "nrng_polar_twopass": (_I32, [_P, _I64, _F32, _F32, _U64, _U64, _I32, _I32, _P, _SZ, _P, _P, _P]),
    "nrng_boxmuller_b3": (_I32, [_P, _I64, _F32, _F32, _U64, _U64, _I32, _P]),
    "nrng_polar_p2": (_I32, [_P, _I64, _F32, _F32, _U64, _U64, _I32, _P, _SZ, _P, _P, _P]),
    "nrng_ratio_workspace_size": (_I32, [_I64, _PSZ]),
    "nrng_ratio": (_I32, [_P, _I64, _F32, _F32, _U64, _U64, _I32, _I32, _P, _SZ, _P, _P, _P]),
    "nrng_eval_points": (_I32, [_I32, _I32, _P, _I64, _F32, _F32, _P, _P, _P]),
    "nrng_batched_workspace_size": (_I32, [_P, _I32, _PSZ]),
    "nrng_batched": (_I32, [_P, _P, _I32, _I32, _I32, _P, _SZ, _P]),
    "nrng_reparam_fwd": (_I32, [_P, _P, _P, _I64, _I64, _I64, _U64, _U64, _I32, _P]),
    "nrng_reparam_bwd": (_I32, [_P, _P, _P, _I64, _I64, _I64, _U64, _U64, _I32, _P]),
    "nrng_get_status": (_I32, [_P, _P, _PI32]),
    "nrng_batched_config_count": (_I32, []),
    "nrng_batched_config_info": (_I32, [_I32, _PI32, _PI32]),
    "nrng_batched_set_config": (_I32, [_I32, _I32, _I32]),
    "nrng_batched_get_config": (_I32, [_I32, _I32, _PI32]),
    "nrng_batched_autotune": (_I32, [_P, _P, _I32, _I32, _I32, _P, _SZ, _I32, _P, _PI32, _PF32]),
    "nrng_batched_graph_create": (_I32, [_P, _P, _I32, _I32, _I32, _P, _SZ, _P, ctypes.POINTER(_P)]),
    "nrng_graph_launch": (_I32, [_P, _P]),
    "nrng_graph_destroy": (_I32, [_P]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """The loaded library.  Raises if it has not been built (or cannot load)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if build_if_missing:
                _build.build()
            else:
                raise RuntimeError(
                    f"libnrng.so is not built ({path}); run "
                    "`python -c 'import __graft_entry__ as g; g.build()'` first. "
                    "There is no CPU fallback.")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(status: int, where: str = "") -> None:
    if int(status) != OK:
        raise NrngError(status, where)
