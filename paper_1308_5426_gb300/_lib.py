"""ctypes binding of libpotts_lr.so (include/potts_lr.h).

Argument marshalling only: every step of the simulation runs in the library's
CUDA kernels.  There is no fallback -- if the library cannot be loaded, or no
GPU is present when a job is created, the call raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpotts_lr.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ESTATE = 0, 1, 2, 3, 4, 5
NEAR_LOG_CAP = 256  # POTTS_LR_NEAR_LOG_CAP
FP64, FP32, FX64 = 0, 1, 2
PRECISIONS = {"fp64": FP64, "fp32": FP32, "fx64": FX64}

# every entry point the header declares (checked by the ABI test)
EXPORTS = [
    "potts_lr_default_opts", "potts_lr_create", "potts_lr_sweep", "potts_lr_exchange",
    "potts_lr_measure", "potts_lr_measure_device", "potts_lr_fields_recompute",
    "potts_lr_fields_error", "potts_lr_get_state", "potts_lr_set_state", "potts_lr_get_spins",
    "potts_lr_get_fields", "potts_lr_get_energy", "potts_lr_stats", "potts_lr_counters",
    "potts_lr_sync", "potts_lr_destroy", "potts_lr_last_error", "potts_lr_jstar",
    "potts_lr_batch_create", "potts_lr_batch_run", "potts_lr_batch_sync", "potts_lr_batch_destroy",
    "potts_lr_batch_sweep", "potts_lr_batch_exchange", "potts_lr_batch_measure",
    "potts_lr_batch_measure_device", "potts_lr_batch_state_size", "potts_lr_batch_get_state",
    "potts_lr_batch_set_state", "potts_lr_probe", "potts_lr_measure_static", "potts_lr_near_log",
    "potts_lr_set_wait_limits", "potts_lr_sweep_info", "potts_lr_set_rebuild_split", "potts_lr_rebuild_info",
]


class PottsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("potts_lr error %d: %s" % (code, msg))
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("recompute_every", ctypes.c_int),
                ("pair_factor", ctypes.c_int), ("cuda_stream", ctypes.c_void_p), ("sweep_variant", ctypes.c_int),
                ("site_order", ctypes.c_int)]


_lib = None


def load(path: str = LIB_PATH):
    """Load the library (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("libpotts_lr.so not built at %s (run __graft_entry__.build())" % path)
    lib = ctypes.CDLL(path)
    P, I, D, U64, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_size_t
    sig = {
        "potts_lr_default_opts": [P],
        "potts_lr_create": [I, I, D, P, I, U64, P, P],
        "potts_lr_sweep": [P, I],
        "potts_lr_exchange": [P],
        "potts_lr_measure": [P, P, P],
        "potts_lr_measure_device": [P, P, P],
        "potts_lr_fields_recompute": [P],
        "potts_lr_fields_error": [P, P],
        "potts_lr_get_state": [P, P, P],
        "potts_lr_set_state": [P, P, SZ],
        "potts_lr_get_spins": [P, P],
        "potts_lr_get_fields": [P, P],
        "potts_lr_get_energy": [P, P],
        "potts_lr_stats": [P, P, P, P],
        "potts_lr_counters": [P, P, P],
        "potts_lr_sync": [P],
        "potts_lr_jstar": [I, D, P],
        "potts_lr_batch_create": [P, I, P, P],
        "potts_lr_batch_run": [P, I, I],
        "potts_lr_batch_sync": [P],
        "potts_lr_batch_sweep": [P, I],
        "potts_lr_batch_exchange": [P],
        "potts_lr_batch_measure": [P, P, P],
        "potts_lr_batch_measure_device": [P, P, P],
        "potts_lr_batch_state_size": [P, P],
        "potts_lr_batch_get_state": [P, P, SZ],
        "potts_lr_batch_set_state": [P, P, SZ],
        "potts_lr_probe": [I, P],
        "potts_lr_measure_static": [P, I, I, I, P, I, P, P, P],
        "potts_lr_near_log": [P, P, I, P],
        "potts_lr_set_wait_limits": [P, U64, U64],
        "potts_lr_sweep_info": [P, P, I],
        "potts_lr_set_rebuild_split": [P, I],
        "potts_lr_rebuild_info": [P, P, P, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = I
    lib.potts_lr_destroy.argtypes = [P]
    lib.potts_lr_destroy.restype = None
    lib.potts_lr_batch_destroy.argtypes = [P]
    lib.potts_lr_batch_destroy.restype = None
    lib.potts_lr_last_error.argtypes = []
    lib.potts_lr_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def check(rc: int):
    if rc != OK:
        raise PottsError(rc, _lib.potts_lr_last_error().decode(errors="replace"))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)
