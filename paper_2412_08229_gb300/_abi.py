"""ctypes declarations of include/lbm.h and the loader of the in-tree liblbm.so.

Argument marshalling only: every computation runs in the CUDA library. There is no
CPU fallback; if the library is missing and cannot be built, load() raises.
"""

import ctypes
import os
import re
from ctypes import POINTER, c_char_p, c_double, c_float, c_int, c_void_p

from . import build as _build

LBM_OK = 0
LBM_ERR_ARG = -1
LBM_ERR_CUDA = -2
LBM_ERR_OOM = -3
LBM_ERR_UNSTABLE = -4
LBM_ERR_TIMEOUT = -5
LBM_ERR_STATE = -6

OPS = {"bgk": 0, "kbc": 1, "nco": 2, "reg": 3}
STORAGES = {"f32": 0, "f16": 1, "bf16": 2}
NETS = {"f32": 0, "bf16": 1, "bf16x3": 2}
BOUNDARIES = {"periodic": 0, "mirror": 1, "tgv_reduced": 2}

STATUS_NAMES = {0: "LBM_OK", -1: "LBM_ERR_ARG", -2: "LBM_ERR_CUDA", -3: "LBM_ERR_OOM",
                -4: "LBM_ERR_UNSTABLE", -5: "LBM_ERR_TIMEOUT", -6: "LBM_ERR_STATE"}


class lbm_config(ctypes.Structure):
    _fields_ = [
        ("nx", c_int), ("ny", c_int), ("nz", c_int),
        ("nu", c_double),
        ("op", c_int), ("storage", c_int), ("net_precision", c_int), ("boundary", c_int),
        ("forcing", c_int),
        ("force_power", c_double), ("force_kf", c_double), ("force_c", c_double),
        ("force_ka", c_double), ("force_kb", c_double),
        ("rho_min", c_double), ("rho_max", c_double),
    ]


_CTX = c_void_p
_SIGNATURES = {
    "lbm_create": (c_int, [POINTER(lbm_config), c_void_p, POINTER(_CTX)]),
    "lbm_destroy": (c_int, [_CTX]),
    "lbm_last_error": (c_char_p, [_CTX]),
    "lbm_init": (c_int, [_CTX, c_void_p, c_void_p]),
    "lbm_set_state": (c_int, [_CTX, c_void_p]),
    "lbm_get_state": (c_int, [_CTX, c_void_p]),
    "lbm_step": (c_int, [_CTX, c_int]),
    "lbm_check": (c_int, [_CTX]),
    "lbm_set_wait_limit": (c_int, [_CTX, ctypes.c_longlong]),
    "lbm_macroscopic": (c_int, [_CTX, c_void_p, c_void_p]),
    "lbm_kinetic_energy": (c_int, [_CTX, c_void_p]),
    "lbm_energy_spectrum": (c_int, [_CTX, c_void_p, c_int, c_void_p]),
    "nco_set_weights": (c_int, [_CTX, c_void_p, c_int]),
    "lbm_force_draws": (c_int, [_CTX, c_void_p, c_void_p, c_int]),
    "lbm_get_force_state": (c_int, [_CTX, c_void_p]),
    "lbm_raw_state_bytes": (ctypes.c_longlong, [_CTX]),
    "lbm_get_raw_state": (c_int, [_CTX, c_void_p]),
    "lbm_set_raw_state": (c_int, [_CTX, c_void_p]),
    "lbm_check_guards": (c_int, [_CTX]),
    "lbm_selftest_guards": (c_int, [_CTX]),
    "lbm_set_force_state": (c_int, [_CTX, c_void_p]),
    "lbm_record_begin": (c_int, [_CTX, c_int]),
    "nco_backward": (c_int, [_CTX, c_void_p, c_void_p, c_void_p, c_void_p]),
    "nco_backward_ke": (c_int, [_CTX, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "lbm_group_tables": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "lbm_spectrum_shells": (c_int, [c_int, c_int, c_int, c_void_p]),
    "lbm_tgv_reduced_table": (c_int, [c_void_p, c_void_p, c_void_p]),
    "lbm_version": (c_char_p, []),
    "lbm_selftest_tensor_cores": (c_int, [POINTER(c_double)]),
    "lbm_kinetic_energy_noalloc": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p]),
    "lbm_batch_create": (c_int, [c_int, POINTER(lbm_config), c_void_p, POINTER(c_void_p)]),
    "lbm_batch_destroy": (c_int, [c_void_p]),
    "lbm_batch_last_error": (c_char_p, [c_void_p]),
    "lbm_batch_get": (c_int, [c_void_p, c_int, POINTER(_CTX)]),
    "lbm_batch_set_weights": (c_int, [c_void_p, c_void_p, c_int]),
    "lbm_batch_autotune": (c_int, [c_void_p, POINTER(c_int)]),
    "lbm_batch_set_tile_shape": (c_int, [c_void_p, c_int]),
    "lbm_batch_step": (c_int, [c_void_p, c_int, c_int]),
    "lbm_batch_check": (c_int, [c_void_p]),
}

_lib = None


def header_functions():
    """Names of every function declared in include/lbm.h."""
    path = os.path.join(_build.ROOT, "include", "lbm.h")
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_]+\**\s+\**\s*([a-z_0-9]+)\s*\(", text, flags=re.M)))


def load(build_if_missing=True):
    """Load liblbm.so (building it in-tree first if it is missing or stale).

    NCO_LBM_LIBRARY, if set, names another build of the same ABI to load instead."""
    global _lib
    if _lib is not None:
        return _lib
    path = os.environ.get("NCO_LBM_LIBRARY")  # an explicitly chosen build of the same ABI
    if not path:
        if build_if_missing and _build.is_stale():
            _build.build()
        path = _build.LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class LbmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def check(status, ctx=None, what="", batch=None):
    if status != LBM_OK:
        if batch is not None:
            msg = load().lbm_batch_last_error(batch).decode()
        else:
            msg = load().lbm_last_error(ctx).decode() if ctx is not None else ""
        raise LbmError(status, f"{what} {msg}".strip())
    return status
