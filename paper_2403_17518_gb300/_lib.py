"""ctypes view of the C ABI in include/dhfwi.h (argument marshalling only).

Loading fails loudly when the compiled library is missing: there is no CPU
or PyTorch fallback for any call.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdhfwi.so")

DHFWI_OK = 0
ERRORS = {
    -1: "DHFWI_ERR_ARG",
    -2: "DHFWI_ERR_GEOM",
    -3: "DHFWI_ERR_CFL",
    -4: "DHFWI_ERR_NONFINITE",
    -5: "DHFWI_ERR_OOM",
    -6: "DHFWI_ERR_TIMEOUT",
    -7: "DHFWI_ERR_CUDA",
    -8: "DHFWI_ERR_STATE",
}
DHFWI_ABS = 0
DHFWI_REL = 1

_IP = ctypes.POINTER(ctypes.c_int)
_FP = ctypes.POINTER(ctypes.c_float)
_VP = ctypes.c_void_p


class Grid(ctypes.Structure):
    _fields_ = [("nz", ctypes.c_int), ("nx", ctypes.c_int), ("nb", ctypes.c_int),
                ("h", ctypes.c_float), ("dt", ctypes.c_float)]


class Geom(ctypes.Structure):
    _fields_ = [("n_shots", ctypes.c_int), ("src_iz", _IP), ("src_ix", _IP), ("nt", _IP),
                ("rec_off", _IP), ("rec_iz", _IP), ("rec_ix", _IP), ("win_x0", _IP), ("win_x1", _IP),
                ("wavelet", _FP), ("nt_max", ctypes.c_int), ("wavelet_shared", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("cell_updates", ctypes.c_longlong), ("kernel_launches", ctypes.c_longlong),
                ("checkpoint_every", ctypes.c_int), ("shot_groups", ctypes.c_int),
                ("workspace_bytes", ctypes.c_double), ("phase_ms", ctypes.c_double * 3),
                ("phase_launches", ctypes.c_longlong * 3), ("phase_cells", ctypes.c_longlong * 3),
                ("step_variant", ctypes.c_int * 4), ("history_steps", ctypes.c_int),
                ("history_cells", ctypes.c_longlong), ("time_block", ctypes.c_int * 2), ("reused", ctypes.c_int)]


class TrainCfg(ctypes.Structure):
    _fields_ = [("base_channels", ctypes.c_int), ("levels", ctypes.c_int), ("patch", ctypes.c_int),
                ("stride", ctypes.c_int), ("batch", ctypes.c_int), ("epochs", ctypes.c_int),
                ("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("seed", ctypes.c_ulonglong), ("mute_rows", ctypes.c_int),
                ("warmup_frac", ctypes.c_float)]


_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) of every exported C function.
SIGNATURES = [
    ("dhfwi_create", ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(Grid), ctypes.c_int]),
    ("dhfwi_destroy", None, [_VP]),
    ("dhfwi_last_error", ctypes.c_char_p, [_VP]),
    ("dhfwi_stats", ctypes.c_int, [_VP, ctypes.POINTER(Stats)]),
    ("dhfwi_set_timing", ctypes.c_int, [_VP, ctypes.c_int]),
    ("dhfwi_set_reuse", ctypes.c_int, [_VP, ctypes.c_int]),
    ("model_shots", ctypes.c_int, [_VP, _VP, ctypes.POINTER(Geom), _VP, _VP]),
    ("fwi_gradient", ctypes.c_int, [_VP, _VP, ctypes.POINTER(Geom), _VP, _VP,
                                    ctypes.POINTER(ctypes.c_double), _VP, _VP]),
    ("born_demig", ctypes.c_int, [_VP, _VP, ctypes.POINTER(Geom), _VP, _VP, ctypes.c_int, _VP]),
    ("rtm_mig", ctypes.c_int, [_VP, _VP, ctypes.POINTER(Geom), _VP, _VP, ctypes.c_int, _VP]),
    ("fwi_update", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_int,
                                  _VP, _VP]),
    ("bb_step", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double), _VP]),
    ("data_misfit", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_longlong, ctypes.POINTER(ctypes.c_double), _VP]),
    ("image_laplacian", ctypes.c_int, [_VP, _VP, _VP, _VP]),
    ("dhfwi_selftest_timeout", ctypes.c_int, [_VP, _VP]),
    ("model_shots_static", ctypes.c_int, [ctypes.POINTER(Grid), _VP, ctypes.POINTER(Geom), _VP, _VP]),
    ("model_shots_static_error", ctypes.c_char_p, []),
    ("dhfwi_net_init", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong]),
    ("dhfwi_net_size", ctypes.c_longlong, [_VP]),
    ("dhfwi_net_get", ctypes.c_int, [_VP, _FP, ctypes.c_size_t]),
    ("dhfwi_net_set", ctypes.c_int, [_VP, _FP, ctypes.c_size_t]),
    ("deblur_forward", ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP]),
    ("deblur_grad", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP,
                                   ctypes.POINTER(ctypes.c_double), _VP]),
    ("deblur_train", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(TrainCfg),
                                    ctypes.c_int, _FP, _VP]),
    ("deblur_apply", ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, _VP, _VP]),
    ("deblur_layer", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, _VP, _VP, _VP, _VP, _VP, _VP]),
]
OPTIONAL = {}


def load(path: str | None = None):
    """Load libdhfwi.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with paper_2403_17518_gb300.build.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(p)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        for name, (res, args) in OPTIONAL.items():
            if hasattr(L, name):
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
        _lib = L
        return L


class DhfwiError(RuntimeError):
    def __init__(self, code: int, msg: str):
        self.code = code
        self.name = ERRORS.get(code, str(code))
        super().__init__(f"{self.name}: {msg}")
