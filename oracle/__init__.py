"""FP64 CPU oracle for the FWI operators and the deblurring network.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package's
``__graft_entry__.smoke()`` check and by the CPU-baseline leg of ``bench.py``.
The product path never imports it, and it imports nothing from the product
package.

* ``fd2d.c`` (plain C, float64): forward modelling, misfit, adjoint-state
  gradient, Born demigration and migration, following Section 2.1 Eqs. 1-2,
  Section 2.2 Eqs. 9-12b and Section 2.3.1 Eqs. 13-15 of arXiv 2403.17518.
* ``nn.py`` (numpy float64 with bfloat16 operand rounding): the U-Net of
  Section 2.4 / Appendix A, its MSE loss, backward pass and Adam with cosine
  annealing.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (float64, no FP contraction, OpenMP over shots)."""
    src = [os.path.join(_HERE, "fd2d.c")]
    if not force and os.path.exists(_LIB_PATH):
        if all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(p) for p in src + [os.path.join(_HERE, "oracle.h")]):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-std=c99", *src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Grid(ctypes.Structure):
    _fields_ = [("nz", ctypes.c_int), ("nx", ctypes.c_int), ("nb", ctypes.c_int),
                ("h", ctypes.c_double), ("dt", ctypes.c_double)]


_IP = ctypes.POINTER(ctypes.c_int)
_DP = ctypes.POINTER(ctypes.c_double)


class _Geom(ctypes.Structure):
    _fields_ = [("n_shots", ctypes.c_int), ("src_iz", _IP), ("src_ix", _IP), ("nt", _IP),
                ("rec_off", _IP), ("rec_iz", _IP), ("rec_ix", _IP), ("win_x0", _IP),
                ("win_x1", _IP), ("wavelet", _DP), ("nt_max", ctypes.c_int),
                ("wavelet_shared", ctypes.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            GP = ctypes.POINTER(_Grid)
            GE = ctypes.POINTER(_Geom)
            L.or_model_shots.argtypes = [GP, _DP, GE, _DP]
            L.or_model_shots.restype = None
            L.or_fwi_gradient.argtypes = [GP, _DP, GE, _DP, _DP, _DP, ctypes.c_int]
            L.or_fwi_gradient.restype = ctypes.c_double
            L.or_born_demig.argtypes = [GP, _DP, GE, _DP, _DP]
            L.or_born_demig.restype = None
            L.or_rtm_mig.argtypes = [GP, _DP, GE, _DP, _DP, ctypes.c_int]
            L.or_rtm_mig.restype = None
            L.or_apply_lap.argtypes = [ctypes.c_int, ctypes.c_int, _DP, _DP]
            L.or_apply_lap.restype = None
            L.or_sponge.argtypes = [GP, ctypes.c_int, _DP]
            L.or_sponge.restype = None
            _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_DP)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_IP)


class _Args:
    """Keeps numpy buffers alive while ctypes structs point at them."""

    def __init__(self, nz, nx, h, dt, nb, geom):
        self.grid = _Grid(int(nz), int(nx), int(nb), float(h), float(dt))
        keep = []

        def ip(x):
            a, p = _i(x)
            keep.append(a)
            return p

        wav, wp = _d(geom.wavelet)
        keep.append(wav)
        self.geom = _Geom(geom.n_shots, ip(geom.src_iz), ip(geom.src_ix), ip(geom.nt),
                          ip(geom.rec_off), ip(geom.rec_iz), ip(geom.rec_ix), ip(geom.win_x0),
                          ip(geom.win_x1), wp, int(wav.shape[-1]), 1 if geom.wavelet_shared else 0)
        self.keep = keep


def _check_geom(nz, nx, geom):
    if np.any(geom.win_x0 < 0) or np.any(geom.win_x1 > nx) or np.any(geom.win_x1 <= geom.win_x0):
        raise ValueError("bad window")
    if geom.wavelet.shape[-1] < geom.nt_max:
        raise ValueError("wavelet shorter than the longest record")
    for s in range(geom.n_shots):
        a, b = int(geom.rec_off[s]), int(geom.rec_off[s + 1])
        for iz, ix in [(geom.src_iz[s], geom.src_ix[s])] + list(zip(geom.rec_iz[a:b], geom.rec_ix[a:b])):
            if not (0 <= iz < nz and geom.win_x0[s] <= ix < geom.win_x1[s]):
                raise ValueError(f"shot {s}: node ({iz},{ix}) outside its window")


def model_shots(v, geom, h, dt, nb):
    """Packed shot records d (float64), per shot [nt_s][nrec_s] (Eq. 1 forward modelling)."""
    v, vp = _d(v)
    nz, nx = v.shape
    _check_geom(nz, nx, geom)
    A = _Args(nz, nx, h, dt, nb, geom)
    d = np.zeros(geom.n_data, dtype=np.float64)
    lib().or_model_shots(ctypes.byref(A.grid), vp, ctypes.byref(A.geom), d.ctypes.data_as(_DP))
    return d


def fwi_gradient(v, geom, d_obs, h, dt, nb, seg=0):
    """(J, dJ/dv, d_syn): misfit of Eq. 2 and its exact discrete gradient (-g of Eq. 13)."""
    v, vp = _d(v)
    nz, nx = v.shape
    _check_geom(nz, nx, geom)
    A = _Args(nz, nx, h, dt, nb, geom)
    do, dop = _d(d_obs)
    g = np.zeros((nz, nx), dtype=np.float64)
    ds = np.zeros(geom.n_data, dtype=np.float64)
    J = lib().or_fwi_gradient(ctypes.byref(A.grid), vp, ctypes.byref(A.geom), dop,
                              g.ctypes.data_as(_DP), ds.ctypes.data_as(_DP), int(seg))
    return float(J), g, ds


def born_demig(v0, geom, dv, h, dt, nb):
    """Born data d = L~ dv (Eqs. 11-12b), absolute velocity perturbation dv in m/s."""
    v0, vp = _d(v0)
    nz, nx = v0.shape
    _check_geom(nz, nx, geom)
    A = _Args(nz, nx, h, dt, nb, geom)
    dv, dvp = _d(dv)
    d = np.zeros(geom.n_data, dtype=np.float64)
    lib().or_born_demig(ctypes.byref(A.grid), vp, ctypes.byref(A.geom), dvp, d.ctypes.data_as(_DP))
    return d


def rtm_mig(v0, geom, d, h, dt, nb, seg=0):
    """Migration img = L~^T d (Eq. 13 applied to arbitrary data)."""
    v0, vp = _d(v0)
    nz, nx = v0.shape
    _check_geom(nz, nx, geom)
    A = _Args(nz, nx, h, dt, nb, geom)
    dd, ddp = _d(d)
    img = np.zeros((nz, nx), dtype=np.float64)
    lib().or_rtm_mig(ctypes.byref(A.grid), vp, ctypes.byref(A.geom), ddp, img.ctypes.data_as(_DP), int(seg))
    return img


def apply_lap(u):
    """Unscaled 8th-order Laplacian D u with zero values outside the array."""
    u, up = _d(u)
    out = np.zeros_like(u)
    lib().or_apply_lap(u.shape[0], u.shape[1], up, out.ctypes.data_as(_DP))
    return out


def sponge(nz, nb, win_w):
    g = _Grid(int(nz), 1, int(nb), 1.0, 1.0)
    out = np.zeros((nz + 2 * nb, win_w + 2 * nb), dtype=np.float64)
    lib().or_sponge(ctypes.byref(g), int(win_w), out.ctypes.data_as(_DP))
    return out


def misfit(d_syn, d_obs):
    """J = 1/2 ||d_s - d_o||^2 (Eq. 2)."""
    r = np.asarray(d_syn, dtype=np.float64) - np.asarray(d_obs, dtype=np.float64)
    return 0.5 * float(np.dot(r, r))
