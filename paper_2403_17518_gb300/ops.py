"""PyTorch-facing binding of the C ABI: same names as include/dhfwi.h.

Every call passes device pointers (``tensor.data_ptr()``) and the current
CUDA stream to libdhfwi.so; all arithmetic of the path runs in the library's
kernels.  PyTorch only allocates device memory and provides the stream.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import DHFWI_ABS, DHFWI_REL, DhfwiError

__all__ = ["Context", "GeomArgs", "FWIMisfit", "DhfwiError", "DHFWI_ABS", "DHFWI_REL"]


class GeomArgs:
    """Holds a ctypes Geom plus the host arrays it points at.

    ``geom`` is any object with the attributes src_iz, src_ix, nt, rec_off,
    rec_iz, rec_ix, win_x0, win_x1, wavelet and wavelet_shared (numpy arrays).
    """

    def __init__(self, geom):
        def i32(a):
            return np.ascontiguousarray(np.asarray(a), dtype=np.int32)

        self.arrays = {k: i32(getattr(geom, k)) for k in
                       ("src_iz", "src_ix", "nt", "rec_off", "rec_iz", "rec_ix", "win_x0", "win_x1")}
        wav = np.ascontiguousarray(np.asarray(geom.wavelet), dtype=np.float32)
        self.wavelet = wav
        self.n_shots = int(self.arrays["src_iz"].shape[0])
        shared = bool(getattr(geom, "wavelet_shared", wav.ndim == 1))
        IP = ctypes.POINTER(ctypes.c_int)
        FP = ctypes.POINTER(ctypes.c_float)
        a = self.arrays
        self.struct = _lib.Geom(
            self.n_shots, a["src_iz"].ctypes.data_as(IP), a["src_ix"].ctypes.data_as(IP),
            a["nt"].ctypes.data_as(IP), a["rec_off"].ctypes.data_as(IP), a["rec_iz"].ctypes.data_as(IP),
            a["rec_ix"].ctypes.data_as(IP), a["win_x0"].ctypes.data_as(IP), a["win_x1"].ctypes.data_as(IP),
            wav.ctypes.data_as(FP), int(wav.shape[-1]), 1 if shared else 0)
        nrec = np.diff(a["rec_off"]).astype(np.int64)
        self.n_data = int(np.sum(a["nt"].astype(np.int64) * nrec))


def _as_geom(geom) -> GeomArgs:
    return geom if isinstance(geom, GeomArgs) else GeomArgs(geom)


class Context:
    """Owns a ``dhfwi_ctx`` (device workspace) for one grid on one device."""

    def __init__(self, nz: int, nx: int, h: float, dt: float, nb: int = 20, device: int = 0):
        self.lib = _lib.load()
        self.nz, self.nx, self.h, self.dt, self.nb = int(nz), int(nx), float(h), float(dt), int(nb)
        self.device = torch.device("cuda", device)
        grid = _lib.Grid(self.nz, self.nx, self.nb, self.h, self.dt)
        handle = ctypes.c_void_p()
        rc = self.lib.dhfwi_create(ctypes.byref(handle), ctypes.byref(grid), int(device))
        if rc != 0:
            raise DhfwiError(rc, self.lib.dhfwi_last_error(None).decode())
        self.handle = handle

    def close(self):
        if getattr(self, "handle", None):
            self.lib.dhfwi_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers ---------------------------------------------------------
    def _check(self, rc: int):
        if rc != 0:
            raise DhfwiError(rc, self.lib.dhfwi_last_error(self.handle).decode())

    def _stream(self, stream=None) -> ctypes.c_void_p:
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        return ctypes.c_void_p(s.cuda_stream)

    def _model(self, t: torch.Tensor, name: str) -> ctypes.c_void_p:
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.device == self.device):
            raise ValueError(f"{name} must be a contiguous float32 tensor on {self.device}")
        if tuple(t.shape) != (self.nz, self.nx):
            raise ValueError(f"{name} must have shape ({self.nz}, {self.nx})")
        return ctypes.c_void_p(t.data_ptr())

    def _data(self, t: torch.Tensor, n: int, name: str) -> ctypes.c_void_p:
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.device == self.device):
            raise ValueError(f"{name} must be a contiguous float32 tensor on {self.device}")
        if t.numel() != n:
            raise ValueError(f"{name} must hold {n} samples")
        return ctypes.c_void_p(t.data_ptr())

    def new_model(self) -> torch.Tensor:
        return torch.empty((self.nz, self.nx), dtype=torch.float32, device=self.device)

    def new_data(self, geom) -> torch.Tensor:
        g = _as_geom(geom)
        return torch.empty(g.n_data, dtype=torch.float32, device=self.device)

    def stats(self) -> dict:
        s = _lib.Stats()
        self._check(self.lib.dhfwi_stats(self.handle, ctypes.byref(s)))
        out = {}
        for k, _ in _lib.Stats._fields_:
            val = getattr(s, k)
            out[k] = list(val) if hasattr(val, "__len__") else val
        return out

    def set_timing(self, on: bool = True):
        self._check(self.lib.dhfwi_set_timing(self.handle, 1 if on else 0))

    # -- the calls of the C ABI ------------------------------------------
    def model_shots(self, v: torch.Tensor, geom, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        g = _as_geom(geom)
        d = out if out is not None else self.new_data(g)
        self._check(self.lib.model_shots(self.handle, self._model(v, "v"), ctypes.byref(g.struct),
                                         self._data(d, g.n_data, "d"), self._stream(stream)))
        return d

    def fwi_gradient(self, v: torch.Tensor, geom, d_obs: torch.Tensor, grad: torch.Tensor | None = None,
                     d_syn: torch.Tensor | None = None, want_misfit: bool = True, stream=None):
        """Returns (J, dJ/dv).  J is None when want_misfit is False (no host sync)."""
        g = _as_geom(geom)
        grad = grad if grad is not None else self.new_model()
        J = ctypes.c_double(0.0)
        self._check(self.lib.fwi_gradient(
            self.handle, self._model(v, "v"), ctypes.byref(g.struct), self._data(d_obs, g.n_data, "d_obs"),
            self._model(grad, "grad"), ctypes.byref(J) if want_misfit else None,
            self._data(d_syn, g.n_data, "d_syn") if d_syn is not None else None, self._stream(stream)))
        return (J.value if want_misfit else None), grad

    def born_demig(self, v0: torch.Tensor, geom, dv: torch.Tensor, rel: bool = False,
                   out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        g = _as_geom(geom)
        d = out if out is not None else self.new_data(g)
        self._check(self.lib.born_demig(self.handle, self._model(v0, "v0"), ctypes.byref(g.struct),
                                        self._model(dv, "dv"), self._data(d, g.n_data, "d"),
                                        DHFWI_REL if rel else DHFWI_ABS, self._stream(stream)))
        return d

    def rtm_mig(self, v0: torch.Tensor, geom, d: torch.Tensor, rel: bool = False,
                out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        g = _as_geom(geom)
        img = out if out is not None else self.new_model()
        self._check(self.lib.rtm_mig(self.handle, self._model(v0, "v0"), ctypes.byref(g.struct),
                                     self._data(d, g.n_data, "d"), self._model(img, "img"),
                                     DHFWI_REL if rel else DHFWI_ABS, self._stream(stream)))
        return img

    def doubly_migrated(self, v0: torch.Tensor, geom, g_img: torch.Tensor) -> torch.Tensor:
        """delta m_1 = L~^T L~ g (Section 2.3.1, Eq. 15)."""
        return self.rtm_mig(v0, geom, self.born_demig(v0, geom, g_img))


class FWIMisfit(torch.autograd.Function):
    """J(v) = 1/2 ||d_s(v) - d_o||^2 with the adjoint-state gradient as backward.

    forward calls ``fwi_gradient`` once (misfit and gradient together) and
    keeps the gradient for backward, which scales it by the incoming grad.
    """

    @staticmethod
    def forward(fctx, v: torch.Tensor, ctx: Context, geom, d_obs: torch.Tensor):
        J, grad = ctx.fwi_gradient(v.detach().contiguous(), geom, d_obs)
        fctx.save_for_backward(grad)
        return torch.tensor(J, dtype=torch.float64, device=v.device)

    @staticmethod
    def backward(fctx, gout):
        (grad,) = fctx.saved_tensors
        return (gout.to(grad.dtype) * grad), None, None, None
