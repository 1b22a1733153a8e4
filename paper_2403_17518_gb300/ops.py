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

    def set_reuse(self, on: bool = True):
        """Reuse the stored forward wavefield in rtm_mig / born_demig at the
        model and geometry of the last gradient or migration (same bits)."""
        self._check(self.lib.dhfwi_set_reuse(self.handle, 1 if on else 0))

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

    def selftest_timeout(self, stream=None):
        """Make one bounded device-side wait run out: the next call raises
        DhfwiError with DHFWI_ERR_TIMEOUT, later calls work normally."""
        self._check(self.lib.dhfwi_selftest_timeout(self.handle, self._stream(stream)))

    def image_laplacian(self, img: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """-(5-point Laplacian) / h^2 of an image, edge values repeated: the
        quality-control filter of migrated images."""
        out = out if out is not None else self.new_model()
        self._check(self.lib.image_laplacian(self.handle, self._model(img, "img"), self._model(out, "out"),
                                             self._stream(stream)))
        return out

    def rtm_qc(self, v: torch.Tensor, geom, d: torch.Tensor, stream=None) -> torch.Tensor:
        """Migration of data d through the model v, then the Laplacian filter
        (imaging with an estimated model to validate it, Section 3.3)."""
        return self.image_laplacian(self.rtm_mig(v, geom, d, stream=stream), stream=stream)

    def fwi_update(self, v: torch.Tensor, direction: torch.Tensor, alpha: float, vmin: float, vmax: float,
                   mute_rows: int = 0, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """clamp(v - alpha * dir / max|dir|, vmin, vmax) with the top rows muted."""
        out = out if out is not None else self.new_model()
        self._check(self.lib.fwi_update(self.handle, self._model(v, "v"), self._model(direction, "dir"),
                                        float(alpha), float(vmin), float(vmax), int(mute_rows),
                                        self._model(out, "out"), self._stream(stream)))
        return out

    def bb_step(self, x_k: torch.Tensor, x_prev: torch.Tensor, g_k: torch.Tensor, g_prev: torch.Tensor,
                mute_rows: int = 0, stream=None):
        """(alpha, max|g_k|): the Barzilai-Borwein short step of Eq. 17 below
        the muted rows; the update is fwi_update(x_k, g_k, alpha * max|g_k|)."""
        a, gm = ctypes.c_double(0.0), ctypes.c_double(0.0)
        self._check(self.lib.bb_step(self.handle, self._model(x_k, "x_k"), self._model(x_prev, "x_prev"),
                                     self._model(g_k, "g_k"), self._model(g_prev, "g_prev"), int(mute_rows),
                                     ctypes.byref(a), ctypes.byref(gm), self._stream(stream)))
        return a.value, gm.value

    def data_misfit(self, a: torch.Tensor, b: torch.Tensor, stream=None) -> float:
        """1/2 ||a - b||^2 accumulated in float64 on the device."""
        if a.numel() != b.numel():
            raise ValueError("a and b must have the same size")
        J = ctypes.c_double(0.0)
        self._check(self.lib.data_misfit(self.handle, self._dense(a, "a"), self._dense(b, "b"), a.numel(),
                                         ctypes.byref(J), self._stream(stream)))
        return J.value

    # -- deblurring network -----------------------------------------------
    def _dense(self, t: torch.Tensor, name: str) -> ctypes.c_void_p:
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.device == self.device):
            raise ValueError(f"{name} must be a contiguous float32 tensor on {self.device}")
        return ctypes.c_void_p(t.data_ptr())

    def net_init(self, base_channels: int = 32, levels: int = 4, seed: int = 29):
        self._check(self.lib.dhfwi_net_init(self.handle, int(base_channels), int(levels), int(seed)))

    def net_size(self) -> int:
        return int(self.lib.dhfwi_net_size(self.handle))

    def net_get(self) -> np.ndarray:
        n = self.net_size()
        out = np.empty(n, dtype=np.float32)
        self._check(self.lib.dhfwi_net_get(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n))
        return out

    def net_set(self, params) -> None:
        a = np.ascontiguousarray(params, dtype=np.float32)
        self._check(self.lib.dhfwi_net_set(self.handle, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size))

    def deblur_forward(self, x: torch.Tensor, stream=None) -> torch.Tensor:
        """Raw network on a batch x [n, h, w] (no normalisation)."""
        n, h, w = x.shape
        out = torch.empty_like(x)
        self._check(self.lib.deblur_forward(self.handle, self._dense(x, "x"), n, h, w, self._dense(out, "out"),
                                            self._stream(stream)))
        return out

    def deblur_grad(self, x: torch.Tensor, y: torch.Tensor, stream=None):
        """(loss, flat parameter gradient) of mean((net(x) - y)^2) on a batch."""
        n, h, w = x.shape
        g = torch.empty(self.net_size(), dtype=torch.float32, device=self.device)
        L = ctypes.c_double(0.0)
        self._check(self.lib.deblur_grad(self.handle, self._dense(x, "x"), self._dense(y, "y"), n, h, w,
                                         self._dense(g, "grad"), ctypes.byref(L), self._stream(stream)))
        return L.value, g

    def deblur_train(self, x_img: torch.Tensor, y_img: torch.Tensor, warm_start: bool = True, base_channels=32,
                     levels=4, patch=128, stride=64, batch=32, epochs=200, lr=1e-3, beta1=0.9, beta2=0.999,
                     eps=1e-8, seed=29, mute_rows=0, warmup_frac=0.0, stream=None):
        """Train x (doubly migrated image) -> y (gradient); returns per-epoch losses."""
        nz, nx = x_img.shape
        cfg = _lib.TrainCfg(int(base_channels), int(levels), int(patch), int(stride), int(batch), int(epochs),
                            float(lr), float(beta1), float(beta2), float(eps), int(seed), int(mute_rows),
                            float(warmup_frac))
        hist = np.zeros(int(epochs), dtype=np.float32)
        self._check(self.lib.deblur_train(self.handle, self._dense(x_img, "x"), self._dense(y_img, "y"), nz, nx,
                                          ctypes.byref(cfg), 1 if warm_start else 0,
                                          hist.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), self._stream(stream)))
        return hist

    def deblur_layer(self, kind: str, op: str, x=None, w=None, b=None, gy=None, n=1, H=1, W=1, ci=8, co=8,
                     stream=None) -> torch.Tensor:
        """One network layer alone (kind "conv3", "convT" or "first", the
        one-input-channel first convolution; op "fwd", "dgrad" or "wgrad"),
        NHWC float32 tensors; see deblur_layer in dhfwi.h."""
        k = {"conv3": 0, "convT": 1, "first": 2}[kind]
        o = {"fwd": 0, "dgrad": 1, "wgrad": 2}[op]
        taps = 4 if k == 1 else 9
        Ho, Wo = (2 * H, 2 * W) if k == 1 else (H, W)
        shape = {0: (n, Ho, Wo, co), 1: (n, H, W, ci), 2: (taps * ci * co + co,)}[o]
        out = torch.empty(shape, dtype=torch.float32, device=self.device)
        ptr = lambda t, nm: self._dense(t, nm) if t is not None else None
        self._check(self.lib.deblur_layer(self.handle, k, o, int(n), int(H), int(W), int(ci), int(co), ptr(x, "x"),
                                          ptr(w, "w"), ptr(b, "b"), ptr(gy, "gy"), self._dense(out, "out"),
                                          self._stream(stream)))
        return out

    def deblur_apply(self, g: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        nz, nx = g.shape
        out = out if out is not None else torch.empty_like(g)
        self._check(self.lib.deblur_apply(self.handle, self._dense(g, "g"), nz, nx, self._dense(out, "out"),
                                          self._stream(stream)))
        return out


def model_shots_static(nz: int, nx: int, h: float, dt: float, nb: int, v: torch.Tensor, geom,
                       out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Forward modelling without device allocation by the library: all
    temporaries live in the library's fixed static device array (see
    model_shots_static in include/dhfwi.h for the limits)."""
    lib = _lib.load()
    g = _as_geom(geom)
    if not (v.is_cuda and v.dtype == torch.float32 and v.is_contiguous() and tuple(v.shape) == (nz, nx)):
        raise ValueError("v must be a contiguous float32 CUDA tensor of shape (nz, nx)")
    d = out if out is not None else torch.empty(g.n_data, dtype=torch.float32, device=v.device)
    if not (d.is_cuda and d.dtype == torch.float32 and d.is_contiguous() and d.numel() == g.n_data):
        raise ValueError("out must be a contiguous float32 CUDA tensor with n_data values")
    if d.device != v.device:
        raise ValueError("out must be on v's device")
    grid = _lib.Grid(int(nz), int(nx), int(nb), float(h), float(dt))
    # The C call runs on the current device: make it v's.
    with torch.cuda.device(v.device):
        s = stream if stream is not None else torch.cuda.current_stream(v.device)
        rc = lib.model_shots_static(ctypes.byref(grid), ctypes.c_void_p(v.data_ptr()), ctypes.byref(g.struct),
                                    ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(s.cuda_stream))
    if rc != 0:
        raise DhfwiError(rc, lib.model_shots_static_error().decode())
    return d


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
