"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module only *creates inputs*: velocity models, source wavelets, acquisition
geometries, random perturbations and data vectors.  It holds none of the
method's arithmetic (no propagation, no adjoint, no imaging, no network), so
that the CPU oracle and the CUDA path, which both consume these inputs, share
no computation.

Every generator draws from ``numpy.random.Generator(PCG64(seed))``.

The paper's own datasets (Marmousi, Section 3.1; Volve, Sections 3.2-3.3) are
not available; seeded layered/faulted models with the shapes of the workloads
stand in for them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Geometry",
    "ricker",
    "two_layer_model",
    "layered_fault_model",
    "smooth_model",
    "surface_geometry",
    "uniform_geometry",
    "tiny_case",
    "config1_case",
    "config2_case",
    "config3_case",
    "config5_case",
    "rng",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------
# Source wavelet
# --------------------------------------------------------------------------
def ricker(f0: float, dt: float, nt: int, t0: float | None = None) -> np.ndarray:
    """Ricker wavelet of peak frequency ``f0`` sampled at t = n*dt, n = 0..nt-1.

    The paper names only the peak frequency of its Ricker sources (5 Hz for
    Marmousi, Section 3.1; 20 Hz for the Volve synthetic, Section 3.2).  The
    delay t0 = 1.5/f0 is a reading (the paper gives none); the amplitude is 1
    at t0.
    Returned in float64.
    """
    if t0 is None:
        t0 = 1.5 / f0
    t = np.arange(nt, dtype=np.float64) * dt - t0
    a = (math.pi * f0 * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


# --------------------------------------------------------------------------
# Velocity models (m/s), layout [nz][nx], x fastest
# --------------------------------------------------------------------------
def two_layer_model(nz: int, nx: int, h: float, z_if: float = 500.0,
                    v_top: float = 1500.0, v_bot: float = 2000.0) -> np.ndarray:
    z = np.arange(nz, dtype=np.float64) * h
    v = np.where(z[:, None] < z_if, v_top, v_bot) * np.ones((1, nx))
    return v.astype(np.float64)


def layered_fault_model(nz: int, nx: int, h: float, seed: int,
                        vmin: float = 1500.0, vmax: float = 4500.0) -> np.ndarray:
    """Seeded layered model with 6-10 dipping interfaces and 2 normal faults.

    Interface depths at x = 0 are uniform over [0.05, 0.95] of the model depth,
    dips uniform in +-8 degrees; layer velocities rise from vmin to vmax with
    +-150 m/s jitter (clipped).  Two normal faults dip at 60 degrees with a throw
    uniform in [50, 250] m applied to the hanging wall.
    """
    g = rng(seed)
    n_if = int(g.integers(6, 11))
    depth = nz * h
    width = nx * h
    z0 = np.sort(g.uniform(0.05, 0.95, n_if)) * depth
    dip = np.deg2rad(g.uniform(-8.0, 8.0, n_if))
    vel = np.linspace(vmin, vmax, n_if + 1) + g.uniform(-150.0, 150.0, n_if + 1)
    vel = np.clip(vel, vmin, vmax)
    faults = []
    for _ in range(2):
        xf = g.uniform(0.2, 0.8) * width
        side = 1.0 if g.uniform() < 0.5 else -1.0
        throw = g.uniform(50.0, 250.0)
        faults.append((xf, side, throw))

    zz, xx = np.meshgrid(np.arange(nz) * h, np.arange(nx) * h, indexing="ij")
    zs = zz.copy()
    # Undo each fault's displacement: points in the hanging wall come from
    # `throw` higher up (the hanging wall of a normal fault moved down).
    for xf, side, throw in faults:
        # Fault plane x = xf + side * z / tan(60 deg); the hanging wall is on
        # the side the plane dips towards.
        xplane = xf + side * zz / math.tan(math.radians(60.0))
        hanging = (xx - xplane) * side > 0.0
        zs = np.where(hanging, zs - throw, zs)
    layer = np.zeros((nz, nx), dtype=np.int64)
    for k in range(n_if):
        layer += (zs > z0[k] + xx * np.tan(dip[k])).astype(np.int64)
    return vel[layer].astype(np.float64)


def smooth_model(v: np.ndarray, sigma: float) -> np.ndarray:
    """Gaussian smoothing (reflecting edges) used to make initial/background models."""
    from scipy.ndimage import gaussian_filter

    return gaussian_filter(np.asarray(v, dtype=np.float64), sigma=sigma, mode="reflect")


# --------------------------------------------------------------------------
# Acquisition geometry
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Geometry:
    """Per-shot acquisition: sources, receivers (CSR), record lengths, windows.

    Coordinates are physical grid indices (row iz in [0, nz), column ix in
    [0, nx)).  Shot s records ``nt[s]`` samples at receivers
    ``rec_iz/rec_ix[rec_off[s]:rec_off[s+1]]`` and propagates inside the
    physical column window ``[win_x0[s], win_x1[s])`` (the sponge is added
    around it by the propagator).  ``wavelet`` is ``[nt_max]`` when
    ``wavelet_shared`` else ``[n_shots][nt_max]``.
    """

    src_iz: np.ndarray
    src_ix: np.ndarray
    nt: np.ndarray
    rec_off: np.ndarray
    rec_iz: np.ndarray
    rec_ix: np.ndarray
    win_x0: np.ndarray
    win_x1: np.ndarray
    wavelet: np.ndarray
    wavelet_shared: bool = True

    @property
    def n_shots(self) -> int:
        return int(self.src_iz.shape[0])

    @property
    def nt_max(self) -> int:
        return int(self.nt.max())

    def nrec(self, s: int) -> int:
        return int(self.rec_off[s + 1] - self.rec_off[s])

    def data_offsets(self) -> np.ndarray:
        """Start of each shot's packed [nt_s][nrec_s] block in the data vector."""
        sizes = self.nt.astype(np.int64) * np.diff(self.rec_off).astype(np.int64)
        return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)

    @property
    def n_data(self) -> int:
        return int(self.data_offsets()[-1])

    def subset(self, shots) -> "Geometry":
        shots = list(shots)
        rec_iz, rec_ix, off = [], [], [0]
        for s in shots:
            a, b = int(self.rec_off[s]), int(self.rec_off[s + 1])
            rec_iz.append(self.rec_iz[a:b])
            rec_ix.append(self.rec_ix[a:b])
            off.append(off[-1] + b - a)
        wav = self.wavelet if self.wavelet_shared else self.wavelet[shots]
        nt = self.nt[shots]
        if self.wavelet_shared:
            wav = wav[: int(nt.max())]
        else:
            wav = wav[:, : int(nt.max())]
        return Geometry(
            src_iz=self.src_iz[shots].copy(), src_ix=self.src_ix[shots].copy(),
            nt=nt.copy(), rec_off=np.asarray(off, dtype=np.int32),
            rec_iz=np.concatenate(rec_iz).astype(np.int32),
            rec_ix=np.concatenate(rec_ix).astype(np.int32),
            win_x0=self.win_x0[shots].copy(), win_x1=self.win_x1[shots].copy(),
            wavelet=np.ascontiguousarray(wav), wavelet_shared=self.wavelet_shared)

    def cell_updates(self, nz: int, nb: int) -> int:
        """Cell updates of one forward pass: sum over shots of nt * padded window cells."""
        w = (self.win_x1 - self.win_x0).astype(np.int64) + 2 * nb
        return int(np.sum(self.nt.astype(np.int64) * (nz + 2 * nb) * w))


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def uniform_geometry(src_ix, rec_ix, nt: int, wavelet: np.ndarray, nx: int,
                     src_iz: int = 0, rec_iz: int = 0) -> Geometry:
    """Every shot sees the same receivers and the full model width."""
    ns = len(src_ix)
    nr = len(rec_ix)
    return Geometry(
        src_iz=_i32([src_iz] * ns), src_ix=_i32(src_ix), nt=_i32([nt] * ns),
        rec_off=_i32(np.arange(ns + 1) * nr),
        rec_iz=_i32(np.full(ns * nr, rec_iz)), rec_ix=_i32(np.tile(rec_ix, ns)),
        win_x0=_i32([0] * ns), win_x1=_i32([nx] * ns),
        wavelet=np.ascontiguousarray(wavelet[:nt], dtype=np.float64), wavelet_shared=True)


def surface_geometry(nx: int, n_shots: int, seed: int, nrec_range=(200, 600),
                     nt_range=(3000, 4000), margin: int = 100, src_lo: int = 20,
                     src_hi: int | None = None, wavelet: np.ndarray | None = None,
                     row: int = 0) -> Geometry:
    """Surface acquisition with uneven apertures and record lengths.

    Sources at x = round(linspace(src_lo, src_hi, n_shots)) on ``row``.  Shot s
    has nrec_s ~ U{nrec_range} receivers on consecutive nodes centred on the
    source (shifted inward at the edges) and nt_s ~ U{nt_range} samples.  Its
    window is the receiver span joined with source +- margin, clipped to the
    model.
    """
    g = rng(seed)
    if src_hi is None:
        src_hi = nx - 21
    sx = np.rint(np.linspace(src_lo, src_hi, n_shots)).astype(np.int64)
    nrec = g.integers(nrec_range[0], nrec_range[1] + 1, n_shots)
    nts = g.integers(nt_range[0], nt_range[1] + 1, n_shots)
    rec_ix, off, x0s, x1s = [], [0], [], []
    for s in range(n_shots):
        n = int(min(nrec[s], nx))
        lo = int(sx[s]) - n // 2
        lo = max(0, min(lo, nx - n))
        rx = np.arange(lo, lo + n)
        rec_ix.append(rx)
        off.append(off[-1] + n)
        x0 = max(0, min(lo, int(sx[s]) - margin))
        x1 = min(nx, max(lo + n, int(sx[s]) + margin + 1))
        x0s.append(x0)
        x1s.append(x1)
    ntmax = int(nts.max())
    if wavelet is None:
        raise ValueError("wavelet required")
    wav = np.ascontiguousarray(np.asarray(wavelet, dtype=np.float64)[:ntmax])
    return Geometry(
        src_iz=_i32([row] * n_shots), src_ix=_i32(sx), nt=_i32(nts),
        rec_off=_i32(off), rec_iz=_i32(np.full(off[-1], row)),
        rec_ix=_i32(np.concatenate(rec_ix)), win_x0=_i32(x0s), win_x1=_i32(x1s),
        wavelet=wav, wavelet_shared=True)


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Case:
    nz: int
    nx: int
    h: float
    dt: float
    nb: int
    v_true: np.ndarray
    v_init: np.ndarray
    geom: Geometry
    name: str = ""


def tiny_case(nz=23, nx=29, h=10.0, dt=1e-3, nt=90, nb=6, n_shots=2, f0=25.0,
              seed=5, windows=True) -> Case:
    """Small random-ish case (odd sizes, shots near the edges) for exact checks."""
    g = rng(seed)
    v = 1800.0 + 400.0 * g.uniform(size=(nz, nx))
    v = smooth_model(v, 1.5)
    v_init = smooth_model(v, 3.0)
    wav = ricker(f0, dt, nt)
    src = np.linspace(2, nx - 3, n_shots).round().astype(int)
    rec_iz, rec_ix, off, x0s, x1s, nts = [], [], [0], [], [], []
    for s in range(n_shots):
        if windows:
            x0 = max(0, int(src[s]) - nx // 3)
            x1 = min(nx, int(src[s]) + nx // 3 + 1)
        else:
            x0, x1 = 0, nx
        rx = np.arange(x0, x1, 2)
        rec_ix.append(rx)
        rec_iz.append(np.full(rx.shape, 1 + (s % 3)))
        off.append(off[-1] + len(rx))
        x0s.append(x0)
        x1s.append(x1)
        nts.append(nt - 7 * s)
    geom = Geometry(
        src_iz=_i32([2 + s % 2 for s in range(n_shots)]), src_ix=_i32(src),
        nt=_i32(nts), rec_off=_i32(off), rec_iz=_i32(np.concatenate(rec_iz)),
        rec_ix=_i32(np.concatenate(rec_ix)), win_x0=_i32(x0s), win_x1=_i32(x1s),
        wavelet=wav, wavelet_shared=True)
    return Case(nz, nx, h, dt, nb, v, v_init, geom, name="tiny")


def config1_case() -> Case:
    """Plain FWI gradient, tiny: 101x101, dx 10 m, two layers (1500 over 2000 m/s
    at z = 500 m), dt 1 ms, nt 500, 20-cell sponge, 15 Hz Ricker, 4 surface
    shots, 51 surface receivers."""
    nz = nx = 101
    h, dt, nt, nb = 10.0, 1e-3, 500, 20
    v = two_layer_model(nz, nx, h)
    v0 = smooth_model(v, 10.0)
    wav = ricker(15.0, dt, nt)
    src = [int(round((k + 0.5) * nx / 4)) for k in range(4)]
    rec = list(range(0, 101, 2))
    geom = uniform_geometry(src, rec, nt, wav, nx)
    return Case(nz, nx, h, dt, nb, v, v0, geom, name="config1-101x101-4shots")


def config2_case(n_shots: int = 64, nt_range=(3000, 4000)) -> Case:
    """Batched shot modelling + gradient: seeded layered-fault model 400x1200,
    dx 12.5 m, dt 1 ms, 8 Hz Ricker, 64 shots with 200-600 receivers and
    3000-4000 samples each."""
    nz, nx, h, dt, nb = 400, 1200, 12.5, 1e-3, 20
    v = layered_fault_model(nz, nx, h, seed=17)
    v0 = smooth_model(v, 10.0)
    wav = ricker(8.0, dt, nt_range[1])
    geom = surface_geometry(nx, n_shots, seed=17, nt_range=nt_range, wavelet=wav,
                            src_lo=20, src_hi=1179)
    return Case(nz, nx, h, dt, nb, v, v0, geom, name="config2-400x1200-64shots")


def config3_case() -> Case:
    """Born demigration-migration pair on the 400x1200 model; background is the
    sigma = 10 cell Gaussian smoothing of the true model."""
    c = config2_case()
    c.name = "config3-400x1200-born-pair"
    return c


def config5_case(n_shots: int = 200, nt: int = 6000) -> Case:
    """Full multiscale FWI loop workload: 600x2000, dx 10 m, dt 0.8 ms, 200 shots."""
    nz, nx, h, dt, nb = 600, 2000, 10.0, 8e-4, 20
    v = layered_fault_model(nz, nx, h, seed=31)
    v0 = smooth_model(v, 10.0)
    wav = ricker(8.0, dt, nt)
    geom = surface_geometry(nx, n_shots, seed=31, nt_range=(int(nt * 0.75), nt),
                            wavelet=wav, src_lo=20, src_hi=nx - 21)
    return Case(nz, nx, h, dt, nb, v, v0, geom, name="config5-600x2000-200shots")


def marmousi_shaped_case(nt: int = 2400) -> Case:
    """A workload with the shape of the paper's Marmousi test (Section 3.1):
    221 x 601 nodes at 15 m (3.3 km x 9 km), 30 sources and 300 receivers
    (every second node) on the surface, a 5 Hz Ricker wavelet.  The Marmousi
    model itself is not available: a seeded layered model with two normal
    faults over Marmousi's velocity range (1500-4700 m/s) stands in for it.
    dt = 1.5 ms keeps the Courant number at 0.47 (the 8th-order limit in 2D
    is 0.555)."""
    nz, nx, h, dt, nb = 221, 601, 15.0, 1.5e-3, 20
    v = layered_fault_model(nz, nx, h, seed=41, vmin=1500.0, vmax=4700.0)
    v0 = smooth_model(v, 10.0)
    wav = ricker(5.0, dt, nt)
    src = np.round(np.linspace(10, nx - 11, 30)).astype(int)
    rec = np.arange(0, 600, 2)
    geom = uniform_geometry(src, rec, nt, wav, nx)
    return Case(nz, nx, h, dt, nb, v, v0, geom, name="marmousi-shaped-221x601-30shots")


def gaussian_field(shape, seed: int) -> np.ndarray:
    """Seeded standard-normal array (used for dot-product tests)."""
    return rng(seed).standard_normal(shape)


def smooth_random_field(nz: int, nx: int, seed: int, sigma: float = 2.0) -> np.ndarray:
    """Seeded smooth random perturbation with unit max-abs."""
    f = smooth_model(rng(seed).standard_normal((nz, nx)), sigma)
    return f / np.abs(f).max()
