"""What the trained network gains over the gradient alone (Section 3.1).

The paper observes that the doubly migrated image delta m_1 = L~^T L~ g
decays more strongly with depth than the gradient g, and that the
network's update net(g) is better balanced over depth than g.  On a seeded
layered model these become inequalities on the depth ratio
  R(x) = rms(deeper half) / rms(shallower half) of the image below the
  source/receiver footprint:   R(delta m_1) < R(g) < R(net(g)).
(The paper's "lower resolution" remark is not asserted: no simple spectral
measure here separates it from the near-surface footprint.)
"""
import numpy as np
import pytest

import synth
from gpu_helpers import gpu_ctx, to_dev, to_host

pytestmark = pytest.mark.gpu


def depth_ratio(img, top):
    a = img[top:]
    half = a.shape[0] // 2
    return float(np.sqrt(np.mean(a[half:] ** 2)) / np.sqrt(np.mean(a[:half] ** 2)))


def test_doubly_migrated_image_and_network_update():
    nz, nx, h, dt, nt = 128, 320, 10.0, 1e-3, 900
    v = synth.layered_fault_model(nz, nx, h, seed=5, vmin=1500.0, vmax=3000.0)
    v0 = synth.smooth_model(v, 8.0)
    wav = synth.ricker(15.0, dt, nt)
    geom = synth.surface_geometry(nx, 16, seed=5, nrec_range=(160, 220), nt_range=(nt, nt), margin=60, src_lo=10,
                                  src_hi=nx - 11, wavelet=wav)
    case = synth.Case(nz, nx, h, dt, 20, v, v0, geom)
    ctx = gpu_ctx(case)
    d_obs = ctx.model_shots(to_dev(v), geom)
    _, g = ctx.fwi_gradient(to_dev(v0), geom, d_obs)
    dm1 = ctx.doubly_migrated(to_dev(v0), geom, g)
    hist = ctx.deblur_train(dm1, g, warm_start=False, base_channels=32, levels=4, patch=64, stride=32, batch=16,
                            epochs=150, lr=1e-3, seed=29)
    assert hist[-1] < 0.5 * hist[0], hist[[0, -1]]
    out = to_host(ctx.deblur_apply(g))
    G, M1 = to_host(g), to_host(dm1)
    top = 10
    assert depth_ratio(M1, top) < depth_ratio(G, top) < depth_ratio(out, top)
