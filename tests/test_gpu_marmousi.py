"""GPU parity on the workload with the shape of the paper's Marmousi test
(Section 3.1: 221 x 601 nodes at 15 m, 30 surface sources, 300 receivers,
5 Hz), on its first and last shots (sources 10 nodes from either edge) with
records of 600 samples (0.9 s, so the FP64 oracle finishes in seconds):
records, misfit, gradient, Born data and migrated image within 1e-5.  The model is a seeded stand-in (the Marmousi
model is not available).  A host-side test checks the case itself."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import f32, f32_geom, gpu_ctx, rel_l2, to_dev, to_host

TOL = 1e-5


def _case():
    c = synth.marmousi_shaped_case(nt=600)
    c.geom = c.geom.subset([0, 29])
    return c


def test_marmousi_shaped_case_layout():
    c = synth.marmousi_shaped_case()
    g = c.geom
    assert (c.nz, c.nx, c.h) == (221, 601, 15.0)
    assert g.n_shots == 30 and all(g.nrec(s) == 300 for s in range(30))
    assert np.all(g.src_iz == 0) and np.all(g.rec_iz == 0)
    assert np.all(np.diff(g.rec_ix[:300]) == 2)
    assert 1500.0 <= c.v_true.min() and c.v_true.max() <= 4700.0
    # Leapfrog stability of the 8th-order 2D Laplacian: C^2 * 2 * S <= 4 with
    # S = |c0| + 2 sum |ck| of the 1D stencil.
    S = 205 / 72 + 2 * (8 / 5 + 1 / 5 + 8 / 315 + 1 / 560)
    C = c.v_true.max() * c.dt / c.h
    assert C * C * 2 * S <= 4.0
    # The wavelet peaks at 5 Hz.
    w = g.wavelet
    f = np.fft.rfftfreq(8 * len(w), c.dt)
    assert abs(f[np.argmax(np.abs(np.fft.rfft(w, 8 * len(w))))] - 5.0) < 0.1


@pytest.mark.gpu
def test_marmousi_shaped_parity():
    import torch

    c = _case()
    ctx = gpu_ctx(c)
    geom = f32_geom(c.geom)
    v, v0 = f32(c.v_true), f32(c.v_init)
    d_ref = oracle.model_shots(v, geom, c.h, c.dt, c.nb)
    d = to_host(ctx.model_shots(to_dev(v), geom))
    assert rel_l2(d, d_ref) <= TOL
    # Well-conditioned residual (|r| ~ |d|).
    d_obs = f32(0.5 * d_ref)
    J_ref, g_ref, ds_ref = oracle.fwi_gradient(v0, geom, d_obs, c.h, c.dt, c.nb)
    ds = torch.empty(geom.n_data, dtype=torch.float32, device="cuda")
    J, g = ctx.fwi_gradient(to_dev(v0), geom, to_dev(d_obs), d_syn=ds)
    assert rel_l2(to_host(ds), ds_ref) <= TOL
    assert abs(J - J_ref) <= TOL * abs(J_ref)
    assert rel_l2(to_host(g), g_ref) <= TOL
    dv = f32(synth.smooth_random_field(c.nz, c.nx, 43) * 100.0)
    b_ref = oracle.born_demig(v0, geom, dv, c.h, c.dt, c.nb)
    assert rel_l2(to_host(ctx.born_demig(to_dev(v0), geom, to_dev(dv))), b_ref) <= TOL
    m_ref = oracle.rtm_mig(v0, geom, d_obs, c.h, c.dt, c.nb)
    assert rel_l2(to_host(ctx.rtm_mig(to_dev(v0), geom, to_dev(d_obs))), m_ref) <= TOL
    ctx.close()
