"""GPU parity of the finite-difference path against the FP64 oracle.

Tolerances: wavefields, records and gradients relative L2 <= 1e-5; the
FP32 dot-product test <= 1e-4.  All calls go through the C ABI
(libdhfwi.so) via the ctypes binding.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import f32, f32_geom, gpu_ctx, rel_l2, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _cases():
    tiny = synth.tiny_case()
    tiny2 = synth.tiny_case(nz=37, nx=141, nt=150, nb=20, n_shots=3, seed=8)
    one = synth.tiny_case(nz=9, nx=11, nt=40, nb=4, n_shots=1, seed=2, windows=False)
    return {"tiny": tiny, "ragged": tiny2, "single": one, "config1": synth.config1_case()}


CASES = _cases()


@pytest.mark.parametrize("name", list(CASES))
def test_model_shots_parity(name):
    c = CASES[name]
    ctx = gpu_ctx(c)
    v, geom = f32(c.v_true), f32_geom(c.geom)
    d_ref = oracle.model_shots(v, geom, c.h, c.dt, c.nb)
    d = to_host(ctx.model_shots(to_dev(v), geom))
    assert rel_l2(d, d_ref) <= TOL


@pytest.mark.parametrize("name", list(CASES))
def test_fwi_gradient_parity(name):
    """Well-conditioned residual (d_obs = data of another model scaled by 1/2,
    so |r| ~ |d|): misfit, records and gradient within 1e-5."""
    c = CASES[name]
    ctx = gpu_ctx(c)
    geom = f32_geom(c.geom)
    v0 = f32(c.v_init)
    d_obs = f32(0.5 * oracle.model_shots(f32(c.v_true), geom, c.h, c.dt, c.nb))
    J_ref, g_ref, ds_ref = oracle.fwi_gradient(v0, geom, d_obs, c.h, c.dt, c.nb)
    import torch

    ds = torch.empty(geom.n_data, dtype=torch.float32, device="cuda")
    J, g = ctx.fwi_gradient(to_dev(v0), geom, to_dev(d_obs), d_syn=ds)
    assert rel_l2(to_host(ds), ds_ref) <= TOL
    assert abs(J - J_ref) <= TOL * abs(J_ref)
    assert rel_l2(to_host(g), g_ref) <= TOL


@pytest.mark.parametrize("name", ["tiny", "config1"])
def test_fwi_gradient_parity_small_residual(name):
    """Physical case d_obs = F(v_true).  The residual is a small difference of
    two records (for config 1 the interface reflection arrives after the
    0.5 s record, so |r| ~ |d| / 1e4), so FP32 record errors are amplified by
    kappa_r = |d_s| / |r| in the misfit.  The adjoint part is checked on its
    own: the GPU gradient equals the oracle migration of the GPU residual."""
    c = CASES[name]
    ctx = gpu_ctx(c)
    import torch

    geom = f32_geom(c.geom)
    v0 = f32(c.v_init)
    d_obs = f32(oracle.model_shots(f32(c.v_true), geom, c.h, c.dt, c.nb))
    J_ref, g_ref, ds_ref = oracle.fwi_gradient(v0, geom, d_obs, c.h, c.dt, c.nb)
    kappa_r = np.linalg.norm(ds_ref) / np.linalg.norm(ds_ref - d_obs)
    ds = torch.empty(geom.n_data, dtype=torch.float32, device="cuda")
    J, g = ctx.fwi_gradient(to_dev(v0), geom, to_dev(d_obs), d_syn=ds)
    assert rel_l2(to_host(ds), ds_ref) <= TOL
    assert abs(J - J_ref) <= 2 * TOL * kappa_r * abs(J_ref)
    r_gpu = (ds - to_dev(d_obs)).double().cpu().numpy()
    g_mig = oracle.rtm_mig(v0, geom, r_gpu, c.h, c.dt, c.nb)
    assert rel_l2(to_host(g), g_mig) <= TOL


@pytest.mark.parametrize("name", ["tiny", "ragged", "config1"])
@pytest.mark.parametrize("rel", [False, True])
def test_born_parity(name, rel):
    c = CASES[name]
    ctx = gpu_ctx(c)
    geom = f32_geom(c.geom)
    v0 = f32(c.v_init)
    dv = f32(synth.smooth_random_field(c.nz, c.nx, 5) * (0.05 if rel else 100.0))
    dv_abs = v0 * dv if rel else dv
    d_ref = oracle.born_demig(v0, geom, dv_abs, c.h, c.dt, c.nb)
    d = to_host(ctx.born_demig(to_dev(v0), geom, to_dev(dv), rel=rel))
    assert rel_l2(d, d_ref) <= TOL


@pytest.mark.parametrize("name", ["tiny", "ragged", "config1"])
@pytest.mark.parametrize("rel", [False, True])
def test_rtm_parity(name, rel):
    c = CASES[name]
    ctx = gpu_ctx(c)
    geom = f32_geom(c.geom)
    v0 = f32(c.v_init)
    d = f32(synth.gaussian_field(geom.n_data, 11))
    img_ref = oracle.rtm_mig(v0, geom, d, c.h, c.dt, c.nb)
    if rel:
        img_ref = img_ref * v0
    img = to_host(ctx.rtm_mig(to_dev(v0), geom, to_dev(d), rel=rel))
    assert rel_l2(img, img_ref) <= TOL


@pytest.mark.parametrize("name", ["tiny", "config1"])
def test_dot_product_fp32(name):
    c = CASES[name]
    ctx = gpu_ctx(c)
    v0 = to_dev(c.v_init)
    x = synth.gaussian_field((c.nz, c.nx), 23)
    y = synth.gaussian_field(c.geom.n_data, 24)
    Lx = to_host(ctx.born_demig(v0, c.geom, to_dev(x)))
    LTy = to_host(ctx.rtm_mig(v0, c.geom, to_dev(y)))
    a, b = float(np.dot(Lx, f32(y))), float(np.sum(f32(x) * LTy))
    assert abs(a - b) <= 1e-4 * max(abs(a), abs(b))


def test_gradient_equals_migration_of_residual():
    c = CASES["tiny"]
    ctx = gpu_ctx(c)
    import torch

    v0 = to_dev(c.v_init)
    d_obs = ctx.model_shots(to_dev(c.v_true), c.geom)
    ds = torch.empty_like(d_obs)
    _, g = ctx.fwi_gradient(v0, c.geom, d_obs, d_syn=ds)
    img = ctx.rtm_mig(v0, c.geom, ds - d_obs)
    assert rel_l2(to_host(g), to_host(img)) <= 1e-6


def test_deterministic():
    c = CASES["ragged"]
    ctx = gpu_ctx(c)
    v0 = to_dev(c.v_init)
    d_obs = ctx.model_shots(to_dev(c.v_true), c.geom)
    J1, g1 = ctx.fwi_gradient(v0, c.geom, d_obs)
    J2, g2 = ctx.fwi_gradient(v0, c.geom, d_obs)
    assert J1 == J2
    assert np.array_equal(to_host(g1), to_host(g2))


def test_autograd_function():
    c = CASES["tiny"]
    ctx = gpu_ctx(c)
    import torch

    from paper_2403_17518_gb300.ops import FWIMisfit

    d_obs = ctx.model_shots(to_dev(c.v_true), c.geom)
    v = to_dev(c.v_init).requires_grad_(True)
    J = FWIMisfit.apply(v, ctx, c.geom, d_obs)
    (3.0 * J).backward()
    _, g = ctx.fwi_gradient(to_dev(c.v_init), c.geom, d_obs)
    assert torch.allclose(v.grad, 3.0 * g)


def test_errors_are_reported():
    c = CASES["tiny"]
    ctx = gpu_ctx(c)
    from paper_2403_17518_gb300.ops import DhfwiError

    v = c.v_true.copy()
    v[3, 4] = np.nan
    with pytest.raises(DhfwiError, match="NONFINITE"):
        ctx.model_shots(to_dev(v), c.geom)
    with pytest.raises(DhfwiError, match="CFL"):
        ctx.model_shots(to_dev(c.v_true * 40.0), c.geom)
    bad = f32_geom(c.geom)
    bad.src_ix = bad.src_ix.copy()
    bad.src_ix[0] = c.nx + 5
    with pytest.raises(DhfwiError, match="GEOM"):
        ctx.model_shots(to_dev(c.v_true), bad)
    # The context stays usable after errors.
    d = ctx.model_shots(to_dev(c.v_true), c.geom)
    assert np.isfinite(to_host(d)).all()


def test_bounded_wait_timeout_is_reported_and_context_survives():
    """A device-side wait that runs out (a barrier nothing arrives at, the
    step kernels' ~1 s limit) is reported by the next call as
    DHFWI_ERR_TIMEOUT; the call after that computes the records correctly."""
    c = CASES["tiny"]
    ctx = gpu_ctx(c)
    from paper_2403_17518_gb300.ops import DhfwiError

    v, geom = f32(c.v_true), f32_geom(c.geom)
    ctx.selftest_timeout()
    with pytest.raises(DhfwiError) as e:
        ctx.model_shots(to_dev(v), geom)
    assert e.value.code == -6 and "TIMEOUT" in str(e.value)
    d = to_host(ctx.model_shots(to_dev(v), geom))
    assert rel_l2(d, oracle.model_shots(v, geom, c.h, c.dt, c.nb)) <= TOL
    # A call that synchronises anyway (data_misfit) reports the timeout itself.
    dd = to_dev(d)
    ctx.selftest_timeout()
    with pytest.raises(DhfwiError) as e:
        ctx.data_misfit(dd, dd)
    assert e.value.code == -6
    assert ctx.data_misfit(dd, dd) == 0.0


# ---------------------------------------------------------------------------
# Full-size workload (400 x 1200, 64 shots, nt 3000-4000): the batched launch
# the benchmark times, checked on shots the oracle computes one by one.
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def config2():
    return synth.config2_case()


def test_config2_model_shots_sampled(config2):
    c = config2
    ctx = gpu_ctx(c)
    geom = f32_geom(c.geom)
    v = f32(c.v_true)
    d = to_host(ctx.model_shots(to_dev(v), geom))
    off = geom.data_offsets()
    for s in (0, 37):  # shots run inside the full 64-shot batch
        sub = geom.subset([s])
        ref = oracle.model_shots(v, sub, c.h, c.dt, c.nb)
        assert rel_l2(d[off[s]:off[s + 1]], ref) <= TOL, s


def test_config2_gradient_two_shots(config2):
    c = config2
    ctx = gpu_ctx(c)
    geom = f32_geom(c.geom).subset([5, 50])
    v0 = f32(c.v_init)
    d_obs = f32(0.5 * oracle.model_shots(f32(c.v_true), geom, c.h, c.dt, c.nb))
    J_ref, g_ref, _ = oracle.fwi_gradient(v0, geom, d_obs, c.h, c.dt, c.nb)
    J, g = ctx.fwi_gradient(to_dev(v0), geom, to_dev(d_obs))
    assert abs(J - J_ref) <= TOL * J_ref
    assert rel_l2(to_host(g), g_ref) <= TOL


def test_config2_born_and_migration_two_shots(config2):
    """Born demigration and migration at the full record lengths of the
    64-shot workload (3000-4000 steps, where FP32 error grows most), on two
    of its shots, element-wise against the oracle; and the FP32 dot-product
    test at that length."""
    c = config2
    ctx = gpu_ctx(c)
    geom = f32_geom(c.geom).subset([5, 50])
    assert int(geom.nt.min()) >= 3000
    v0 = f32(c.v_init)
    dv = f32(synth.smooth_random_field(c.nz, c.nx, 5) * 100.0)
    d_ref = oracle.born_demig(v0, geom, dv, c.h, c.dt, c.nb)
    d = to_host(ctx.born_demig(to_dev(v0), geom, to_dev(dv)))
    assert rel_l2(d, d_ref) <= TOL
    y = f32(synth.gaussian_field(geom.n_data, 24))
    img_ref = oracle.rtm_mig(v0, geom, y, c.h, c.dt, c.nb)
    img = to_host(ctx.rtm_mig(to_dev(v0), geom, to_dev(y)))
    assert rel_l2(img, img_ref) <= TOL
    x = f32(synth.gaussian_field((c.nz, c.nx), 23))
    Lx = to_host(ctx.born_demig(to_dev(v0), geom, to_dev(x)))
    a, b = float(np.dot(Lx, y)), float(np.sum(x * img))
    assert abs(a - b) <= 1e-4 * max(abs(a), abs(b))


@pytest.mark.parametrize("name", ["ragged", "config1"])
def test_doubly_migrated_image_parity(name):
    """The chain of the doubly migrated image (Eq. 15): the gradient of a
    physical misfit, then delta m_1 = L~^T L~ g, against the oracle's
    composition on the same (float32-rounded) gradient."""
    c = CASES[name]
    ctx = gpu_ctx(c)
    geom = f32_geom(c.geom)
    v0 = f32(c.v_init)
    d_obs = ctx.model_shots(to_dev(f32(c.v_true)), geom)
    _, g = ctx.fwi_gradient(to_dev(v0), geom, d_obs)
    g_host = to_host(g)
    dm1 = to_host(ctx.doubly_migrated(to_dev(v0), geom, g))
    ref = oracle.rtm_mig(v0, geom, oracle.born_demig(v0, geom, g_host, c.h, c.dt, c.nb), c.h, c.dt, c.nb)
    assert rel_l2(dm1, ref) <= TOL


def test_fwi_update_and_data_misfit():
    c = CASES["tiny"]
    ctx = gpu_ctx(c)
    g = np.random.Generator(np.random.PCG64(12))
    v = f32(c.v_init)
    d = f32(g.standard_normal(v.shape))
    from oracle import fwi_step

    out = to_host(ctx.fwi_update(to_dev(v), to_dev(d), 25.0, 1500.0, 2200.0, 3))
    ref = fwi_step.update(v, d, 25.0, 1500.0, 2200.0, mute_rows=3)
    assert np.abs(out - ref).max() <= 1e-3
    a, b = f32(g.standard_normal(1000)), f32(g.standard_normal(1000))
    J = ctx.data_misfit(to_dev(a), to_dev(b))
    assert J == pytest.approx(oracle.misfit(a, b), rel=1e-6)


def test_bb_step_matches_oracle():
    """The Barzilai-Borwein short step (Eq. 17) over the unmuted rows and
    max|g_k| there, against the oracle; the BB update through fwi_update."""
    c = CASES["ragged"]
    ctx = gpu_ctx(c)
    from oracle import fwi_step

    g = np.random.Generator(np.random.PCG64(21))
    xp, xk = f32(c.v_init), f32(c.v_init + g.standard_normal((c.nz, c.nx)))
    gp, gk = f32(g.standard_normal((c.nz, c.nx))), f32(g.standard_normal((c.nz, c.nx)))
    gk[:4] = 1e3  # muted rows: left out of both sums and of the max
    alpha, gmax = ctx.bb_step(to_dev(xk), to_dev(xp), to_dev(gk), to_dev(gp), mute_rows=4)
    ref = fwi_step.bb_short(xk[4:], xp[4:], gk[4:], gp[4:])
    assert alpha == pytest.approx(ref, rel=1e-12)
    assert gmax == np.abs(gk[4:]).max()
    out = to_host(ctx.fwi_update(to_dev(xk), to_dev(gk), alpha * gmax, 100.0, 9000.0, 4))
    exp = xk.copy()
    exp[4:] -= alpha * gk[4:]
    assert np.abs(out - exp).max() <= 1e-3
    from paper_2403_17518_gb300.ops import DhfwiError

    with pytest.raises(DhfwiError, match="NONFINITE"):
        ctx.bb_step(to_dev(xk), to_dev(xp), to_dev(gp), to_dev(gp))


def test_image_laplacian_and_rtm_qc():
    """The image QC filter against its definition (float64, edge values
    repeated), and rtm_qc = filter(rtm_mig) bit for bit."""
    c = CASES["ragged"]
    ctx = gpu_ctx(c)
    g = np.random.Generator(np.random.PCG64(5))
    img = f32(g.standard_normal((c.nz, c.nx)))
    out = to_host(ctx.image_laplacian(to_dev(img)))
    x = img.astype(np.float64)
    p = np.pad(x, 1, mode="edge")
    ref = -((p[:-2, 1:-1] - x) + (p[2:, 1:-1] - x) + (p[1:-1, :-2] - x) + (p[1:-1, 2:] - x)) / c.h ** 2
    assert np.abs(out - ref).max() <= 1e-6 * np.abs(ref).max()
    geom = f32_geom(c.geom)
    v0 = to_dev(f32(c.v_init))
    d = to_dev(f32(oracle.model_shots(f32(c.v_true), geom, c.h, c.dt, c.nb)))
    qc = to_host(ctx.rtm_qc(v0, geom, d))
    np.testing.assert_array_equal(qc, to_host(ctx.image_laplacian(ctx.rtm_mig(v0, geom, d))))
