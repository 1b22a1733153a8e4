"""Pins for the FP64 CPU oracle of the wave-equation operators.

Each test checks the oracle against something fixed by physics or
mathematics, not against itself:

* the 8th-order stencil is exact on polynomials of degree <= 9 (and not 10);
* forward modelling (Section 2.1, Eq. 1) matches the analytic 2D Green's
  function convolved with the Ricker wavelet, converging at second order;
* the discrete scheme is reciprocal (source/receiver swap);
* the sponge absorbs (boundary reflections below 5 %, 63 % without it);
* the gradient of Eq. 2 matches central finite differences (sign included);
* Born (Eqs. 9-12b) is the tangent of forward modelling (slope 2);
* migration is the exact adjoint of Born (dot-product test, Eq. 13);
* L~^T L~ is symmetric positive semi-definite (Eqs. 14-15).
"""
import numpy as np
import pytest

import synth


# --------------------------------------------------------------------------
# Stencil and wavelet
# --------------------------------------------------------------------------
def test_stencil_exact_on_polynomials(oracle_lib):
    n = 31
    z, x = np.meshgrid(np.arange(n) - 15.0, np.arange(n) - 15.0, indexing="ij")
    inner = (slice(4, n - 4), slice(4, n - 4))
    for a in range(0, 10):
        for b in (0, 1, 2, 3):
            u = x**a * z**b
            exact = a * (a - 1) * x ** max(a - 2, 0) * z**b + b * (b - 1) * x**a * z ** max(b - 2, 0)
            got = oracle_lib.apply_lap(u)
            scale = max(1.0, np.abs(u[inner]).max())
            assert np.abs(got[inner] - exact[inner]).max() <= 1e-11 * scale, (a, b)
    # Degree 10 is not reproduced: the stencil is exactly 8th order.
    u = x**10
    got = oracle_lib.apply_lap(u)
    assert np.abs(got[inner] - 90 * x[inner] ** 8).max() > 1.0


def test_stencil_zero_outside():
    import oracle

    u = np.zeros((9, 9))
    u[0, 0] = 1.0
    out = oracle.apply_lap(u)
    # Only the cross of radius 4 around (0, 0), inside the array, is touched.
    nz = np.argwhere(out != 0)
    assert len(nz) == 9
    assert out[0, 0] == pytest.approx(2 * (-205.0 / 72.0))


def test_ricker_properties():
    f0, dt, nt = 15.0, 1e-4, 4000
    w = synth.ricker(f0, dt, nt)
    t0 = 1.5 / f0
    assert np.argmax(w) == int(round(t0 / dt))
    assert w.max() == pytest.approx(1.0, abs=1e-12)
    assert abs(np.sum(w) * dt) < 1e-8  # zero mean
    spec = np.abs(np.fft.rfft(w, 1 << 16))
    freqs = np.fft.rfftfreq(1 << 16, dt)
    assert freqs[np.argmax(spec)] == pytest.approx(f0, rel=0.01)


# --------------------------------------------------------------------------
# Forward modelling vs the analytic Green's function
# --------------------------------------------------------------------------
def _green_ricker(r, c, f0, t):
    """u(r, t) = (G * f)(t) for (1/c^2) u_tt - lap u = f(t) delta(x) in 2D.

    G = H(t - r/c) / (2 pi sqrt(t^2 - r^2/c^2)).  With sigma = t - tau - r/c
    = s^2 the convolution becomes the smooth integral
    (1/pi) int_0^sqrt(t - r/c) f(t - r/c - s^2) / sqrt(s^2 + 2r/c) ds.
    """
    tau = t - r / c
    out = np.zeros_like(t)
    m = tau > 0
    S = np.sqrt(tau[m])
    x = np.linspace(0.0, 1.0, 4001)
    wts = np.ones_like(x)
    wts[1:-1:2] = 4
    wts[2:-1:2] = 2
    wts *= (x[1] - x[0]) / 3
    s = S[:, None] * x[None, :]
    arg = tau[m][:, None] - s**2
    a = (np.pi * f0 * (arg - 1.5 / f0)) ** 2
    f = (1 - 2 * a) * np.exp(-a)
    out[m] = S / np.pi * ((f / np.sqrt(s**2 + 2 * r / c)) @ wts)
    return out


def _green_errors(oracle, h, dt, offs, L=700.0, c=2000.0, f0=15.0):
    n = int(round(2 * L / h)) + 1
    mid = n // 2
    v = np.full((n, n), c)
    nt = int(round((max(offs) / c + 0.25) / dt))
    wav = synth.ricker(f0, dt, nt)
    rec = [mid + int(round(o / h)) for o in offs]
    g = synth.uniform_geometry([mid], rec, nt, wav, n, src_iz=mid, rec_iz=mid)
    g.win_x0[:] = 3  # a window that does not start at column 0
    g.win_x1[:] = n - 2
    d = oracle.model_shots(v, g, h, dt, 20).reshape(nt, len(rec))
    t = (np.arange(nt) + 1) * dt  # d[n] samples u^{n+1}
    errs = []
    for k, o in enumerate(offs):
        ref = _green_ricker(o, c, f0, t)
        errs.append(np.linalg.norm(d[:, k] - ref) / np.linalg.norm(ref))
    return np.array(errs)


def test_forward_matches_analytic_green_function(oracle_lib):
    offs = [200.0, 300.0, 400.0]
    e1 = _green_errors(oracle_lib, 5.0, 5e-4, offs)
    assert np.all(e1 <= 0.02), e1
    e2 = _green_errors(oracle_lib, 2.5, 2.5e-4, offs)
    # Second-order convergence (time discretisation dominates).
    assert np.all(e2 <= e1 / 3.0), (e1, e2)


# --------------------------------------------------------------------------
# Discrete symmetry and the sponge
# --------------------------------------------------------------------------
def test_reciprocity(oracle_lib):
    nz, nx, h, dt, nb, nt = 41, 53, 10.0, 1e-3, 10, 400
    v = synth.smooth_model(1700 + 600 * synth.rng(3).uniform(size=(nz, nx)), 2.0)
    wav = synth.ricker(20.0, dt, nt)
    A, B = (2, 10), (17, 40)
    g = synth.Geometry(
        src_iz=np.array([A[0], B[0]], np.int32), src_ix=np.array([A[1], B[1]], np.int32),
        nt=np.array([nt, nt], np.int32), rec_off=np.array([0, 1, 2], np.int32),
        rec_iz=np.array([B[0], A[0]], np.int32), rec_ix=np.array([B[1], A[1]], np.int32),
        win_x0=np.array([3, 3], np.int32), win_x1=np.array([50, 50], np.int32), wavelet=wav)
    d = oracle_lib.model_shots(v, g, h, dt, nb).reshape(2, nt)
    assert np.abs(d[0]).max() > 1e-3
    assert np.linalg.norm(d[0] - d[1]) <= 1e-12 * np.linalg.norm(d[0])


def test_sponge_absorbs(oracle_lib):
    nt, h, dt = 700, 10.0, 1e-3
    wav = synth.ricker(15.0, dt, nt)

    def trace(n, nb):
        v = np.full((n, n), 2000.0)
        g = synth.uniform_geometry([n // 2], [n // 2 + 10], nt, wav, n, src_iz=n // 2, rec_iz=n // 2)
        return oracle_lib.model_shots(v, g, h, dt, nb)

    ref = trace(401, 0)  # boundary too far to reach the receiver within nt
    err20 = np.abs(trace(81, 20) - ref).max() / np.abs(ref).max()
    err0 = np.abs(trace(81, 0) - ref).max() / np.abs(ref).max()
    assert err20 < 0.05, err20
    assert err0 > 0.3, err0
    w = oracle_lib.sponge(11, 20, 13)
    assert np.all(w[20:31, 20:33] == 1.0)
    assert np.all((w > 0.8) & (w <= 1.0))
    assert np.all(np.diff(w[25, :20]) > 0)


# --------------------------------------------------------------------------
# Gradient, Born and migration
# --------------------------------------------------------------------------
def _perturbed_case(per_shot_wavelet=False):
    c = synth.tiny_case(nz=19, nx=27, nt=110, nb=5, n_shots=3)
    if per_shot_wavelet:
        g = c.geom
        w = np.stack([synth.ricker(f, c.dt, g.nt_max) for f in (20.0, 25.0, 30.0)])
        g.wavelet = w
        g.wavelet_shared = False
    return c


@pytest.mark.parametrize("per_shot_wavelet", [False, True])
def test_gradient_matches_finite_differences(oracle_lib, per_shot_wavelet):
    c = _perturbed_case(per_shot_wavelet)
    d_obs = oracle_lib.model_shots(c.v_true, c.geom, c.h, c.dt, c.nb)
    J, grad, _ = oracle_lib.fwi_gradient(c.v_init, c.geom, d_obs, c.h, c.dt, c.nb)
    assert J > 0
    for seed in (3, 4):
        e = synth.smooth_random_field(c.nz, c.nx, seed, sigma=1.5)
        eps = 1e-5 * np.abs(c.v_init).max()
        Jp = oracle_lib.misfit(oracle_lib.model_shots(c.v_init + eps * e, c.geom, c.h, c.dt, c.nb), d_obs)
        Jm = oracle_lib.misfit(oracle_lib.model_shots(c.v_init - eps * e, c.geom, c.h, c.dt, c.nb), d_obs)
        fd = (Jp - Jm) / (2 * eps)
        an = float(np.sum(grad * e))
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


def test_gradient_checkpointing_is_exact(oracle_lib):
    c = _perturbed_case()
    d_obs = oracle_lib.model_shots(c.v_true, c.geom, c.h, c.dt, c.nb)
    _, g_all, _ = oracle_lib.fwi_gradient(c.v_init, c.geom, d_obs, c.h, c.dt, c.nb, seg=0)
    _, g_seg, _ = oracle_lib.fwi_gradient(c.v_init, c.geom, d_obs, c.h, c.dt, c.nb, seg=7)
    assert np.array_equal(g_all, g_seg)


def test_gradient_is_migration_of_residual(oracle_lib):
    c = _perturbed_case()
    d_obs = oracle_lib.model_shots(c.v_true, c.geom, c.h, c.dt, c.nb)
    J, grad, d_syn = oracle_lib.fwi_gradient(c.v_init, c.geom, d_obs, c.h, c.dt, c.nb)
    assert J == pytest.approx(oracle_lib.misfit(d_syn, d_obs), rel=1e-14)
    img = oracle_lib.rtm_mig(c.v_init, c.geom, d_syn - d_obs, c.h, c.dt, c.nb)
    assert np.abs(img - grad).max() <= 1e-13 * np.abs(grad).max()


def test_born_is_tangent_of_forward(oracle_lib):
    c = _perturbed_case()
    dv = synth.smooth_random_field(c.nz, c.nx, 9, sigma=1.5)
    Ldv = oracle_lib.born_demig(c.v_init, c.geom, dv, c.h, c.dt, c.nb)
    errs = []
    for eps in (40.0, 20.0, 10.0):
        Fp = oracle_lib.model_shots(c.v_init + eps * dv, c.geom, c.h, c.dt, c.nb)
        Fm = oracle_lib.model_shots(c.v_init - eps * dv, c.geom, c.h, c.dt, c.nb)
        errs.append(np.linalg.norm((Fp - Fm) / (2 * eps) - Ldv) / np.linalg.norm(Ldv))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 1e-3
    assert np.all(np.abs(slopes - 2.0) < 0.15), (errs, slopes)


def test_born_migration_dot_product(oracle_lib):
    c = _perturbed_case(per_shot_wavelet=True)
    x = synth.gaussian_field((c.nz, c.nx), 23)
    y = synth.gaussian_field(c.geom.n_data, 24)
    Lx = oracle_lib.born_demig(c.v_init, c.geom, x, c.h, c.dt, c.nb)
    LTy = oracle_lib.rtm_mig(c.v_init, c.geom, y, c.h, c.dt, c.nb)
    a, b = float(np.dot(Lx, y)), float(np.sum(x * LTy))
    assert abs(a - b) <= 1e-12 * max(abs(a), abs(b))


def test_linearised_misfit_gradient(oracle_lib):
    """Phi(x) = 1/2 ||L~ x - d||^2: central FD equals <L~^T(L~x - d), e> (Eq. 13-14)."""
    c = _perturbed_case()
    x = synth.smooth_random_field(c.nz, c.nx, 31)
    d = synth.gaussian_field(c.geom.n_data, 32) * 1e-3
    e = synth.smooth_random_field(c.nz, c.nx, 33)

    def phi(m):
        r = oracle_lib.born_demig(c.v_init, c.geom, m, c.h, c.dt, c.nb) - d
        return 0.5 * float(np.dot(r, r))

    r = oracle_lib.born_demig(c.v_init, c.geom, x, c.h, c.dt, c.nb) - d
    an = float(np.sum(oracle_lib.rtm_mig(c.v_init, c.geom, r, c.h, c.dt, c.nb) * e))
    eps = 1.0
    fd = (phi(x + eps * e) - phi(x - eps * e)) / (2 * eps)
    assert abs(fd - an) <= 1e-10 * abs(an)


def test_normal_operator_symmetric_psd(oracle_lib):
    c = _perturbed_case()

    def N(m):
        return oracle_lib.rtm_mig(c.v_init, c.geom, oracle_lib.born_demig(c.v_init, c.geom, m, c.h, c.dt, c.nb),
                                  c.h, c.dt, c.nb)

    x = synth.gaussian_field((c.nz, c.nx), 41)
    y = synth.gaussian_field((c.nz, c.nx), 42)
    Nx, Ny = N(x), N(y)
    a, b = float(np.sum(x * Ny)), float(np.sum(Nx * y))
    assert abs(a - b) <= 1e-12 * max(abs(a), abs(b))
    Lx = oracle_lib.born_demig(c.v_init, c.geom, x, c.h, c.dt, c.nb)
    q = float(np.sum(x * Nx))
    assert q > 0
    assert q == pytest.approx(float(np.dot(Lx, Lx)), rel=1e-12)
