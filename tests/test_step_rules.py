"""CPU pins of the model-update step rules (oracle/fwi_step.py) and of the
driver's host logic (paper_2403_17518_gb300/fwi.py): the update of Eq. 4
with a scalar step, the two-trial parabolic line search, the
Barzilai-Borwein short step (Eq. 17) and the zero-phase band low-pass.
"""
import math

import numpy as np
import pytest

from oracle import fwi_step as ofs


# --------------------------------------------------------------------------
# Oracle pins
# --------------------------------------------------------------------------
def test_update_hand_values():
    v = np.array([[2000.0, 2000.0], [2000.0, 1600.0], [2000.0, 4400.0]])
    d = np.array([[500.0, -900.0], [2.0, -4.0], [1.0, 3.0]])  # row 0 muted: max |d| below is 4
    out = ofs.update(v, d, alpha=100.0, vmin=1500.0, vmax=4450.0, mute_rows=1)
    # v - 100 * d / 4, clamped to [1500, 4450]; the muted row is unchanged.
    ref = np.array([[2000.0, 2000.0], [1950.0, 1700.0], [1975.0, 4325.0]])
    assert np.array_equal(out, ref)
    # Clamping at both ends.
    out = ofs.update(v, d, alpha=4000.0, vmin=1500.0, vmax=4450.0, mute_rows=1)
    assert out[1, 0] == 1500.0 and out[1, 1] == 4450.0 and out[2, 1] == 1500.0


def test_parabola_alpha_recovers_the_vertex():
    a1 = 20.0
    for a_star in (12.0, 20.0, 33.3, 71.0):  # a trial must improve: a_star > a1 / 2
        J = lambda a: 3.5 * (a - a_star) ** 2 + 10.0
        alpha, ok = ofs.parabola_alpha(J(0), J(a1), J(2 * a1), a1)
        assert ok and alpha == pytest.approx(a_star, rel=1e-12)
    # Vertex beyond 4 a1: clamped.
    J = lambda a: (a - 500.0) ** 2
    assert ofs.parabola_alpha(J(0), J(a1), J(2 * a1), a1) == (4 * a1, True)
    # Neither trial lowers the misfit: no step.
    assert ofs.parabola_alpha(1.0, 1.5, 3.0, a1) == (0.0, False)
    # Concave (no minimiser) but improving: the better trial (then always the second).
    assert ofs.parabola_alpha(10.0, 9.8, 9.0, a1) == (2 * a1, True)
    assert ofs.parabola_alpha(10.0, 9.9, 9.0, a1) == (2 * a1, True)


def test_bb_short_step_is_the_inverse_curvature():
    g = np.random.Generator(np.random.PCG64(3))
    # J = 1/2 lam |x|^2: the gradient difference is lam dx, alpha = 1 / lam.
    lam = 2.75
    x0, x1 = g.standard_normal(50), g.standard_normal(50)
    assert ofs.bb_short(x1, x0, lam * x1, lam * x0) == pytest.approx(1 / lam, rel=1e-14)
    # J = 1/2 x^T A x, A diagonal: alpha = dx.A dx / dx.A^2 dx lies in [1/lam_max, 1/lam_min].
    A = np.linspace(0.5, 8.0, 50)
    a = ofs.bb_short(x1, x0, A * x1, A * x0)
    dx = x1 - x0
    assert a == pytest.approx(np.dot(dx, A * dx) / np.dot(A * dx, A * dx), rel=1e-13)
    assert 1 / 8.0 <= a <= 1 / 0.5
    # Swapping the roles of x and g gives the long step (Eq. 16), not the short one.
    assert ofs.bb_short(A * x1, A * x0, x1, x0) != pytest.approx(a)


# --------------------------------------------------------------------------
# The driver's host logic against the oracle and the closed forms
# --------------------------------------------------------------------------
def test_driver_parabolic_alpha_matches_oracle():
    from paper_2403_17518_gb300.fwi import parabolic_alpha

    g = np.random.Generator(np.random.PCG64(9))
    a1 = 37.5
    for _ in range(500):
        J0, J1, J2 = g.uniform(0.5, 2.0, 3)
        a, ok = parabolic_alpha(J0, J1, J2, a1)
        b, okb = ofs.parabola_alpha(J0, J1, J2, a1)
        assert ok == okb and a == pytest.approx(b, rel=1e-9, abs=1e-9)
    for a_star in (20.0, 50.0, 149.0):
        J = lambda a: 0.25 * (a - a_star) ** 2 + 1.0
        a, ok = parabolic_alpha(J(0), J(a1), J(2 * a1), a1)
        assert ok and a == pytest.approx(a_star, rel=1e-12)


def _lowpass():
    from paper_2403_17518_gb300.fwi import lowpass

    return lowpass


def test_lowpass_is_zero_phase():
    lowpass = _lowpass()
    n, dt = 1001, 1e-3
    x = np.zeros(n)
    x[500] = 1.0
    y = lowpass(x, dt, 8.0)
    k = np.arange(1, 480)
    assert np.abs(y[500 + k] - y[500 - k]).max() <= 1e-12 * np.abs(y).max()
    assert np.argmax(y) == 500


def test_lowpass_passes_below_and_stops_above():
    lowpass = _lowpass()
    n, dt, fc = 4000, 1e-3, 5.0
    t = np.arange(n) * dt
    win = np.sin(np.pi * np.arange(n) / (n - 1)) ** 2  # Hann window: little leakage
    low = win * (np.sin(2 * np.pi * 1.5 * t) + 0.5 * np.cos(2 * np.pi * 3.0 * t + 0.3))
    high = win * (np.sin(2 * np.pi * 9.0 * t) + np.cos(2 * np.pi * 14.0 * t))
    assert np.abs(lowpass(low, dt, fc) - low).max() <= 2e-3 * np.abs(low).max()
    assert np.abs(lowpass(high, dt, fc)).max() <= 2e-3 * np.abs(high).max()
    # Linear, and along any axis.
    both = np.stack([low, high], axis=1)
    out = lowpass(both, dt, fc, axis=0)
    assert np.allclose(out[:, 0], lowpass(low, dt, fc), atol=1e-12)
    assert np.allclose(out[:, 1], lowpass(high, dt, fc), atol=1e-12)


def test_lowpass_taper_midpoint():
    """Half gain at the middle of the cosine taper (1.125 fc)."""
    lowpass = _lowpass()
    n, dt, fc = 8192, 1e-3, 8.0
    t = np.arange(n) * dt
    f = 1.125 * fc
    win = np.sin(np.pi * np.arange(n) / (n - 1)) ** 2
    x = win * np.sin(2 * np.pi * f * t)
    y = lowpass(x, dt, fc)
    mid = slice(n // 4, 3 * n // 4)
    ratio = np.dot(y[mid], x[mid]) / np.dot(x[mid], x[mid])
    assert ratio == pytest.approx(0.5, abs=0.02)


def test_bb_iteration_on_a_quadratic_converges():
    """Host logic of the BB arm on J = 1/2 x^T A x: a first scalar step, then
    x_{k+1} = x_k - alpha_k g_k with the oracle's Eq. 17 step."""
    A = np.linspace(1.0, 20.0, 40)
    x_prev = np.ones(40)
    g_prev = A * x_prev
    x = x_prev - 0.01 * g_prev
    for _ in range(60):
        g = A * x
        a = ofs.bb_short(x, x_prev, g, g_prev)
        x_prev, g_prev = x, g
        x = x - a * g
    assert np.linalg.norm(x) <= 1e-6 * math.sqrt(40)
