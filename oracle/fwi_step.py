"""FP64 oracle of the FWI model-update step rules (test infrastructure only).

TEST INFRASTRUCTURE ONLY: used by ``tests/``; the product path never imports
it.  Nothing here is shared with the CUDA library or the product's driver.

* ``update``: the model update of Eq. 4 with the inverse Hessian replaced by
  a scalar step (or by the network, whose output is the direction):
  v_out = clamp(v - alpha * d / max|d|, vmin, vmax), with the direction taken
  as zero in the first mute_rows rows (which are also left out of the max).
* ``parabola_alpha``: the two-trial parabolic line search the driver uses for
  the step length (the paper gives no step rule for its delta m arm): the
  parabola through (0, J0), (a1, J1), (2 a1, J2), its minimiser clamped to
  [0, 4 a1]; a trial set that lowers the misfit nowhere gives 0, and a
  parabola without a minimiser in the interval falls back to the better trial.
* ``bb_short``: the Barzilai-Borwein short step of Section 3.1, Eq. 17,
  alpha = (dx . dg) / (dg . dg) for the differences of two successive models
  and gradients.
"""
from __future__ import annotations

import numpy as np


def update(v, d, alpha, vmin, vmax, mute_rows=0):
    """clamp(v - alpha * d / max|d|, vmin, vmax), d zero in the first mute_rows rows."""
    v = np.asarray(v, dtype=np.float64)
    dm = np.array(d, dtype=np.float64)
    dm[:mute_rows] = 0.0
    scale = np.max(np.abs(dm))
    step = dm / scale if scale > 0 else dm
    return np.minimum(np.maximum(v - alpha * step, vmin), vmax)


def parabola_alpha(J0, J1, J2, a1):
    """Step from the misfits at 0, a1 and 2 a1.  Returns (alpha, improved).

    The quadratic q(a) = c0 + c1 a + c2 a^2 through the three points is found
    by solving its 3 x 3 Vandermonde system; its minimiser -c1 / (2 c2) is used
    when c2 > 0, else the better of the two trials.  The result is clamped to
    [0, 4 a1].  If neither trial lowers the misfit the step is 0; if they do
    but the clamped vertex is 0, the better trial is taken."""
    A = np.array([[1.0, 0.0, 0.0], [1.0, a1, a1 * a1], [1.0, 2 * a1, 4 * a1 * a1]])
    c0, c1, c2 = np.linalg.solve(A, np.array([J0, J1, J2], dtype=np.float64))
    best_trial = a1 if J1 <= J2 else 2 * a1
    alpha = -c1 / (2 * c2) if c2 > 0 else best_trial
    alpha = min(max(alpha, 0.0), 4 * a1)
    improved = min(J1, J2) < J0
    if not improved:
        return 0.0, False
    if alpha == 0.0:
        alpha = best_trial
    return float(alpha), True


def bb_short(x_k, x_km1, g_k, g_km1):
    """Eq. 17: (dx . dg) / (dg . dg), dx = x_k - x_{k-1}, dg = g_k - g_{k-1}."""
    dx = np.ravel(np.asarray(x_k, dtype=np.float64) - np.asarray(x_km1, dtype=np.float64))
    dg = np.ravel(np.asarray(g_k, dtype=np.float64) - np.asarray(g_km1, dtype=np.float64))
    return float(np.dot(dx, dg) / np.dot(dg, dg))
