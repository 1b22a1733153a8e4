"""CPU tests of the FWI driver's host logic (paper_2403_17518_gb300/fwi.py):
the sequencing of every arm (plain, BB, deblurred, hybrid), the line search
and its fallback, the BB step, band handling and solve counting.

The driver is run against a stand-in context with the C ABI's method names
whose arithmetic is the FP64 oracle (forward modelling, gradient, Born,
migration, the update of Eq. 4 and the BB step of Eq. 17), with a stand-in
network (the identity, or a direction that raises the misfit to force the
fallback).  Nothing here needs a GPU.
"""
import time

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import fwi_step


class CpuTimer:
    def __init__(self):
        self.t = 0.0

    def __enter__(self):
        self.t0 = time.perf_counter()
        return self

    def __exit__(self, *a):
        self.t += time.perf_counter() - self.t0

    def seconds(self):
        return self.t


class FakeContext:
    """The Context API over the oracle (float64 on the host)."""

    def __init__(self, case, bad_network=False):
        self.c = case
        self.device = torch.device("cpu")
        self.bad_network = bad_network
        self.calls = {}

    def _count(self, k):
        self.calls[k] = self.calls.get(k, 0) + 1

    def _geom(self, ga):
        a = ga.arrays
        return synth.Geometry(src_iz=a["src_iz"], src_ix=a["src_ix"], nt=a["nt"], rec_off=a["rec_off"],
                              rec_iz=a["rec_iz"], rec_ix=a["rec_ix"], win_x0=a["win_x0"], win_x1=a["win_x1"],
                              wavelet=ga.wavelet.astype(np.float64), wavelet_shared=True)

    def _g(self, geom):
        return geom if isinstance(geom, synth.Geometry) else self._geom(geom)

    def new_model(self):
        return torch.zeros((self.c.nz, self.c.nx), dtype=torch.float32)

    def new_data(self, ga):
        return torch.zeros(ga.n_data, dtype=torch.float32)

    def model_shots(self, v, geom, out=None):
        self._count("model_shots")
        d = oracle.model_shots(v.double().numpy(), self._g(geom), self.c.h, self.c.dt, self.c.nb)
        t = torch.tensor(d, dtype=torch.float32)
        if out is not None:
            out.copy_(t)
            return out
        return t

    def fwi_gradient(self, v, ga, d_obs, grad=None):
        self._count("fwi_gradient")
        J, g, _ = oracle.fwi_gradient(v.double().numpy(), self._g(ga), d_obs.double().numpy(), self.c.h, self.c.dt,
                                      self.c.nb)
        grad.copy_(torch.tensor(g, dtype=torch.float32))
        return J, grad

    def born_demig(self, v, ga, dv, out=None):
        self._count("born_demig")
        out.copy_(torch.tensor(oracle.born_demig(v.double().numpy(), self._g(ga), dv.double().numpy(), self.c.h,
                                                 self.c.dt, self.c.nb), dtype=torch.float32))
        return out

    def rtm_mig(self, v, ga, d, out=None):
        self._count("rtm_mig")
        out.copy_(torch.tensor(oracle.rtm_mig(v.double().numpy(), self._g(ga), d.double().numpy(), self.c.h,
                                              self.c.dt, self.c.nb), dtype=torch.float32))
        return out

    def deblur_train(self, x, y, warm_start=True, epochs=1, **kw):
        self._count("deblur_train_warm" if warm_start else "deblur_train_cold")
        return np.linspace(1.0, 0.5, epochs)

    def deblur_apply(self, g, out=None):
        self._count("deblur_apply")
        # Identity network, or (bad_network) the ascent direction.
        out.copy_(-g if self.bad_network else g)
        return out

    def fwi_update(self, v, d, alpha, vmin, vmax, mute_rows, out=None):
        self._count("fwi_update")
        r = fwi_step.update(v.double().numpy(), d.double().numpy(), alpha, vmin, vmax, mute_rows)
        out.copy_(torch.tensor(r, dtype=torch.float32))
        return out

    def data_misfit(self, a, b):
        self._count("data_misfit")
        return oracle.misfit(a.double().numpy(), b.double().numpy())

    def bb_step(self, xk, xp, gk, gp, mute_rows=0):
        self._count("bb_step")
        m = mute_rows
        return (fwi_step.bb_short(xk[m:].double().numpy(), xp[m:].double().numpy(), gk[m:].double().numpy(),
                                  gp[m:].double().numpy()), float(gk[m:].abs().max()))


def _case():
    c = synth.tiny_case(nz=21, nx=31, nt=80, nb=6, n_shots=2, seed=14)
    c.v_true = c.v_true.astype(np.float32).astype(np.float64)
    c.v_init = c.v_init.astype(np.float32).astype(np.float64)
    return c


def _run(mode, iters=2, bands=(12.0, 20.0), bad_network=False, hybrid_iters=0):
    from paper_2403_17518_gb300.fwi import run_arm

    c = _case()
    ctx = FakeContext(c, bad_network)
    hist = run_arm(ctx, c, mode, list(bands), iters, dict(base_channels=8), 3, 1, 1500.0, 2600.0, mute_rows=1,
                   hybrid_iters=hybrid_iters, timer=CpuTimer())
    return hist, ctx.calls


def test_plain_arm_sequence_and_descent():
    hist, calls = _run("plain")
    assert len(hist) == 1 + 2 * 2
    # Per iteration: one gradient (2 solves) and a two-trial line search (2 solves).
    assert [r["solves"] for r in hist[1:]] == [4, 8, 12, 16]
    assert calls["fwi_gradient"] == 4 and calls["data_misfit"] == 8
    assert calls.get("born_demig", 0) == 0 and calls.get("bb_step", 0) == 0
    # The misfit of a band falls from its first iteration to its second (the
    # tiny case constrains the model poorly, so its error is not checked).
    assert hist[2]["misfit"] < hist[1]["misfit"] and hist[4]["misfit"] < hist[3]["misfit"]
    assert all(0 < r["alpha"] <= 4 * 0.01 * float(np.mean(_case().v_init)) + 1e-9 for r in hist[1:])


def test_bb_arm_takes_the_short_step_after_the_first_iteration():
    hist, calls = _run("bb", iters=3)
    # The first iteration of each band: line search (no curvature estimate
    # yet); then the step of Eq. 17 with no misfit trials.
    assert calls["bb_step"] == 2 * 2
    a4 = 4 * 0.01 * float(np.mean(_case().v_init))
    # A BB step that is not positive (no curvature estimate) falls back to
    # the line search (two more misfit trials); a positive one is taken,
    # bounded by the line search's largest change.
    n_ls = sum(1 for k in (2, 3, 5, 6) if hist[k]["solves"] - hist[k - 1]["solves"] == 4)
    assert calls["data_misfit"] == 2 * (2 + n_ls)
    assert all(0 <= r["alpha"] <= a4 + 1e-9 for r in hist[1:])
    assert hist[6]["misfit"] < hist[4]["misfit"]


def test_deblurred_arm_trains_cold_per_band_then_warm():
    hist, calls = _run("deblur")
    # Born modelling and its adjoint add two solves per iteration (Section 3.1).
    assert [r["solves"] for r in hist[1:]] == [6, 12, 18, 24]
    assert calls["born_demig"] == calls["rtm_mig"] == calls["deblur_apply"] == 4
    # Re-initialised in each band (cold), warm-started within it.
    assert calls["deblur_train_cold"] == 2 and calls["deblur_train_warm"] == 2
    assert all(r["net"] for r in hist[1:]) and not any(r["fallback"] for r in hist[1:])


def test_network_direction_that_raises_the_misfit_falls_back_to_the_gradient():
    hist, calls = _run("deblur", iters=1, bands=(12.0,), bad_network=True)
    r = hist[1]
    assert r["fallback"] and r["alpha"] > 0
    # gradient 2 + Born pair 2 + failed line search 2, its backtracked
    # trials 2 + gradient line search 2
    assert r["solves"] == 10 and calls["data_misfit"] == 6 and not r["stalled"]


class NoDescentContext(FakeContext):
    """Every line-search trial raises the misfit."""

    def data_misfit(self, a, b):
        self._count("data_misfit")
        return 1e30


def test_a_stalled_band_ends():
    """When no trial, nor a backtracked one, lowers the misfit the iteration
    takes no step and its band ends (the next iteration would repeat it
    exactly)."""
    from paper_2403_17518_gb300.fwi import run_arm

    c = _case()
    ctx = NoDescentContext(c)
    hist = run_arm(ctx, c, "plain", [12.0, 20.0], 5, dict(base_channels=8), 3, 1, 1500.0, 2600.0, mute_rows=1,
                   timer=CpuTimer())
    assert [r["band"] for r in hist[1:]] == [12.0, 20.0]
    assert all(r["stalled"] and r["alpha"] == 0.0 for r in hist[1:])
    assert hist[1]["model_rms"] == hist[0]["model_rms"]
    # gradient 2 + two rounds of trials 4 per band
    assert [r["solves"] for r in hist[1:]] == [6, 12] and ctx.calls["data_misfit"] == 8


def test_hybrid_arm_switches_to_the_gradient():
    hist, calls = _run("hybrid", iters=2, hybrid_iters=3)
    assert [r["net"] for r in hist[1:]] == [True, True, True, False]
    assert calls["born_demig"] == 3


def test_error_at_and_summary():
    from paper_2403_17518_gb300.fwi import error_at, summarize

    a = [{"gpu_s": 0.0, "solves": 0, "model_rms": 10.0}, {"gpu_s": 1.0, "solves": 4, "model_rms": 8.0},
         {"gpu_s": 2.0, "solves": 8, "model_rms": 7.0}]
    b = [{"gpu_s": 0.0, "solves": 0, "model_rms": 10.0}, {"gpu_s": 1.5, "solves": 6, "model_rms": 7.5}]
    assert error_at(a, 1.5) == 8.0 and error_at(a, 2.0) == 7.0 and error_at(a, 0.5) == 10.0
    s = summarize({"a": a, "b": b})
    assert s["equal_gpu_s"] == 1.5 and s["a_model_rms"] == 8.0 and s["b_model_rms"] == 7.5
    assert s["equal_solves"] == 6 and s["a_model_rms_at_solves"] == 8.0
