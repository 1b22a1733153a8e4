"""GPU parity on the degenerate geometries of the shot batch, against the
FP64 oracle (records, misfit, gradient, Born data, migrated image within
1e-5) and between the one-step and two-step (time-blocked) kernels (bit for
bit):

* receivers sharing a cell, at the surface and at depth (the adjoint sums
  their data in a fixed order before injecting);
* a shot without receivers;
* records of 1, 2 and 3 samples and an odd record length (the two-step
  kernels take a single step at the end of a record);
* a window three columns wide, a window on the model's edge with the source
  next to it;
* a source on a window's edge column;

and with a^n taken from the stored history, recomputed from checkpoints, or
both.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import f32, f32_geom, gpu_ctx, rel_l2, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _case():
    nz, nx, h, dt, nb, nt = 150, 220, 10.0, 1e-3, 20, 160
    g = synth.rng(41)
    v = synth.smooth_model(1800.0 + 400.0 * g.uniform(size=(nz, nx)), 1.5)
    v0 = synth.smooth_model(v, 3.0)
    shots = [
        # (src_iz, src_ix, nt, win_x0, win_x1, receivers [(iz, ix)])
        (3, 110, 160, 40, 180, [(2, x) for x in range(50, 171, 3)] + [(2, 101)] * 3 + [(90, 120)] * 2),
        (5, 10, 1, 0, 60, [(1, x) for x in (0, 5, 10, 20, 59)] + [(5, 10)]),  # one at the source
        (4, 200, 2, 199, 202, [(1, 199), (1, 200), (1, 201)]),
        (2, 150, 3, 100, 200, []),
        (2, 30, 159, 0, 220, [(1, x) for x in range(0, 220, 2)]),
        (6, 149, 157, 100, 150, [(3, x) for x in range(100, 150, 7)]),  # source on the window's last column
    ]
    rec_iz, rec_ix, off = [], [], [0]
    for s in shots:
        rec_iz += [r[0] for r in s[5]]
        rec_ix += [r[1] for r in s[5]]
        off.append(off[-1] + len(s[5]))
    geom = synth.Geometry(
        src_iz=synth._i32([s[0] for s in shots]), src_ix=synth._i32([s[1] for s in shots]),
        nt=synth._i32([s[2] for s in shots]), rec_off=synth._i32(off), rec_iz=synth._i32(rec_iz),
        rec_ix=synth._i32(rec_ix), win_x0=synth._i32([s[3] for s in shots]),
        win_x1=synth._i32([s[4] for s in shots]), wavelet=synth.ricker(20.0, dt, nt), wavelet_shared=True)
    return synth.Case(nz, nx, h, dt, nb, v, v0, geom, name="edge")


CASE = _case()
DV = f32(synth.gaussian_field((CASE.nz, CASE.nx), seed=43))


def _run(blocking, monkeypatch, history_mb=None):
    import torch

    monkeypatch.setenv("DHFWI_TIME_BLOCK", "1" if blocking else "0")
    if history_mb is None:
        monkeypatch.delenv("DHFWI_HISTORY_MB", raising=False)
    else:
        monkeypatch.setenv("DHFWI_HISTORY_MB", str(history_mb))
    c = CASE
    ctx = gpu_ctx(c)
    geom = f32_geom(c.geom)
    v, v0 = to_dev(f32(c.v_true)), to_dev(f32(c.v_init))
    d = ctx.model_shots(v, geom)
    d_obs = 0.5 * d
    ds = torch.empty(geom.n_data, dtype=torch.float32, device="cuda")
    J, g = ctx.fwi_gradient(v0, geom, d_obs, d_syn=ds)
    m = ctx.rtm_mig(v0, geom, d_obs)
    b = ctx.born_demig(v0, geom, to_dev(DV))
    ctx.close()
    return {"d": to_host(d), "ds": to_host(ds), "g": to_host(g), "m": to_host(m), "b": to_host(b), "J": J}


@pytest.fixture(scope="module")
def oracle_ref():
    c = CASE
    geom = f32_geom(c.geom)
    d = oracle.model_shots(f32(c.v_true), geom, c.h, c.dt, c.nb)
    d_obs = f32(0.5 * f32(d))
    J, g, ds = oracle.fwi_gradient(f32(c.v_init), geom, d_obs, c.h, c.dt, c.nb)
    m = oracle.rtm_mig(f32(c.v_init), geom, d_obs, c.h, c.dt, c.nb)
    b = oracle.born_demig(f32(c.v_init), geom, DV, c.h, c.dt, c.nb)
    return {"d": d, "ds": ds, "g": g, "m": m, "b": b, "J": J}


@pytest.mark.parametrize("blocking", [False, True])
def test_edge_geometry_matches_oracle(blocking, oracle_ref, monkeypatch):
    out = _run(blocking, monkeypatch)
    for k in ("d", "ds", "g", "m", "b"):
        assert rel_l2(out[k], oracle_ref[k]) <= TOL, k
    assert abs(out["J"] - oracle_ref["J"]) <= TOL * abs(oracle_ref["J"])
    # Every shot's records on their own (the short ones are invisible in the
    # norm of the whole vector).
    off = CASE.geom.data_offsets()
    for s in range(CASE.geom.n_shots):
        ref = oracle_ref["d"][off[s]:off[s + 1]]
        got = out["d"][off[s]:off[s + 1]]
        scale = max(np.linalg.norm(ref), 1e-30)
        assert np.linalg.norm(got - ref) <= TOL * scale or np.linalg.norm(ref) == 0.0, s


def test_edge_geometry_two_step_bitwise(monkeypatch):
    one = _run(False, monkeypatch)
    two = _run(True, monkeypatch)
    for k in ("d", "ds", "g", "m", "b"):
        np.testing.assert_array_equal(two[k], one[k], err_msg=k)
    assert two["J"] == one["J"]


@pytest.mark.parametrize("history_mb", [0, 40])
def test_edge_geometry_recompute_bitwise(history_mb, monkeypatch):
    """a^n recomputed from checkpoints for every segment (0), or for all but
    the first (a 40 MiB history holds one segment of this case): the same
    results bit for bit as the full history."""
    full = _run(True, monkeypatch)
    part = _run(True, monkeypatch, history_mb)
    for k in ("d", "ds", "g", "m", "b"):
        np.testing.assert_array_equal(part[k], full[k], err_msg=k)
    assert part["J"] == full["J"]


def test_edge_case_layout():
    """Host-side check that the case holds what the docstring lists."""
    g = CASE.geom
    cells = list(zip(g.rec_iz.tolist(), g.rec_ix.tolist()))
    assert len(cells) > len(set(cells))  # shared cells
    assert 0 in np.diff(g.rec_off)  # a shot without receivers
    assert {1, 2, 3} <= set(g.nt.tolist()) and any(n % 2 for n in g.nt.tolist() if n > 3)
    assert (g.win_x1 - g.win_x0).min() == 3
    assert any(g.src_ix[s] == g.win_x1[s] - 1 for s in range(g.n_shots))


def _dense_case():
    """Receivers on five rows of 71 consecutive cells: one tile's grown region
    holds 355 receiver entries, more than the two-step adjoint's in-kernel
    injection list takes, so the plan uses the separate injection pass."""
    nz, nx, h, dt, nb, nt = 120, 160, 10.0, 1e-3, 20, 120
    g = synth.rng(47)
    v = synth.smooth_model(1800.0 + 400.0 * g.uniform(size=(nz, nx)), 1.5)
    v0 = synth.smooth_model(v, 3.0)
    shots = [
        (3, 80, 120, 0, 160, [(z, x) for z in range(1, 6) for x in range(40, 111)]),
        (2, 30, 117, 10, 100, [(1, x) for x in range(10, 100, 3)]),
    ]
    rec_iz, rec_ix, off = [], [], [0]
    for s in shots:
        rec_iz += [r[0] for r in s[5]]
        rec_ix += [r[1] for r in s[5]]
        off.append(off[-1] + len(s[5]))
    geom = synth.Geometry(
        src_iz=synth._i32([s[0] for s in shots]), src_ix=synth._i32([s[1] for s in shots]),
        nt=synth._i32([s[2] for s in shots]), rec_off=synth._i32(off), rec_iz=synth._i32(rec_iz),
        rec_ix=synth._i32(rec_ix), win_x0=synth._i32([s[3] for s in shots]),
        win_x1=synth._i32([s[4] for s in shots]), wavelet=synth.ricker(20.0, dt, nt), wavelet_shared=True)
    return synth.Case(nz, nx, h, dt, nb, v, v0, geom, name="dense")


DENSE = _dense_case()


def _run_dense(blocking, monkeypatch):
    import torch

    monkeypatch.setenv("DHFWI_TIME_BLOCK", "1" if blocking else "0")
    c = DENSE
    ctx = gpu_ctx(c)
    geom = f32_geom(c.geom)
    v, v0 = to_dev(f32(c.v_true)), to_dev(f32(c.v_init))
    d = ctx.model_shots(v, geom)
    d_obs = 0.5 * d
    J, g = ctx.fwi_gradient(v0, geom, d_obs)
    m = ctx.rtm_mig(v0, geom, d_obs)
    ctx.close()
    return {"d": to_host(d), "g": to_host(g), "m": to_host(m), "J": J}


def test_dense_receivers_separate_injection(monkeypatch):
    """The separate injection pass (too many receivers for the in-kernel
    list): gradient and migration match the oracle, and the two-step kernels
    the one-step ones bit for bit."""
    c = DENSE
    geom = f32_geom(c.geom)
    d = oracle.model_shots(f32(c.v_true), geom, c.h, c.dt, c.nb)
    d_obs = f32(0.5 * f32(d))
    J, g, _ = oracle.fwi_gradient(f32(c.v_init), geom, d_obs, c.h, c.dt, c.nb)
    m = oracle.rtm_mig(f32(c.v_init), geom, d_obs, c.h, c.dt, c.nb)
    two = _run_dense(True, monkeypatch)
    assert rel_l2(two["g"], g) <= TOL and rel_l2(two["m"], m) <= TOL
    assert abs(two["J"] - J) <= TOL * abs(J)
    one = _run_dense(False, monkeypatch)
    for k in ("d", "g", "m"):
        np.testing.assert_array_equal(two[k], one[k], err_msg=k)
