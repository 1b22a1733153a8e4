"""Every step-kernel variant (cp.async staging with 2/4/8 rows per thread,
TMA staging with 4/8/16, and the two-step time-blocked forward kernel)
computes the same arithmetic in the same order, so records, gradients and
images agree bit for bit across variants, and each matches the FP64 oracle
within 1e-5.  So do the three ways the backward sweep gets a^n: stored
history, checkpoint recompute, or history for some segments only.

The case has odd window widths of different sizes (a common pool pitch
leaves padding columns that the TMA variants read as the zero boundary),
tiles in the sponge-free interior (the TMA fast path) and half of the
receivers deep inside those interior tiles.
"""
import copy

import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import f32, f32_geom, gpu_ctx, rel_l2, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL = 1e-5
VARIANTS = list(range(7))  # 5 and 6: single-stage Born kernels (the others fall back to their last)
TMA_VARIANTS = [3, 4, 5]


def _case():
    c = synth.tiny_case(nz=150, nx=301, nt=220, nb=20, n_shots=3, seed=11)
    g = copy.deepcopy(c.geom)
    g.rec_iz = g.rec_iz.copy()
    g.rec_iz[1::2] = 100
    c.geom = g
    return c


CASE = _case()
DV = f32(synth.gaussian_field((CASE.nz, CASE.nx), seed=12))
KEYS = ("d", "ds", "g", "m", "b")


def _run(variant, monkeypatch, blocking=False):
    import torch

    monkeypatch.setenv("DHFWI_STEP_VARIANT", str(variant))
    monkeypatch.setenv("DHFWI_TIME_BLOCK", "1" if blocking else "0")
    c = CASE
    ctx = gpu_ctx(c)
    geom = f32_geom(c.geom)
    v, v0 = to_dev(f32(c.v_true)), to_dev(f32(c.v_init))
    d = ctx.model_shots(v, geom)
    d_obs = 0.5 * d
    ds = torch.empty(geom.n_data, dtype=torch.float32, device="cuda")
    J, g = ctx.fwi_gradient(v0, geom, d_obs, d_syn=ds)
    m = ctx.rtm_mig(v0, geom, d_obs)
    st = ctx.stats()
    used = st["step_variant"]
    b = ctx.born_demig(v0, geom, to_dev(DV))
    ctx.close()
    return {"d": to_host(d), "ds": to_host(ds), "g": to_host(g), "m": to_host(m), "b": to_host(b), "J": J,
            "history_steps": st["history_steps"], "checkpoint_every": st["checkpoint_every"]}, used


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


@pytest.fixture(scope="module")
def reference_variant():
    mp = pytest.MonkeyPatch()
    try:
        return _run(1, mp)[0]
    finally:
        mp.undo()


@pytest.mark.parametrize("variant", VARIANTS)
def test_variants_agree_bitwise(variant, reference_variant, monkeypatch):
    out, used = _run(variant, monkeypatch)
    assert used[0] == used[1] == min(variant, 5)
    assert used[2] == min(variant, 4) and used[3] == variant
    for k in KEYS:
        np.testing.assert_array_equal(out[k], reference_variant[k], err_msg=k)
    assert out["J"] == reference_variant["J"]


@pytest.mark.parametrize("variant", [1, 4])
def test_two_step_kernel_agrees_bitwise(variant, reference_variant, monkeypatch):
    """Time-blocked forward passes (two steps per launch, also in the
    gradient's segment recompute): the same records, gradient and image bit
    for bit.  Shot 1's record length is odd, so its last launch takes one
    step; nt_max is even and the checkpoint segments are 50 steps."""
    assert CASE.geom.nt[1] % 2 == 1
    out, used = _run(variant, monkeypatch, blocking=True)
    for k in KEYS:
        np.testing.assert_array_equal(out[k], reference_variant[k], err_msg=k)
    assert out["J"] == reference_variant["J"]


def test_autotuned_kernels_and_depth_agree_bitwise(reference_variant, monkeypatch):
    """Nothing pinned: the autotuner picks the variants and the time-blocking
    depth of the forward and adjoint sweeps; the results are the same bits."""
    import torch

    monkeypatch.delenv("DHFWI_STEP_VARIANT", raising=False)
    monkeypatch.delenv("DHFWI_TIME_BLOCK", raising=False)
    c = CASE
    ctx = gpu_ctx(c)
    geom = f32_geom(c.geom)
    v, v0 = to_dev(f32(c.v_true)), to_dev(f32(c.v_init))
    d = ctx.model_shots(v, geom)
    ds = torch.empty(geom.n_data, dtype=torch.float32, device="cuda")
    J, g = ctx.fwi_gradient(v0, geom, 0.5 * d, d_syn=ds)
    st = ctx.stats()
    assert all(x in (1, 2) for x in st["time_block"])
    m = ctx.rtm_mig(v0, geom, 0.5 * d)
    b = ctx.born_demig(v0, geom, to_dev(DV))
    out = {"d": to_host(d), "ds": to_host(ds), "g": to_host(g), "m": to_host(m), "b": to_host(b)}
    ctx.close()
    for k in KEYS:
        np.testing.assert_array_equal(out[k], reference_variant[k], err_msg=k)
    assert J == reference_variant["J"]


def history_cap_mb(case, segs, K=50):
    """MiB that hold the a^n history of the first `segs` segments of K steps:
    each step keeps its active shots (nt > n) as NZ x pitch slots, plus one
    spare pool of all shots."""
    g, nb = case.geom, case.nb
    NZ = case.nz + 2 * nb
    pitch = -(-int((g.win_x1 - g.win_x0).max() + 2 * nb) // 64) * 64
    slot = 4 * NZ * pitch
    nt = np.asarray(g.nt)
    total = slot * len(nt) + sum(int((nt > n).sum()) * slot for n in range(min(segs * K, int(nt.max()))))
    return -(-total // (1 << 20))


@pytest.mark.parametrize("blocking", [False, True])
@pytest.mark.parametrize("history", ["none", "first-segment", "all"])
def test_history_modes_agree_bitwise(history, blocking, reference_variant, monkeypatch):
    """The backward sweep takes a^n from the history stored by the forward
    pass, or recomputes it from checkpoints, or both (a history of the first
    of five segments, the cap set through DHFWI_HISTORY_MB): the same
    records, gradient and image bit for bit."""
    if history == "all":
        monkeypatch.delenv("DHFWI_HISTORY_MB", raising=False)
    else:
        monkeypatch.setenv("DHFWI_HISTORY_MB", "0" if history == "none" else str(history_cap_mb(CASE, 1)))
    out, _ = _run(4, monkeypatch, blocking=blocking)
    K, nt_max = out["checkpoint_every"], int(CASE.geom.nt.max())
    assert K == 50 and -(-nt_max // K) == 5
    assert out["history_steps"] == {"none": 0, "first-segment": K, "all": nt_max}[history]
    for k in KEYS:
        np.testing.assert_array_equal(out[k], reference_variant[k], err_msg=k)
    assert out["J"] == reference_variant["J"]


@pytest.mark.parametrize("variant", TMA_VARIANTS)
def test_tma_variants_match_oracle(variant, oracle_ref, monkeypatch):
    out, _ = _run(variant, monkeypatch)
    for k in KEYS:
        assert rel_l2(out[k], oracle_ref[k]) <= TOL, k
    assert abs(out["J"] - oracle_ref["J"]) <= TOL * abs(oracle_ref["J"])


def test_case_exercises_the_fast_path_and_padding():
    """Host-side check of the case itself: odd, unequal window widths and at
    least one tile fully inside the sponge-free interior with receivers."""
    c, nb, TX = CASE, CASE.nb, 64
    NZ = c.nz + 2 * nb
    widths = [int(x1 - x0) + 2 * nb for x0, x1 in zip(c.geom.win_x0, c.geom.win_x1)]
    assert any(w % 2 for w in widths) and len(set(widths)) > 1
    interior_with_rec = False
    for s, w in enumerate(widths):
        for z0 in range(0, NZ, TX):
            for x0 in range(0, w, TX):
                full = z0 >= nb and z0 + TX <= NZ - nb and x0 >= nb and x0 + TX <= w - nb
                if not full:
                    continue
                lo, hi = c.geom.rec_off[s], c.geom.rec_off[s + 1]
                rz = c.geom.rec_iz[lo:hi] + nb
                rx = c.geom.rec_ix[lo:hi] - c.geom.win_x0[s] + nb
                if np.any((rz >= z0) & (rz < z0 + TX) & (rx >= x0) & (rx < x0 + TX)):
                    interior_with_rec = True
    assert interior_with_rec


@pytest.mark.parametrize("history", ["all", "first-segment", "none"])
def test_reuse_of_the_forward_pass_is_bitwise(history, reference_variant, monkeypatch):
    """dhfwi_set_reuse: after a gradient at v0, the migration at v0 skips its
    forward pass (the history and, beyond it, the checkpoints kept intact by
    the backward sweep's recompute), and Born at v0 advances only the
    scattered field when the history holds every step; the same bits as
    propagating.  At another model nothing is reused."""
    import torch

    monkeypatch.delenv("DHFWI_STEP_VARIANT", raising=False)
    monkeypatch.delenv("DHFWI_TIME_BLOCK", raising=False)
    if history == "all":
        monkeypatch.delenv("DHFWI_HISTORY_MB", raising=False)
    else:
        monkeypatch.setenv("DHFWI_HISTORY_MB", "0" if history == "none" else str(history_cap_mb(CASE, 1)))
    c = CASE
    ctx = gpu_ctx(c)
    ctx.set_reuse(True)
    geom = f32_geom(c.geom)
    v, v0 = to_dev(f32(c.v_true)), to_dev(f32(c.v_init))
    d = ctx.model_shots(v, geom)
    ds = torch.empty(geom.n_data, dtype=torch.float32, device="cuda")
    J, g = ctx.fwi_gradient(v0, geom, 0.5 * d, d_syn=ds)
    b = ctx.born_demig(v0, geom, to_dev(DV))
    assert ctx.stats()["reused"] == (2 if history == "all" else 0)
    m = ctx.rtm_mig(v0, geom, 0.5 * d)
    assert ctx.stats()["reused"] == 1
    out = {"d": to_host(d), "ds": to_host(ds), "g": to_host(g), "m": to_host(m), "b": to_host(b)}
    for k in KEYS:
        np.testing.assert_array_equal(out[k], reference_variant[k], err_msg=k)
    assert J == reference_variant["J"]
    # Another model: propagated again (no stale reuse), equal to a fresh context.
    v1 = v0 + 7.0
    b1 = to_host(ctx.born_demig(v1, geom, to_dev(DV)))
    assert ctx.stats()["reused"] == 0
    m1 = to_host(ctx.rtm_mig(v1, geom, 0.5 * d))
    assert ctx.stats()["reused"] == 0
    ctx.close()
    ref = gpu_ctx(c)
    np.testing.assert_array_equal(b1, to_host(ref.born_demig(v1, geom, to_dev(DV))))
    np.testing.assert_array_equal(m1, to_host(ref.rtm_mig(v1, geom, 0.5 * d)))
    ref.close()
