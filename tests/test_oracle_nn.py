"""Pins for the FP64 network oracle (Section 2.4 and Appendix A): each
layer against its definition evaluated by brute force, the backward pass
against central finite differences, Adam and the cosine schedule against
their closed forms, bf16 rounding against torch's conversion, and the
architecture against the channel table printed in Appendix A."""
import math
import os

import numpy as np
import pytest

from oracle import nn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "unet_appendix_a.txt")


def rng(s):
    return np.random.Generator(np.random.PCG64(s))


def test_channel_table_matches_appendix_a():
    spec = nn.UNetSpec(base=128, levels=4)
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    want = {name: int(c) for name, c in rows[1:]}
    got = {}
    for name, kind, ci, co in nn.param_specs(spec):
        key = name.split(".")[0]
        got[key] = co
    for k, c in want.items():
        assert got[k] == c, (k, got[k], c)


def test_conv3x3_matches_direct_sum():
    g = rng(1)
    x = g.standard_normal((2, 3, 5, 6))
    W = g.standard_normal((4, 3, 3, 3))
    b = g.standard_normal(4)
    y = nn.conv3x3(x, W, b)
    ref = np.zeros_like(y)
    for n in range(2):
        for o in range(4):
            for h in range(5):
                for w in range(6):
                    acc = b[o]
                    for c in range(3):
                        for dh in range(3):
                            for dw in range(3):
                                hh, ww = h + dh - 1, w + dw - 1
                                if 0 <= hh < 5 and 0 <= ww < 6:
                                    acc += W[o, dh, dw, c] * x[n, c, hh, ww]
                    ref[n, o, h, w] = acc
    assert np.abs(y - ref).max() < 1e-12


def test_convT_and_pool_match_direct_sum():
    g = rng(2)
    x = g.standard_normal((1, 3, 3, 4))
    W = g.standard_normal((2, 2, 2, 3))
    b = g.standard_normal(2)
    y = nn.convT2x2(x, W, b)
    for o in range(2):
        for h in range(6):
            for w in range(8):
                ref = b[o] + sum(W[o, h % 2, w % 2, i] * x[0, i, h // 2, w // 2] for i in range(3))
                assert abs(y[0, o, h, w] - ref) < 1e-12
    x = g.standard_normal((1, 2, 8, 6))
    p = nn.avgpool3s2(x)
    assert p.shape == (1, 2, 4, 3)
    for c in range(2):
        for i in range(4):
            for j in range(3):
                s = sum(x[0, c, 2 * i + a - 1, 2 * j + bb - 1] for a in range(3) for bb in range(3)
                        if 0 <= 2 * i + a - 1 < 8 and 0 <= 2 * j + bb - 1 < 6)
                assert abs(p[0, c, i, j] - s / 9.0) < 1e-12  # padding counted


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    g = rng(3)
    x = np.concatenate([g.standard_normal(10000) * 10.0 ** g.integers(-8, 8, 10000),
                        [1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-8, -2.5, 0.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(nn.bf16(x), ref)
    assert nn.bf16(1.0 + 2**-8) == 1.0            # tie to even
    assert nn.bf16(1.0 + 3 * 2**-8) == 1.0 + 2**-6


def _tiny():
    spec = nn.UNetSpec(base=2, levels=2)
    flat = nn.init_params(spec, 7).astype(np.float64)
    x = rng(4).standard_normal((2, 1, 8, 8))
    R = rng(5).standard_normal((2, 1, 8, 8))
    return spec, flat, x, R


def test_backward_matches_finite_differences():
    spec, flat, x, R = _tiny()

    def loss(th):
        out, _ = nn.forward(th, x, spec, round_bf16=False)
        return float(np.sum(out * R))

    out, cache = nn.forward(flat, x, spec, round_bf16=False)
    g = nn.backward(flat, cache, R, spec, round_bf16=False)
    for s in range(4):
        e = rng(10 + s).standard_normal(flat.shape)
        eps = 1e-6
        fd = (loss(flat + eps * e) - loss(flat - eps * e)) / (2 * eps)
        an = float(np.dot(g, e))
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (fd, an)
    # Single coordinates in every tensor (catches a transposed or dropped term).
    k = 0
    for name, kind, ci, co in nn.param_specs(spec):
        cnt = int(np.prod(nn.weight_shape(kind, ci, co))) + co
        for idx in (k, k + cnt - 1):
            e = np.zeros_like(flat)
            e[idx] = 1.0
            fd = (loss(flat + 1e-6 * e) - loss(flat - 1e-6 * e)) / 2e-6
            assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(g[idx])), (name, idx)
        k += cnt


def test_backward_with_rounding_is_close_to_exact():
    spec, flat, x, R = _tiny()
    out, cache = nn.forward(flat, x, spec, round_bf16=True)
    gb = nn.backward(flat, cache, R, spec, round_bf16=True)
    out2, cache2 = nn.forward(flat, x, spec, round_bf16=False)
    g = nn.backward(flat, cache2, R, spec, round_bf16=False)
    assert np.linalg.norm(gb - g) <= 0.05 * np.linalg.norm(g)


def test_adam_first_step_closed_form():
    g = rng(6).standard_normal(100)
    th = np.zeros(100)
    th1, m, v = nn.adam_step(th, g, np.zeros(100), np.zeros(100), 1, 1e-3)
    # After bias correction m_hat = g, v_hat = g^2: step = -lr g / (|g| + eps).
    assert np.allclose(th1, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)


def test_cosine_schedule():
    assert nn.cosine_lr(1e-3, 0, 100) == 1e-3
    assert nn.cosine_lr(1e-3, 50, 100) == pytest.approx(5e-4)
    assert nn.cosine_lr(1e-3, 100, 100) == pytest.approx(0.0, abs=1e-18)
    assert nn.cosine_lr(1e-3, 25, 100) == pytest.approx(0.5e-3 * (1 + math.cos(math.pi / 4)))


def test_patches_and_permutation():
    # 400 x 1200 with 128-pixel patches at stride 64, edge aligned: 6 x 18.
    assert len(nn.patch_origins(400, 128, 64)) == 6
    assert len(nn.patch_origins(1200, 128, 64)) == 18
    assert nn.patch_origins(400, 128, 64)[-1] == 272
    p = nn.permutation(108, 29, 3)
    assert sorted(p) == list(range(108)) and p != list(range(108))
    assert p != nn.permutation(108, 29, 4)


def test_init_bounds_and_determinism():
    spec = nn.UNetSpec(base=4, levels=2)
    a = nn.init_params(spec, 29)
    b = nn.init_params(spec, 29)
    assert np.array_equal(a, b) and a.dtype == np.float32
    d = nn.unflatten(a, spec)
    for name, kind, ci, co in nn.param_specs(spec):
        bound = 1 / math.sqrt(nn.fan_in(kind, ci))
        W, bb = d[name]
        assert np.abs(W).max() <= bound and np.abs(bb).max() <= bound
        assert np.abs(W).max() > 0.5 * bound


def test_training_reduces_loss():
    spec = nn.UNetSpec(base=4, levels=2)
    g = rng(8)
    img = np.cumsum(g.standard_normal((24, 40)), axis=1)
    from scipy.ndimage import gaussian_filter

    x = gaussian_filter(img, 1.5)  # blurred input, sharp target
    cfg = nn.TrainCfg(patch=16, stride=8, batch=4, epochs=10, lr=1e-2, seed=1)
    flat = nn.init_params(spec, 3)
    _, hist = nn.train(flat, x, img, spec, cfg)
    assert hist[-1] < 0.7 * hist[0], hist
