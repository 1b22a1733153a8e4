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


def test_adam_three_steps_hand_derived():
    """Three Adam steps of one parameter with beta1 = 1/2, beta2 = 3/4, eps = 0,
    lr = 1 and gradients 1, -2, 3, derived by hand:
      t=1: m = 1/2,   v = 1/4,      m^ = 1,   v^ = 1      -> theta = -1
      t=2: m = -3/4,  v = 19/16,    m^ = -1,  v^ = 19/7   -> theta = -1 + sqrt(7/19)
      t=3: m = 9/8,   v = 201/64,   m^ = 9/7, v^ = 201/37 -> theta -= (9/7) sqrt(37/201)
    (swapping the betas, or dropping a bias correction, changes steps 2 and 3)."""
    th, m, v = np.zeros(1), np.zeros(1), np.zeros(1)
    out = []
    for t, g in enumerate((1.0, -2.0, 3.0), start=1):
        th, m, v = nn.adam_step(th, np.array([g]), m, v, t, 1.0, b1=0.5, b2=0.75, eps=0.0)
        out.append((float(th[0]), float(m[0]), float(v[0])))
    th2 = -1.0 + math.sqrt(7.0 / 19.0)
    th3 = th2 - (9.0 / 7.0) * math.sqrt(37.0 / 201.0)
    ref = [(-1.0, 0.5, 0.25), (th2, -0.75, 19.0 / 16.0), (th3, 9.0 / 8.0, 201.0 / 64.0)]
    for got, want in zip(out, ref):
        assert got == pytest.approx(want, rel=1e-14, abs=1e-15)


def test_train_learning_rate_sequence(monkeypatch):
    """The rate train() passes to Adam: lr0 (1 + cos(pi t / T)) / 2 times the
    warm-up factor min(1, (t+1)/W), W = ceil(warmup_frac T), with Adam's step
    count t+1.  3 patches, batch 2 -> 2 steps per epoch, 2 epochs -> T = 4;
    warmup_frac 0.5 -> W = 2."""
    seen = []
    real = nn.adam_step

    def spy(theta, grad, m, v, t, lr, *a, **k):
        seen.append((t, lr))
        return real(theta, grad, m, v, t, lr, *a, **k)

    monkeypatch.setattr(nn, "adam_step", spy)
    spec = nn.UNetSpec(base=4, levels=1)
    g = rng(3)
    img = g.standard_normal((8, 16))
    cfg = nn.TrainCfg(patch=8, stride=4, batch=2, epochs=2, lr=0.4, seed=2, warmup_frac=0.5)
    nn.train(nn.init_params(spec, 1), img, img, spec, cfg)
    lr0 = 0.4
    want = [(1, lr0 * 0.5), (2, 0.5 * lr0 * (1 + math.cos(math.pi / 4))), (3, 0.5 * lr0),
            (4, 0.5 * lr0 * (1 + math.cos(3 * math.pi / 4)))]
    assert [t for t, _ in seen] == [t for t, _ in want]
    for (_, a), (_, b) in zip(seen, want):
        assert a == pytest.approx(b, rel=1e-14)


def test_normalize_mutes_and_scales():
    img = np.array([[900.0, -1000.0, 5.0], [1.0, -3.0, 2.0], [0.5, 1.5, -2.5]])
    out, m = nn.normalize(img, mute_rows=1)
    assert m == 3.0
    assert np.array_equal(out, np.array([[0.0, 0.0, 0.0], [1 / 3, -1.0, 2 / 3], [0.5 / 3, 0.5, -2.5 / 3]]))
    out0, m0 = nn.normalize(img)
    assert m0 == 1000.0 and out0[0, 1] == -1.0


def test_train_sees_muted_normalised_patches(monkeypatch):
    """The patches train() feeds the network: rows above mute_rows zero, the
    rest scaled by the max below the mute (so the largest |value| is 1)."""
    batches = []
    real = nn.forward

    def spy(flat, x, spec, round_bf16=True):
        batches.append(np.array(x))
        return real(flat, x, spec, round_bf16)

    monkeypatch.setattr(nn, "forward", spy)
    spec = nn.UNetSpec(base=4, levels=1)
    g = rng(4)
    img = g.standard_normal((8, 12))
    img[:2] = 50.0  # the footprint rows that the mute removes
    cfg = nn.TrainCfg(patch=8, stride=4, batch=8, epochs=1, lr=1e-3, seed=2, mute_rows=2)
    nn.train(nn.init_params(spec, 1), img, img, spec, cfg)
    X = np.concatenate(batches)
    assert X.shape == (2, 1, 8, 8)
    assert np.all(X[:, :, :2] == 0.0)
    assert np.abs(X).max() == 1.0
    ref = img / np.abs(img[2:]).max()
    got = sorted(float(X[k, 0, 2:].sum()) for k in range(2))
    exp = sorted(float(ref[2:, x0:x0 + 8].sum()) for x0 in (0, 4))
    assert got == pytest.approx(exp, rel=1e-12)


def test_apply_pads_crops_and_rescales(monkeypatch):
    """apply(): the network sees the muted image over its max, zero-padded at
    the bottom and right to a multiple of 2^levels; its output is cropped
    back and multiplied by that max (checked with a stand-in network)."""
    seen = []

    def fake(flat, x, spec, round_bf16=True):
        seen.append(np.array(x))
        H, W = x.shape[2:]
        ramp = np.arange(H * W, dtype=np.float64).reshape(1, 1, H, W)
        return 3.0 * x + ramp, None

    monkeypatch.setattr(nn, "forward", fake)
    spec = nn.UNetSpec(base=4, levels=2)
    g = rng(5)
    img = g.standard_normal((13, 22))
    out = nn.apply(None, img, spec, mute_rows=3)
    (x,) = seen
    assert x.shape == (1, 1, 16, 24)
    m = np.abs(img[3:]).max()
    exp_in = np.zeros((16, 24))
    exp_in[3:13, :22] = img[3:] / m
    assert np.array_equal(x[0, 0], exp_in)
    ramp = np.arange(16 * 24, dtype=np.float64).reshape(16, 24)
    assert np.allclose(out, (3.0 * exp_in + ramp)[:13, :22] * m, rtol=1e-15, atol=0)


def test_apply_is_scale_equivariant():
    """apply(c g) = c apply(g) for c > 0: the normalisation takes out the
    scale and the output rescaling puts it back (exactly, in exact arithmetic;
    here with bfloat16 rounding off)."""
    spec = nn.UNetSpec(base=4, levels=2)
    flat = nn.init_params(spec, 11)
    img = rng(6).standard_normal((16, 20))
    a = nn.apply(flat, img, spec, round_bf16=False, mute_rows=2)
    b = nn.apply(flat, 7.25 * img, spec, round_bf16=False, mute_rows=2)
    assert np.allclose(b, 7.25 * a, rtol=1e-12, atol=1e-12 * np.abs(b).max())


def test_full_image_training_is_the_one_patch_case():
    """patch 0 (the whole image, padded to a multiple of 2^levels, as the
    only sample) gives exactly the patch-mode training whose single patch is
    the whole image, when the image needs no padding."""
    spec = nn.UNetSpec(base=4, levels=2)
    g = rng(12)
    img = g.standard_normal((16, 16))
    x = img + 0.3 * g.standard_normal((16, 16))
    flat = nn.init_params(spec, 2)
    a = nn.train(flat, x, img, spec, nn.TrainCfg(patch=0, epochs=3, lr=1e-2, seed=1, mute_rows=2))
    b = nn.train(flat, x, img, spec, nn.TrainCfg(patch=16, stride=8, batch=4, epochs=3, lr=1e-2, seed=1,
                                                   mute_rows=2))
    assert np.array_equal(a[0], b[0]) and a[1] == b[1]


def test_full_image_training_pads_the_sample(monkeypatch):
    """A 13 x 22 image trains as one 16 x 24 sample, zero outside the image."""
    seen = []
    real = nn.forward

    def spy(flat, x, spec, round_bf16=True):
        seen.append(np.array(x))
        return real(flat, x, spec, round_bf16)

    monkeypatch.setattr(nn, "forward", spy)
    spec = nn.UNetSpec(base=4, levels=2)
    img = rng(13).standard_normal((13, 22))
    _, hist = nn.train(nn.init_params(spec, 2), img, img, spec, nn.TrainCfg(patch=0, epochs=2, lr=1e-3, seed=1))
    assert len(hist) == 2 and len(seen) == 2
    x = seen[0]
    assert x.shape == (1, 1, 16, 24)
    assert np.all(x[0, 0, 13:] == 0) and np.all(x[0, 0, :, 22:] == 0)
    assert np.array_equal(x[0, 0, :13, :22], img / np.abs(img).max())
