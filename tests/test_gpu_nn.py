"""GPU parity of the deblurring network against the FP64 oracle that rounds
operands to bfloat16 at the same points (Section 2.4 / Appendix A).

Tolerances: bitwise initialisation; network output and whole parameter
gradient relative L2 <= 1e-2 end to end; each parameter tensor's gradient
<= 0.1.  The per-tensor bound comes from the oracle's own sensitivity: bf16
rounding decisions flip when pre-rounding values move by as little as 1e-7
relative (below float32 accumulation error), and perturbing the oracle that
way moves its deeper tensors' gradients by 5-7 % (whole gradient 0.35 %).  A
wrong layout in a layer gives ~100 %.  Training: per-epoch loss within 2e-2;
weights after 24 Adam steps within 0.1 (Adam's sign-like steps amplify the
same flips).  All calls go through the C ABI.
"""
import numpy as np
import pytest

from gpu_helpers import rel_l2
from oracle import nn as onn

pytestmark = pytest.mark.gpu


def _ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_17518_gb300 import build
    from paper_2403_17518_gb300.ops import Context

    build()
    return Context(16, 16, 10.0, 1e-3, 4)


def _dev(a):
    import torch

    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


@pytest.mark.parametrize("base,levels", [(8, 2), (16, 3)])
def test_init_is_bitwise_identical(base, levels):
    ctx = _ctx()
    ctx.net_init(base, levels, seed=5)
    spec = onn.UNetSpec(base=base, levels=levels)
    assert ctx.net_size() == onn.n_params(spec)
    assert np.array_equal(ctx.net_get(), onn.init_params(spec, 5))


# The convolution GEMMs: mma.sync with per-tap gathers (halo tiles off),
# mma.sync with the shared-memory halo tile for 3x3 convolutions (the
# default), tcgen05 for the other forward-form GEMMs.
GEMMS = ["mma", "halo", "tc", "default"]


def _set_gemm(monkeypatch, gemm):
    """mma: mma.sync gathering kernels only; halo: mma.sync with halo tiles;
    tc: the cp.async-fed tcgen05 kernel for every forward-form GEMM (with the
    mma.sync weight gradient); default: the TMA-fed tcgen05 kernels for the
    3x3 convolutions with >= 64 channels (forward, input gradient and weight
    gradient), mma.sync halo tiles for the rest."""
    if gemm == "default":
        monkeypatch.delenv("DHFWI_NN_GEMM", raising=False)
        monkeypatch.delenv("DHFWI_NN_WGRAD", raising=False)
    else:
        monkeypatch.setenv("DHFWI_NN_GEMM", "tc" if gemm == "tc" else "mma")
        monkeypatch.setenv("DHFWI_NN_WGRAD", "mma")
    monkeypatch.setenv("DHFWI_NN_HALO", "0" if gemm == "mma" else "1")


@pytest.mark.parametrize("gemm", GEMMS)
@pytest.mark.parametrize("base,levels,n,h,w", [(8, 2, 2, 32, 32), (16, 3, 3, 24, 40), (32, 4, 2, 128, 128)])
def test_forward_and_gradient_parity(base, levels, n, h, w, gemm, monkeypatch):
    _set_gemm(monkeypatch, gemm)
    ctx = _ctx()
    spec = onn.UNetSpec(base=base, levels=levels)
    ctx.net_init(base, levels, seed=11)
    g = np.random.Generator(np.random.PCG64(3))
    x = g.standard_normal((n, h, w)).astype(np.float32)
    y = g.standard_normal((n, h, w)).astype(np.float32)
    out = ctx.deblur_forward(_dev(x)).cpu().numpy()
    flat = onn.init_params(spec, 11)
    ref, cache = onn.forward(flat, x[:, None].astype(np.float64), spec)
    assert rel_l2(out, ref[:, 0]) <= 1e-2
    loss, grad = ctx.deblur_grad(_dev(x), _dev(y))
    lref, dout = onn.mse(ref, y[:, None].astype(np.float64))
    gref = onn.backward(flat, cache, dout, spec)
    assert abs(loss - lref) <= 1e-3 * lref
    grad = grad.cpu().numpy()
    assert rel_l2(grad, gref) <= 1e-2
    # Every tensor individually (catches a wrong layout in one layer).
    k = 0
    for name, kind, ci, co in onn.param_specs(spec):
        cnt = int(np.prod(onn.weight_shape(kind, ci, co))) + co
        assert rel_l2(grad[k:k + cnt], gref[k:k + cnt]) <= 0.1, name
        k += cnt


def test_gradient_is_deterministic():
    ctx = _ctx()
    ctx.net_init(8, 2, seed=1)
    g = np.random.Generator(np.random.PCG64(9))
    x, y = _dev(g.standard_normal((4, 32, 32))), _dev(g.standard_normal((4, 32, 32)))
    l1, g1 = ctx.deblur_grad(x, y)
    l2, g2 = ctx.deblur_grad(x, y)
    assert l1 == l2 and bool((g1 == g2).all())


@pytest.mark.parametrize("gemm", GEMMS)
def test_training_and_apply_parity(gemm, monkeypatch):
    _set_gemm(monkeypatch, gemm)
    ctx = _ctx()
    from scipy.ndimage import gaussian_filter

    g = np.random.Generator(np.random.PCG64(8))
    img = np.cumsum(g.standard_normal((40, 72)), axis=1)
    x = gaussian_filter(img, 1.5).astype(np.float32)
    y = img.astype(np.float32)
    spec = onn.UNetSpec(base=8, levels=2)
    cfg = onn.TrainCfg(patch=16, stride=8, batch=4, epochs=3, lr=1e-2, seed=4)
    hist = ctx.deblur_train(_dev(x), _dev(y), warm_start=False, base_channels=8, levels=2, patch=16, stride=8,
                            batch=4, epochs=3, lr=1e-2, seed=4)
    theta, href = onn.train(onn.init_params(spec, 4), x.astype(np.float64), y.astype(np.float64), spec, cfg)
    assert np.allclose(hist, href, rtol=2e-2), (hist, href)
    w = ctx.net_get()
    assert rel_l2(w, theta) <= 0.1
    out = ctx.deblur_apply(_dev(y)).cpu().numpy()
    ref = onn.apply(w.astype(np.float64), y.astype(np.float64), spec)
    assert rel_l2(out, ref) <= 1e-2
    # Warm start continues from the trained weights (lower first-epoch loss).
    hist2 = ctx.deblur_train(_dev(x), _dev(y), warm_start=True, base_channels=8, levels=2, patch=16, stride=8,
                             batch=4, epochs=1, lr=1e-2, seed=4)
    assert hist2[0] < hist[0]
    # Muted top rows and a learning-rate warm-up: training and apply match the oracle.
    ctx.net_set(w)
    hist3 = ctx.deblur_train(_dev(x), _dev(y), warm_start=True, base_channels=8, levels=2, patch=16, stride=8,
                             batch=4, epochs=2, lr=1e-2, seed=4, mute_rows=5, warmup_frac=0.25)
    cfg3 = onn.TrainCfg(patch=16, stride=8, batch=4, epochs=2, lr=1e-2, seed=4, mute_rows=5, warmup_frac=0.25)
    w3, href3 = onn.train(w.astype(np.float64), x.astype(np.float64), y.astype(np.float64), spec, cfg3)
    assert np.allclose(hist3, href3, rtol=2e-2), (hist3, href3)
    out3 = ctx.deblur_apply(_dev(y)).cpu().numpy()
    ref3 = onn.apply(ctx.net_get().astype(np.float64), y.astype(np.float64), spec, mute_rows=5)
    assert rel_l2(out3, ref3) <= 1e-2


def test_training_parity_base32():
    """Training at the workload's width (base 32, 4 levels) on 64 x 64
    patches, so the default tcgen05 kernels (3x3 convolutions and weight
    gradients of every level below the top) run inside the training loop."""
    ctx = _ctx()
    from scipy.ndimage import gaussian_filter

    g = np.random.Generator(np.random.PCG64(31))
    img = np.cumsum(g.standard_normal((64, 128)), axis=1)
    x = gaussian_filter(img, 2.0).astype(np.float32)
    y = img.astype(np.float32)
    spec = onn.UNetSpec(base=32, levels=4)
    cfg = onn.TrainCfg(patch=64, stride=32, batch=3, epochs=2, lr=1e-3, seed=6)
    hist = ctx.deblur_train(_dev(x), _dev(y), warm_start=False, base_channels=32, levels=4, patch=64, stride=32,
                            batch=3, epochs=2, lr=1e-3, seed=6)
    theta, href = onn.train(onn.init_params(spec, 6), x.astype(np.float64), y.astype(np.float64), spec, cfg)
    assert np.allclose(hist, href, rtol=2e-2), (hist, href)
    w = ctx.net_get()
    assert rel_l2(w, theta) <= 0.1
    out = ctx.deblur_apply(_dev(y)).cpu().numpy()
    ref = onn.apply(w.astype(np.float64), y.astype(np.float64), spec)
    assert rel_l2(out, ref) <= 1e-2


@pytest.mark.parametrize("overlap", ["1", "0"])
def test_graph_replay_is_bitwise_eager(overlap, monkeypatch):
    """A pass is run eagerly the first time its shape is seen, captured into a
    CUDA graph the second time and replayed after: training (two batch
    sizes: 40 patches in batches of 12 leave a tail of 4), the full-image
    apply and the gradient give the same bits as with every pass eager
    (DHFWI_NN_GRAPH=0), with and without the side stream of the weight
    gradients."""
    from scipy.ndimage import gaussian_filter

    monkeypatch.setenv("DHFWI_NN_OVERLAP", overlap)
    g = np.random.Generator(np.random.PCG64(41))
    img = np.cumsum(g.standard_normal((80, 176)), axis=1)
    x = gaussian_filter(img, 2.0).astype(np.float32)
    y = img.astype(np.float32)
    kw = dict(base_channels=32, levels=4, patch=32, stride=16, batch=12, lr=1e-3, seed=6)
    res = {}
    for graph in ("1", "0"):
        monkeypatch.setenv("DHFWI_NN_GRAPH", graph)
        ctx = _ctx()
        hist = ctx.deblur_train(_dev(x), _dev(y), warm_start=False, epochs=4, **kw)
        outs = [ctx.deblur_apply(_dev(y)).cpu().numpy() for _ in range(3)]
        grads = [ctx.deblur_grad(_dev(x[:64, :64].reshape(1, 64, 64)), _dev(y[:64, :64].reshape(1, 64, 64)))
                 for _ in range(3)]
        res[graph] = (np.asarray(hist), ctx.net_get(), outs, [(l, gr.cpu().numpy()) for l, gr in grads])
    (h1, w1, o1, g1), (h0, w0, o0, g0) = res["1"], res["0"]
    assert np.array_equal(h1, h0) and np.array_equal(w1, w0)
    assert all(np.array_equal(a, b) for a, b in zip(o1, o0))
    assert all(l1 == l0 and np.array_equal(a, b) for (l1, a), (l0, b) in zip(g1, g0))


@pytest.mark.parametrize("base,levels,shape,epochs,lr", [(8, 2, (38, 70), 4, 1e-2), (128, 4, (30, 40), 2, 1e-4)],
                         ids=["base8", "paper-size-base128"])
def test_full_image_training_parity(base, levels, shape, epochs, lr):
    """Full-image training (patch 0, the paper's choice): the whole image,
    padded to a multiple of 2^levels, is the one sample of every step.  Also
    at the paper's width (base 128 doubling to 2048 channels, four levels)."""
    ctx = _ctx()
    from scipy.ndimage import gaussian_filter

    g = np.random.Generator(np.random.PCG64(40 + base))
    img = np.cumsum(g.standard_normal(shape), axis=1)
    x = gaussian_filter(img, 1.5).astype(np.float32)
    y = img.astype(np.float32)
    spec = onn.UNetSpec(base=base, levels=levels)
    cfg = onn.TrainCfg(patch=0, epochs=epochs, lr=lr, seed=5, mute_rows=3)
    hist = ctx.deblur_train(_dev(x), _dev(y), warm_start=False, base_channels=base, levels=levels, patch=0,
                            epochs=epochs, lr=lr, seed=5, mute_rows=3)
    theta, href = onn.train(onn.init_params(spec, 5), x.astype(np.float64), y.astype(np.float64), spec, cfg)
    assert np.allclose(hist, href, rtol=2e-2), (hist, href)
    w = ctx.net_get()
    assert w.size == onn.n_params(spec)
    assert rel_l2(w, theta) <= 0.1
    out = ctx.deblur_apply(_dev(y)).cpu().numpy()
    ref = onn.apply(w.astype(np.float64), y.astype(np.float64), spec, mute_rows=3)
    assert rel_l2(out, ref) <= 1e-2


def test_network_errors():
    ctx = _ctx()
    from paper_2403_17518_gb300.ops import DhfwiError

    with pytest.raises(DhfwiError, match="STATE"):
        ctx.deblur_apply(_dev(np.ones((16, 16))))
    with pytest.raises(DhfwiError, match="ARG"):
        ctx.deblur_train(_dev(np.ones((16, 16))), _dev(np.ones((16, 16))), base_channels=12)
    ctx.net_init(8, 2, 1)
    with pytest.raises(DhfwiError, match="ARG"):
        ctx.deblur_forward(_dev(np.ones((1, 18, 16))))
