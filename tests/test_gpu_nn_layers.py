"""Per-layer GPU parity of the deblurring network's convolutions against the
oracle's layer definitions (Appendix A layers: 3x3 convolutions and 2x2
stride-2 transposed convolutions), forward, input gradient and weight
gradient, each within 1e-3 relative L2.

Inputs are rounded to bfloat16 on both sides where the network rounds them
(activations, weights, output gradients); the oracle accumulates in float64,
the GPU in float32.  The shapes reach every GEMM path the network runs: the
8-channel first layer, the 32-channel top level (shared-memory halo tiles),
the tcgen05 kernels for >= 64 output channels (32- and 64-channel sources),
the split-k paths of the deepest levels, M tails (pixel counts that are not a
multiple of the 128-row tile) and the transposed convolutions; each case runs
under every GEMM selection (the default choice, without the patch kernels,
the one-tile-per-CTA and the persistent TMA-fed convolutions forced, the
one-tile and the persistent patch kernels forced, DHFWI_NN_GEMM "mma" and
"tc").
"""
import math

import numpy as np
import pytest

from gpu_helpers import gpu_ctx, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-3

# (ci, co, n, H, W) of 3x3 convolutions.
CONV3 = [
    (8, 32, 2, 20, 24),     # first layer (1 channel padded to 8)
    (32, 32, 3, 17, 23),    # top level; 1173 pixels (M tail), split-k weight gradient
    (64, 32, 2, 16, 16),    # top decoder conv on [skip, up]
    (32, 64, 2, 12, 20),    # down1.0: tcgen05 with a 32-channel source
    (64, 64, 2, 9, 13),     # ragged 16-wide pixel blocks
    (128, 128, 4, 8, 8),
    (256, 512, 8, 4, 4),    # deepest level: few pixels, split-k
    (512, 512, 16, 4, 4),
    (512, 256, 4, 8, 8),    # up1.0 on [skip, up]
    (32, 32, 4, 128, 128),  # the top level of the benchmark's patches: persistent patch kernel by default
    (64, 64, 4, 64, 64),    # 64-channel patches, 128 tiles
]
# (ci, co, n, H, W) of transposed convolutions (H, W: the coarse input grid).
CONVT = [
    (512, 256, 8, 4, 4),
    (128, 64, 3, 5, 7),
    (64, 32, 2, 8, 12),
]
# nopatch: without the patch-reuse tcgen05 kernels (DHFWI_NN_PATCH=0); tile / persistent: also the
# one-tile-per-CTA or the persistent TMA-fed tcgen05 conv kernel forced (DHFWI_NN_CONV); patchtile /
# patchp: the one-tile or the persistent patch kernel forced (DHFWI_NN_PATCH=tile / persistent, the
# latter on two CTAs per N-tile so that each walks many tiles)
MODES = ["default", "nopatch", "tile", "persistent", "patchtile", "patchp", "mma", "tc"]


def _data(seed, kind, ci, co, n, H, W):
    g = np.random.Generator(np.random.PCG64(seed))
    taps = 9 if kind == "conv3" else 4
    Ho, Wo = (H, W) if kind == "conv3" else (2 * H, 2 * W)
    x = g.standard_normal((n, H, W, ci)).astype(np.float32)
    w = (g.standard_normal((co, taps, ci)) / math.sqrt(taps * ci)).astype(np.float32)
    b = (0.1 * g.standard_normal(co)).astype(np.float32)
    gy = g.standard_normal((n, Ho, Wo, co)).astype(np.float32)
    return x, w, b, gy


def _oracle(kind, op, x, w, b, gy):
    from oracle import nn as onn

    co, taps, ci = w.shape
    xb = onn.bf16(x).transpose(0, 3, 1, 2)
    gb = onn.bf16(gy).transpose(0, 3, 1, 2)
    if kind == "conv3":
        Wb = onn.bf16(w).reshape(co, 3, 3, ci)
        if op == "fwd":
            y = onn.bf16(onn.leaky(onn.conv3x3(xb, Wb, b.astype(np.float64)), 0.2))
            return y.transpose(0, 2, 3, 1)
        if op == "dgrad":
            return onn.conv3x3_dgrad(gb, Wb).transpose(0, 2, 3, 1)
        dW, db = onn.conv3x3_wgrad(xb, gb)
    else:
        Wb = onn.bf16(w).reshape(co, 2, 2, ci)
        if op == "fwd":
            return onn.bf16(onn.convT2x2(xb, Wb, b.astype(np.float64))).transpose(0, 2, 3, 1)
        if op == "dgrad":
            return onn.convT2x2_dgrad(gb, Wb).transpose(0, 2, 3, 1)
        dW, db = onn.convT2x2_wgrad(xb, gb)
    return np.concatenate([dW.ravel(), db])


def _run(monkeypatch, mode, kind, shape, seed):
    import torch

    monkeypatch.delenv("DHFWI_NN_CONV", raising=False)
    monkeypatch.delenv("DHFWI_NN_PATCH", raising=False)
    if mode in ("patchtile", "patchp"):
        monkeypatch.delenv("DHFWI_NN_GEMM", raising=False)
        monkeypatch.setenv("DHFWI_NN_PATCH", "tile" if mode == "patchtile" else "persistent")
    elif mode in ("default", "nopatch", "tile", "persistent"):
        monkeypatch.delenv("DHFWI_NN_GEMM", raising=False)
        if mode != "default":
            monkeypatch.setenv("DHFWI_NN_PATCH", "0")
        if mode in ("tile", "persistent"):
            monkeypatch.setenv("DHFWI_NN_CONV", mode)
    else:
        monkeypatch.setenv("DHFWI_NN_GEMM", mode)
    ci, co, n, H, W = shape
    x, w, b, gy = _data(seed, kind, ci, co, n, H, W)
    from synth import tiny_case

    ctx = gpu_ctx(tiny_case())
    dev = lambda a: torch.as_tensor(a, device="cuda").contiguous()
    errs = {}
    for op in ("fwd", "dgrad", "wgrad"):
        out = ctx.deblur_layer(kind, op, x=dev(x), w=dev(w), b=dev(b), gy=dev(gy), n=n, H=H, W=W, ci=ci, co=co)
        got = out.cpu().numpy().astype(np.float64)
        ref = _oracle(kind, op, x, w, b, gy)
        if op == "wgrad":
            nw = w.size
            # Weight and bias gradients are checked separately: the bias
            # gradient is a plain sum with a far smaller norm.
            errs["wgrad"] = rel_l2(got[:nw], ref[:nw])
            errs["bgrad"] = rel_l2(got[nw:], ref[nw:])
        else:
            errs[op] = rel_l2(got.reshape(ref.shape), ref)
    ctx.close()
    assert all(e <= TOL for e in errs.values()), errs


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("shape", CONV3, ids=lambda s: "x".join(map(str, s)))
def test_conv3_layer_parity(monkeypatch, mode, shape):
    _run(monkeypatch, mode, "conv3", shape, seed=sum(shape))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("shape", CONVT, ids=lambda s: "x".join(map(str, s)))
def test_convT_layer_parity(monkeypatch, mode, shape):
    _run(monkeypatch, mode, "convT", shape, seed=7 + sum(shape))


def test_wgrad_mma_path(monkeypatch):
    """The mma.sync weight gradient kept behind DHFWI_NN_WGRAD=mma for the
    layers the tcgen05 one takes by default."""
    monkeypatch.setenv("DHFWI_NN_WGRAD", "mma")
    _run(monkeypatch, "default", "conv3", (128, 128, 4, 8, 8), seed=3)


# (co, n, H, W) of the first layer (one input channel).
FIRST = [(32, 4, 128, 128), (16, 2, 20, 24), (128, 1, 30, 40)]


@pytest.mark.parametrize("shape", FIRST, ids=lambda s: "x".join(map(str, s)))
def test_first_layer_parity(shape):
    """The first 3x3 convolution (one input channel, padded to 8 for the
    GEMMs but run on CUDA cores): forward and weight / bias gradients within
    1e-3 of the oracle's layer."""
    import torch

    co, n, H, W = shape
    x, w, b, gy = _data(sum(shape), "conv3", 1, co, n, H, W)
    from synth import tiny_case

    ctx = gpu_ctx(tiny_case())
    dev = lambda a: torch.as_tensor(a, device="cuda").contiguous()
    errs = {}
    for op in ("fwd", "wgrad"):
        out = ctx.deblur_layer("first", op, x=dev(x), w=dev(w), b=dev(b), gy=dev(gy), n=n, H=H, W=W, ci=1, co=co)
        got = out.cpu().numpy().astype(np.float64)
        ref = _oracle("conv3", op, x, w, b, gy)
        if op == "wgrad":
            nw = w.size
            errs["wgrad"] = rel_l2(got[:nw], ref[:nw])
            errs["bgrad"] = rel_l2(got[nw:], ref[nw:])
        else:
            errs[op] = rel_l2(got.reshape(ref.shape), ref)
    with pytest.raises(Exception):
        ctx.deblur_layer("first", "dgrad", x=dev(x), w=dev(w), b=dev(b), gy=dev(gy), n=n, H=H, W=W, ci=1, co=co)
    ctx.close()
    assert all(e <= TOL for e in errs.values()), errs
