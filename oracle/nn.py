"""FP64 oracle of the deblurring network (test infrastructure only).

The network of Section 2.4 / Appendix A of arXiv 2403.17518: a UNet-like
encoder-decoder.  Input block = two (3x3 conv, stride 1, pad 1, LeakyReLU
0.2); `levels` down blocks = AvgPool 3x3 stride 2 then a double conv,
channels doubling; `levels` up blocks = transposed conv halving the channels,
concatenation with the encoder output of the same resolution, double conv;
output = 1x1 conv to one channel.  Trained with MSE and Adam under a cosine
annealing schedule (Section 2.4), mapping the doubly migrated image to the
gradient (Section 2.3.1).

Readings where the paper is silent (shared with the CUDA path by
specification only): AvgPool padding 1 counting the padding; transposed conv
kernel 2x2 stride 2; concatenation order [skip, up]; biases in every conv;
Adam betas (0.9, 0.999), eps 1e-8, fresh moments at each training session,
an optional linear learning-rate warm-up over the first steps of a session;
lr_t = lr0 (1 + cos(pi t / T)) / 2; Kaiming-uniform init bound 1/sqrt(fan_in)
drawn from SplitMix64; LeakyReLU derivative 0.2 at 0.

Precision model of the CUDA path, reproduced here: every convolution
operand (weights, activations, output gradients) is rounded to bfloat16
(round to nearest even) where the CUDA path stores or feeds it; products are
accumulated in float64 here (float32 on the GPU); bias, LeakyReLU, pooling,
loss and Adam run in float64 here (float32 on the GPU).  `round_bf16=False`
turns the rounding off (for finite-difference checks).

Layouts: images NCHW here; parameters are one flat float32 vector, tensor by
tensor in `param_specs` order: 3x3 conv weight [Cout][3][3][Cin] then bias
[Cout]; transposed conv weight [Cout][2][2][Cin] (output (2h+a, 2w+b) gets
W[co][a][b][:] . x[h][w]) then bias; 1x1 conv weight [Cout][Cin] then bias.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


# --------------------------------------------------------------------------
# Counter-based generator: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014)
# --------------------------------------------------------------------------
def splitmix64(x: int) -> int:
    """The SplitMix64 output function applied to state x (already advanced)."""
    z = x & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def rand_u64(seed: int, counter: int) -> int:
    """Value number `counter` of the stream `seed`: state = seed + (counter+1) * golden."""
    return splitmix64((seed + (counter + 1) * GOLDEN) & MASK64)


def rand_unit_f32(seed: int, counter: int) -> np.float32:
    """Uniform in [0, 1) with 24 random bits, exactly representable in float32."""
    return np.float32((rand_u64(seed, counter) >> 40) * (1.0 / (1 << 24)))


# --------------------------------------------------------------------------
# bfloat16 rounding
# --------------------------------------------------------------------------
def bf16(x):
    """Round to bfloat16 (nearest, ties to even) through float32; returns float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    b = a.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64).reshape(a.shape)


# --------------------------------------------------------------------------
# Network description
# --------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class UNetSpec:
    base: int = 32
    levels: int = 4
    in_ch: int = 1
    out_ch: int = 1
    slope: float = 0.2

    def channels(self, level: int) -> int:
        return self.base << level


def param_specs(spec: UNetSpec):
    """[(name, kind, cin, cout)] in storage order; kind in {'c3', 'ct', 'c1'}."""
    out = [("inc.0", "c3", spec.in_ch, spec.base), ("inc.1", "c3", spec.base, spec.base)]
    for l in range(1, spec.levels + 1):
        ci, co = spec.channels(l - 1), spec.channels(l)
        out += [(f"down{l}.0", "c3", ci, co), (f"down{l}.1", "c3", co, co)]
    for l in range(1, spec.levels + 1):
        hi, lo = spec.channels(spec.levels - l + 1), spec.channels(spec.levels - l)
        out += [(f"up{l}.t", "ct", hi, lo), (f"up{l}.0", "c3", 2 * lo, lo), (f"up{l}.1", "c3", lo, lo)]
    out += [("outc", "c1", spec.base, spec.out_ch)]
    return out


def weight_shape(kind, cin, cout):
    return {"c3": (cout, 3, 3, cin), "ct": (cout, 2, 2, cin), "c1": (cout, cin)}[kind]


def fan_in(kind, cin):
    return {"c3": 9 * cin, "ct": cin, "c1": cin}[kind]


def n_params(spec: UNetSpec) -> int:
    n = 0
    for _, kind, ci, co in param_specs(spec):
        n += int(np.prod(weight_shape(kind, ci, co))) + co
    return n


def init_params(spec: UNetSpec, seed: int) -> np.ndarray:
    """Flat float32 parameters: value k of the flat vector is
    bound * (2 u_k - 1), u_k = rand_unit_f32(seed, k), bound = 1/sqrt(fan_in)
    of its tensor (weights and biases alike), computed in float32."""
    vals = np.empty(n_params(spec), dtype=np.float32)
    k = 0
    for _, kind, ci, co in param_specs(spec):
        bound = np.float32(1.0 / math.sqrt(fan_in(kind, ci)))
        cnt = int(np.prod(weight_shape(kind, ci, co))) + co
        for i in range(cnt):
            u = rand_unit_f32(seed, k + i)
            vals[k + i] = bound * (np.float32(2.0) * u - np.float32(1.0))
        k += cnt
    return vals


def unflatten(flat, spec: UNetSpec):
    """Dict name -> (W float64, b float64)."""
    flat = np.asarray(flat, dtype=np.float64)
    out, k = {}, 0
    for name, kind, ci, co in param_specs(spec):
        shp = weight_shape(kind, ci, co)
        nw = int(np.prod(shp))
        out[name] = (flat[k:k + nw].reshape(shp), flat[k + nw:k + nw + co])
        k += nw + co
    return out


def flatten(d, spec: UNetSpec) -> np.ndarray:
    parts = []
    for name, _, _, _ in param_specs(spec):
        W, b = d[name]
        parts += [np.ravel(W), np.ravel(b)]
    return np.concatenate(parts)


# --------------------------------------------------------------------------
# Layers (NCHW, float64).  Each is written from its definition.
# --------------------------------------------------------------------------
def conv3x3(x, W, b):
    """y[n,o,h,w] = b[o] + sum_{c,dh,dw} W[o,dh,dw,c] x[n,c,h+dh-1,w+dw-1] (zero padding 1)."""
    N, C, H, Wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    y = np.zeros((N, W.shape[0], H, Wd))
    for dh in range(3):
        for dw in range(3):
            y += np.tensordot(W[:, dh, dw, :], xp[:, :, dh:dh + H, dw:dw + Wd], axes=([1], [1])).transpose(1, 0, 2, 3)
    return y + b[None, :, None, None]


def conv3x3_dgrad(g, W):
    """dx[n,c,i,j] = sum_{o,dh,dw} W[o,dh,dw,c] g[n,o,i+1-dh,j+1-dw]."""
    N, O, H, Wd = g.shape
    dxp = np.zeros((N, W.shape[3], H + 2, Wd + 2))
    for dh in range(3):
        for dw in range(3):
            dxp[:, :, dh:dh + H, dw:dw + Wd] += np.tensordot(W[:, dh, dw, :], g, axes=([0], [1])).transpose(1, 0, 2, 3)
    return dxp[:, :, 1:H + 1, 1:Wd + 1]


def conv3x3_wgrad(x, g):
    """dW[o,dh,dw,c] = sum_{n,h,w} g[n,o,h,w] x[n,c,h+dh-1,w+dw-1]; db[o] = sum g."""
    N, C, H, Wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    dW = np.zeros((g.shape[1], 3, 3, C))
    for dh in range(3):
        for dw in range(3):
            dW[:, dh, dw, :] = np.tensordot(g, xp[:, :, dh:dh + H, dw:dw + Wd], axes=([0, 2, 3], [0, 2, 3]))
    return dW, g.sum(axis=(0, 2, 3))


def convT2x2(x, W, b):
    """y[n,o,2h+a,2w+c] = b[o] + sum_i W[o,a,c,i] x[n,i,h,w]."""
    N, C, H, Wd = x.shape
    y = np.zeros((N, W.shape[0], 2 * H, 2 * Wd))
    for a in range(2):
        for c in range(2):
            y[:, :, a::2, c::2] = np.tensordot(W[:, a, c, :], x, axes=([1], [1])).transpose(1, 0, 2, 3)
    return y + b[None, :, None, None]


def convT2x2_dgrad(g, W):
    dx = 0.0
    for a in range(2):
        for c in range(2):
            dx = dx + np.tensordot(W[:, a, c, :], g[:, :, a::2, c::2], axes=([0], [1])).transpose(1, 0, 2, 3)
    return dx


def convT2x2_wgrad(x, g):
    dW = np.zeros((g.shape[1], 2, 2, x.shape[1]))
    for a in range(2):
        for c in range(2):
            dW[:, a, c, :] = np.tensordot(g[:, :, a::2, c::2], x, axes=([0, 2, 3], [0, 2, 3]))
    return dW, g.sum(axis=(0, 2, 3))


def conv1x1(x, W, b):
    return np.tensordot(W, x, axes=([1], [1])).transpose(1, 0, 2, 3) + b[None, :, None, None]


def avgpool3s2(x):
    """y[n,c,i,j] = (1/9) sum_{a,b in 0..2} xp[n,c,2i+a,2j+b], xp = x zero-padded by 1."""
    N, C, H, Wd = x.shape
    Ho, Wo = (H - 1) // 2 + 1, (Wd - 1) // 2 + 1
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    y = np.zeros((N, C, Ho, Wo))
    for a in range(3):
        for b in range(3):
            y += xp[:, :, a:a + 2 * Ho - 1:2, b:b + 2 * Wo - 1:2]
    return y / 9.0


def avgpool3s2_bwd(g, H, Wd):
    N, C, Ho, Wo = g.shape
    dxp = np.zeros((N, C, H + 2, Wd + 2))
    for a in range(3):
        for b in range(3):
            dxp[:, :, a:a + 2 * Ho - 1:2, b:b + 2 * Wo - 1:2] += g / 9.0
    return dxp[:, :, 1:H + 1, 1:Wd + 1]


def leaky(z, slope):
    return np.where(z > 0, z, slope * z)


def leaky_grad_from_output(a, slope):
    """dA/dZ from the activation itself (sign is preserved for slope > 0)."""
    return np.where(a > 0, 1.0, slope)


# --------------------------------------------------------------------------
# Forward / backward of the whole network
# --------------------------------------------------------------------------
def forward(flat, x, spec: UNetSpec, round_bf16: bool = True):
    """Network output for input x [N,1,H,W] (H, W divisible by 2**levels).
    Returns (out, cache)."""
    rb = bf16 if round_bf16 else (lambda t: np.asarray(t, dtype=np.float64))
    P = unflatten(flat, spec)
    cache = {}
    sl = spec.slope

    def block(name, inp):
        W, b = P[name]
        xin = rb(inp)
        a = rb(leaky(conv3x3(xin, rb(W), b), sl))
        cache[name] = (xin, a)
        return a

    a = block("inc.1", block("inc.0", x))
    skips = [a]
    for l in range(1, spec.levels + 1):
        p = rb(avgpool3s2(a))
        cache[f"pool{l}"] = a.shape
        a = block(f"down{l}.1", block(f"down{l}.0", p))
        skips.append(a)
    for l in range(1, spec.levels + 1):
        W, b = P[f"up{l}.t"]
        xin = rb(a)
        u = rb(convT2x2(xin, rb(W), b))
        cache[f"up{l}.t"] = xin
        skip = skips[spec.levels - l]
        cat = np.concatenate([skip, u], axis=1)
        a = block(f"up{l}.1", block(f"up{l}.0", cat))
    W, b = P["outc"]
    xin = rb(a)
    out = conv1x1(xin, rb(W), b)
    cache["outc"] = xin
    return out, cache


def backward(flat, cache, dout, spec: UNetSpec, round_bf16: bool = True):
    """Gradient of a scalar loss with respect to the flat parameters, given
    dL/dout.  Returns the flat gradient (float64)."""
    rb = bf16 if round_bf16 else (lambda t: np.asarray(t, dtype=np.float64))
    P = unflatten(flat, spec)
    G = {}
    sl = spec.slope
    W, b = P["outc"]
    g = rb(dout)
    xin = cache["outc"]
    G["outc"] = (np.tensordot(g, xin, axes=([0, 2, 3], [0, 2, 3])), g.sum(axis=(0, 2, 3)))
    dA = np.tensordot(rb(W), g, axes=([0], [1])).transpose(1, 0, 2, 3)

    def block_bwd(name, dA):
        W, _ = P[name]
        xin, a = cache[name]
        gz = rb(dA * leaky_grad_from_output(a, sl))
        G[name] = conv3x3_wgrad(xin, gz)
        return conv3x3_dgrad(gz, rb(W))

    dskip = {}
    for l in range(spec.levels, 0, -1):
        dA = block_bwd(f"up{l}.0", block_bwd(f"up{l}.1", dA))
        cs = spec.channels(spec.levels - l)
        dskip[spec.levels - l] = dA[:, :cs]
        gu = rb(dA[:, cs:])
        W, _ = P[f"up{l}.t"]
        G[f"up{l}.t"] = convT2x2_wgrad(cache[f"up{l}.t"], gu)
        dA = convT2x2_dgrad(gu, rb(W))
    # dA is now the gradient of the bottom activation a_L (not a skip).
    for l in range(spec.levels, 0, -1):
        if l < spec.levels:
            dA = dA + dskip[l]
        dP = block_bwd(f"down{l}.0", block_bwd(f"down{l}.1", dA))
        H, Wd = cache[f"pool{l}"][2:]
        dA = avgpool3s2_bwd(dP, H, Wd)
    dA = dA + dskip[0]
    block_bwd("inc.0", block_bwd("inc.1", dA))
    return flatten(G, spec)


def mse(out, y):
    """L = mean((out - y)^2) and dL/dout."""
    r = out - y
    return float(np.mean(r * r)), 2.0 * r / r.size


# --------------------------------------------------------------------------
# Optimiser and schedule
# --------------------------------------------------------------------------
def cosine_lr(lr0: float, t: int, T: int) -> float:
    """Cosine annealing to zero over T steps: lr0 (1 + cos(pi t / T)) / 2."""
    return 0.5 * lr0 * (1.0 + math.cos(math.pi * t / T))


def adam_step(theta, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t is the 1-based step count); returns (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1**t)
    vh = v / (1 - b2**t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


# --------------------------------------------------------------------------
# Training data and loop
# --------------------------------------------------------------------------
def patch_origins(n: int, p: int, stride: int):
    """Edge-aligned origins 0, stride, ... plus n - p so the last patch touches the edge."""
    if n < p:
        raise ValueError("image smaller than the patch")
    o = list(range(0, n - p + 1, stride))
    if o[-1] != n - p:
        o.append(n - p)
    return o


def extract_patches(img, p: int, stride: int):
    zs, xs = patch_origins(img.shape[0], p, stride), patch_origins(img.shape[1], p, stride)
    return np.stack([img[z:z + p, x:x + p] for z in zs for x in xs])


def permutation(n: int, seed: int, epoch: int):
    """Fisher-Yates with j = rand_u64(seed ^ epoch_key, i) mod (i + 1), i = n-1 .. 1."""
    key = (seed ^ ((epoch + 1) * 0xD1B54A32D192ED03)) & MASK64
    perm = list(range(n))
    for i in range(n - 1, 0, -1):
        j = rand_u64(key, i) % (i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    return perm


def normalize(img, mute_rows: int = 0):
    """img / max|img| with the first mute_rows rows taken as 0 (and left out of the max)."""
    a = np.array(img, dtype=np.float64)
    a[:mute_rows] = 0.0
    m = float(np.max(np.abs(a)))
    return (a / m if m > 0 else a), m


@dataclasses.dataclass
class TrainCfg:
    # patch 0: full-image training (the paper's choice, Section 2.4): the
    # whole image, zero-padded at the bottom and right to a multiple of
    # 2**levels, is the one sample of every step (batch 1, epochs = steps).
    patch: int = 128
    stride: int = 64
    batch: int = 32
    epochs: int = 200
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    seed: int = 29
    mute_rows: int = 0
    warmup_frac: float = 0.0


def train(flat, x_img, y_img, spec: UNetSpec, cfg: TrainCfg, round_bf16: bool = True):
    """Train from `flat` on (x_img -> y_img), each normalised by its max |.|,
    with fresh Adam moments.  The learning rate at step t of T is the cosine
    value times min(1, (t+1)/W), W = ceil(warmup_frac T).  Returns (flat
    float64, per-epoch mean batch loss list)."""
    xn, _ = normalize(x_img, cfg.mute_rows)
    yn, _ = normalize(y_img, cfg.mute_rows)
    if cfg.patch == 0:
        X, Y = pad_to_levels(xn, spec)[None, None], pad_to_levels(yn, spec)[None, None]
    else:
        X = extract_patches(xn, cfg.patch, cfg.stride)[:, None]
        Y = extract_patches(yn, cfg.patch, cfg.stride)[:, None]
    n = X.shape[0]
    nb = -(-n // cfg.batch)
    T = cfg.epochs * nb
    theta = np.asarray(flat, dtype=np.float64).copy()
    m, v = np.zeros_like(theta), np.zeros_like(theta)
    W = math.ceil(cfg.warmup_frac * T)
    hist, t = [], 0
    for e in range(cfg.epochs):
        perm = permutation(n, cfg.seed, e)
        tot = 0.0
        for k in range(nb):
            idx = perm[k * cfg.batch:(k + 1) * cfg.batch]
            out, cache = forward(theta, X[idx], spec, round_bf16)
            loss, dout = mse(out, Y[idx])
            g = backward(theta, cache, dout, spec, round_bf16)
            lr = cosine_lr(cfg.lr, t, T) * (min(1.0, (t + 1) / W) if W > 0 else 1.0)
            theta, m, v = adam_step(theta, g, m, v, t + 1, lr, cfg.beta1, cfg.beta2, cfg.eps)
            t += 1
            tot += loss * len(idx)
        hist.append(tot / n)
    return theta, hist


def pad_to_levels(img, spec: UNetSpec):
    """img zero-padded at the bottom and right to multiples of 2**levels."""
    H, W = img.shape
    mult = 1 << spec.levels
    out = np.zeros((-(-H // mult) * mult, -(-W // mult) * mult))
    out[:H, :W] = img
    return out


def apply(flat, img, spec: UNetSpec, round_bf16: bool = True, mute_rows: int = 0):
    """net(img / max|img|) * max|img| on the full image (first mute_rows rows
    taken as 0), zero-padded at the bottom/right to a multiple of 2**levels and
    cropped back."""
    xn, m = normalize(img, mute_rows)
    H, W = xn.shape
    out, _ = forward(flat, pad_to_levels(xn, spec)[None, None], spec, round_bf16)
    return out[0, 0, :H, :W] * m
