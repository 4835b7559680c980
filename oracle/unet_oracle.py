"""FP64 numpy oracle of the warm-start U-Net: forward pass and gradients.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): the GPU network in
paper_2409_01076_gb300/unet.py is checked against it; it shares no code with it.

The architecture (fixed by the warm-start specification, not by the paper,
which has no network): a 4-level U-Net with `base` channels at the top level
(32 in use; smaller values for cheap tests), 3x3 convolutions with zero padding,
SiLU activations, 2x2 average pooling, nearest 2x upsampling, skip connections
by channel concatenation, and a 1x1 output convolution to 3 channels.

    enc1: conv(cin -> b), conv(b -> b)                 (H)
    enc2: pool, conv(b -> 2b), conv(2b -> 2b)          (H/2)
    enc3: pool, conv(2b -> 4b), conv(4b -> 4b)         (H/4)
    mid : pool, conv(4b -> 8b), conv(8b -> 8b)         (H/8)
    dec3: up, concat enc3, conv(12b -> 4b), conv(4b -> 4b)
    dec2: up, concat enc2, conv(6b -> 2b), conv(2b -> 2b)
    dec1: up, concat enc1, conv(3b -> b), conv(b -> b)
    head: 1x1 conv(b -> cout), no activation

Tensors are NHWC float64.  A 3x3 weight is (cout, 9 * cin) with column index
(ky * 3 + kx) * cin + c, tap (ky, kx) reading the input at offset (ky - 1, kx - 1).
"""
from __future__ import annotations

import numpy as np


def layer_specs(base: int = 32, cin: int = 3, cout: int = 3):
    """[(name, cin, cout, kernel 3 or 1, activation)] in parameter order."""
    b = base
    return [
        ("enc1a", cin, b, 3, True), ("enc1b", b, b, 3, True),
        ("enc2a", b, 2 * b, 3, True), ("enc2b", 2 * b, 2 * b, 3, True),
        ("enc3a", 2 * b, 4 * b, 3, True), ("enc3b", 4 * b, 4 * b, 3, True),
        ("mida", 4 * b, 8 * b, 3, True), ("midb", 8 * b, 8 * b, 3, True),
        ("dec3a", 12 * b, 4 * b, 3, True), ("dec3b", 4 * b, 4 * b, 3, True),
        ("dec2a", 6 * b, 2 * b, 3, True), ("dec2b", 2 * b, 2 * b, 3, True),
        ("dec1a", 3 * b, b, 3, True), ("dec1b", b, b, 3, True),
        ("head", b, cout, 1, False),
    ]


def init_params(base: int = 32, seed: int = 0, cin: int = 3, cout: int = 3):
    """He-normal weights (std sqrt(2 / fan_in)), small random biases; seeded PCG64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    params = {}
    for name, ci, co, k, _ in layer_specs(base, cin, cout):
        fan_in = ci * k * k
        params[name + ".w"] = rng.normal(0.0, np.sqrt(2.0 / fan_in), size=(co, k * k * ci))
        params[name + ".b"] = rng.normal(0.0, 0.01, size=(co,))
    return params


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def im2col3(x):
    """(N,H,W,C) -> (N*H*W, 9*C), zero padding, column (ky*3+kx)*C + c."""
    n, h, w, c = x.shape
    xp = np.zeros((n, h + 2, w + 2, c))
    xp[:, 1:-1, 1:-1, :] = x
    cols = [xp[:, ky:ky + h, kx:kx + w, :] for ky in range(3) for kx in range(3)]
    return np.concatenate(cols, axis=3).reshape(n * h * w, 9 * c)


def col2im3(dcol, shape):
    """Adjoint of im2col3."""
    n, h, w, c = shape
    d = dcol.reshape(n, h, w, 9, c)
    dxp = np.zeros((n, h + 2, w + 2, c))
    for tap in range(9):
        ky, kx = divmod(tap, 3)
        dxp[:, ky:ky + h, kx:kx + w, :] += d[:, :, :, tap, :]
    return dxp[:, 1:-1, 1:-1, :]


def pool(x):
    n, h, w, c = x.shape
    return x.reshape(n, h // 2, 2, w // 2, 2, c).mean(axis=(2, 4))


def pool_bwd(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) / 4.0


def up(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_bwd(dy):
    n, h, w, c = dy.shape
    return dy.reshape(n, h // 2, 2, w // 2, 2, c).sum(axis=(2, 4))


def _conv(x, wgt, bias, k, act, cache):
    n, h, w_, c = x.shape
    col = im2col3(x) if k == 3 else x.reshape(n * h * w_, c)
    z = col @ wgt.T + bias
    a = silu(z) if act else z
    cache.append((col, z, x.shape, k, act))
    return a.reshape(n, h, w_, -1)


def forward(params, x, base: int = 32, cin: int = 3, cout: int = 3):
    """Returns (y, cache) for input x (N,H,W,cin), H and W divisible by 8."""
    specs = {s[0]: s for s in layer_specs(base, cin, cout)}
    cache = []

    def conv(name, inp):
        _, _, _, k, act = specs[name]
        return _conv(inp, params[name + ".w"], params[name + ".b"], k, act, cache)

    e1 = conv("enc1b", conv("enc1a", x))
    e2 = conv("enc2b", conv("enc2a", pool(e1)))
    e3 = conv("enc3b", conv("enc3a", pool(e2)))
    m = conv("midb", conv("mida", pool(e3)))
    d3 = conv("dec3b", conv("dec3a", np.concatenate([up(m), e3], axis=3)))
    d2 = conv("dec2b", conv("dec2a", np.concatenate([up(d3), e2], axis=3)))
    d1 = conv("dec1b", conv("dec1a", np.concatenate([up(d2), e1], axis=3)))
    y = conv("head", d1)
    return y, cache


def mse(y, t):
    return float(np.mean((y - t) ** 2))


def loss_and_grads(params, x, t, base: int = 32, cin: int = 3, cout: int = 3):
    """L = mean((y - t)^2) and dL/dparam for every parameter (reverse-mode, by hand)."""
    y, cache = forward(params, x, base, cin, cout)
    names = [s[0] for s in layer_specs(base, cin, cout)]
    grads = {}
    order = list(zip(names, cache))     # cache entries are in forward (= parameter) order
    idx = {nm: i for i, nm in enumerate(names)}

    def conv_bwd(name, da):
        col, z, xshape, k, act = order[idx[name]][1]
        n, h, w_, c = xshape
        dz = da.reshape(-1, z.shape[1]) * (silu_grad(z) if act else 1.0)
        grads[name + ".w"] = dz.T @ col
        grads[name + ".b"] = dz.sum(axis=0)
        dcol = dz @ params[name + ".w"]
        return col2im3(dcol, xshape) if k == 3 else dcol.reshape(xshape)

    b = base
    dy = 2.0 * (y - t) / y.size
    dd1 = conv_bwd("head", dy)
    dcat1 = conv_bwd("dec1a", conv_bwd("dec1b", dd1))
    de1 = dcat1[..., 2 * b:]
    dd2 = up_bwd(dcat1[..., :2 * b])
    dcat2 = conv_bwd("dec2a", conv_bwd("dec2b", dd2))
    de2 = dcat2[..., 4 * b:]
    dd3 = up_bwd(dcat2[..., :4 * b])
    dcat3 = conv_bwd("dec3a", conv_bwd("dec3b", dd3))
    de3 = dcat3[..., 8 * b:]
    dm = up_bwd(dcat3[..., :8 * b])
    de3 = de3 + pool_bwd(conv_bwd("mida", conv_bwd("midb", dm)))
    de2 = de2 + pool_bwd(conv_bwd("enc3a", conv_bwd("enc3b", de3)))
    de1 = de1 + pool_bwd(conv_bwd("enc2a", conv_bwd("enc2b", de2)))
    dx = conv_bwd("enc1a", conv_bwd("enc1b", de1))
    return mse(y, t), grads, dx
