"""FP64 CPU U-Net of the learned preconditioner correction (forward and backward).

TEST INFRASTRUCTURE ONLY (see ``oracle.mapmaker``): it pins the GPU training and
inference kernels.  The paper has no learned component; this network is the
correction applied after the circulant preconditioner inside flexible CG.

Architecture for widths (w_1 .. w_L), c_in input and c_out output channels:
  encoder level l:  conv3x3(c -> w_l) + ReLU, conv3x3(w_l -> w_l) + ReLU, and for
                    l < L a 2x2 average pool feeding level l + 1;
  decoder level l < L (from L - 1 down to 1): transposed conv 2x2 stride 2
                    (w_{l+1} -> w_l), concatenation [up, skip_l] (up first),
                    conv3x3(2 w_l -> w_l) + ReLU, conv3x3(w_l -> w_l) + ReLU;
  output:           conv1x1(w_1 -> c_out), no activation.
Convolutions are cross-correlations with zero padding 1.  Parameters form one flat
vector: for every layer in the order above, its weights then its biases; conv
weights are [c_out][c_in][k][k], transposed-conv weights [c_in][c_out][2][2].
Loss: L = 0.5 * mean((out - target)^2) over all elements.
"""
from __future__ import annotations

import numpy as np


def layer_specs(widths, c_in=3, c_out=3):
    """List of (kind, cin, cout) with kind in {conv3, tconv, conv1}."""
    L = len(widths)
    specs = []
    c = c_in
    for l in range(L):
        specs.append(("conv3", c, widths[l]))
        specs.append(("conv3", widths[l], widths[l]))
        c = widths[l]
    for l in range(L - 2, -1, -1):
        specs.append(("tconv", widths[l + 1], widths[l]))
        specs.append(("conv3", 2 * widths[l], widths[l]))
        specs.append(("conv3", widths[l], widths[l]))
    specs.append(("conv1", widths[0], c_out))
    return specs


def weight_shape(kind, cin, cout):
    if kind == "conv3":
        return (cout, cin, 3, 3)
    if kind == "tconv":
        return (cin, cout, 2, 2)
    return (cout, cin, 1, 1)


def param_count(widths, c_in=3, c_out=3):
    return sum(int(np.prod(weight_shape(k, ci, co))) + co for k, ci, co in layer_specs(widths, c_in, c_out))


def unpack(params, widths, c_in=3, c_out=3):
    out, o = [], 0
    for kind, ci, co in layer_specs(widths, c_in, c_out):
        shp = weight_shape(kind, ci, co)
        n = int(np.prod(shp))
        w = params[o:o + n].reshape(shp)
        o += n
        b = params[o:o + co]
        o += co
        out.append((kind, w, b))
    assert o == params.size
    return out


def init_params(widths, seed=0, c_in=3, c_out=3):
    """He-normal weights, zero biases, the output layer scaled by 1e-2."""
    g = np.random.default_rng(seed)
    parts = []
    specs = layer_specs(widths, c_in, c_out)
    for i, (kind, ci, co) in enumerate(specs):
        shp = weight_shape(kind, ci, co)
        fan_in = ci * (4 if kind == "tconv" else shp[2] * shp[3])
        w = g.standard_normal(shp) * np.sqrt(2.0 / fan_in)
        if i == len(specs) - 1:
            w *= 1e-2
        parts += [w.ravel(), np.zeros(co)]
    return np.concatenate(parts)


# ---------------------------------------------------------------- primitives

def conv3(x, w, b):
    B, C, H, W = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    y = np.zeros((B, w.shape[0], H, W))
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("oc,bcyx->boyx", w[:, :, dy, dx], xp[:, :, dy:dy + H, dx:dx + W])
    return y + b[None, :, None, None]


def conv3_back(x, w, g):
    """Gradients of conv3 w.r.t. input, weights and bias given dL/dy = g."""
    B, C, H, W = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for dy in range(3):
        for dx in range(3):
            gw[:, :, dy, dx] = np.einsum("boyx,bcyx->oc", g, xp[:, :, dy:dy + H, dx:dx + W])
            gxp[:, :, dy:dy + H, dx:dx + W] += np.einsum("oc,boyx->bcyx", w[:, :, dy, dx], g)
    return gxp[:, :, 1:-1, 1:-1], gw, g.sum(axis=(0, 2, 3))


def conv1(x, w, b):
    return np.einsum("oc,bcyx->boyx", w[:, :, 0, 0], x) + b[None, :, None, None]


def conv1_back(x, w, g):
    gx = np.einsum("oc,boyx->bcyx", w[:, :, 0, 0], g)
    gw = np.einsum("boyx,bcyx->oc", g, x)[:, :, None, None]
    return gx, gw, g.sum(axis=(0, 2, 3))


def tconv(x, w, b):
    B, C, H, W = x.shape
    y = np.zeros((B, w.shape[1], 2 * H, 2 * W))
    for dy in range(2):
        for dx in range(2):
            y[:, :, dy::2, dx::2] = np.einsum("co,bcyx->boyx", w[:, :, dy, dx], x)
    return y + b[None, :, None, None]


def tconv_back(x, w, g):
    gx = np.zeros_like(x)
    gw = np.zeros_like(w)
    for dy in range(2):
        for dx in range(2):
            gs = g[:, :, dy::2, dx::2]
            gx += np.einsum("co,boyx->bcyx", w[:, :, dy, dx], gs)
            gw[:, :, dy, dx] = np.einsum("bcyx,boyx->co", x, gs)
    return gx, gw, g.sum(axis=(0, 2, 3))


def pool(x):
    B, C, H, W = x.shape
    return x.reshape(B, C, H // 2, 2, W // 2, 2).mean(axis=(3, 5))


def pool_back(g):
    return np.repeat(np.repeat(g, 2, axis=2), 2, axis=3) * 0.25


# ---------------------------------------------------------------- network

def forward(params, x, widths, keep=False):
    """U(x) for x [B, c_in, H, W] (H, W divisible by 2^(L-1))."""
    layers = unpack(params, widths, x.shape[1])
    L = len(widths)
    cache = []
    it = iter(layers)
    skips = []
    h = x
    for l in range(L):
        for _ in range(2):
            _, w, b = next(it)
            hin = h
            h = np.maximum(conv3(hin, w, b), 0.0)
            cache.append(("conv3", hin, w, h))
        if l < L - 1:
            skips.append(h)
            h = pool(h)
            cache.append(("pool", None, None, None))
    for l in range(L - 2, -1, -1):
        _, w, b = next(it)
        hin = h
        h = tconv(hin, w, b)
        cache.append(("tconv", hin, w, None))
        h = np.concatenate([h, skips[l]], axis=1)
        cache.append(("cat", skips[l].shape[1], None, None))
        for _ in range(2):
            _, w, b = next(it)
            hin = h
            h = np.maximum(conv3(hin, w, b), 0.0)
            cache.append(("conv3", hin, w, h))
    _, w, b = next(it)
    y = conv1(h, w, b)
    cache.append(("conv1", h, w, None))
    return (y, cache) if keep else y


def loss_and_grad(params, x, target, widths):
    """L = 0.5 mean((U(x) - target)^2) and dL/dparams (same flat layout)."""
    y, cache = forward(params, x, widths, keep=True)
    diff = y - target
    loss = 0.5 * float(np.mean(diff * diff))
    g = diff / diff.size
    grads = []                       # (gw, gb) in reverse layer order
    skip_grads = []
    for kind, hin, w, hout in reversed(cache):
        if kind == "conv1":
            g, gw, gb = conv1_back(hin, w, g)
            grads.append((gw, gb))
        elif kind == "conv3":
            g = g * (hout > 0)
            g, gw, gb = conv3_back(hin, w, g)
            grads.append((gw, gb))
        elif kind == "cat":
            cs = hin
            skip_grads.append(g[:, -cs:])
            g = g[:, :-cs]
        elif kind == "tconv":
            g, gw, gb = tconv_back(hin, w, g)
            grads.append((gw, gb))
        elif kind == "pool":
            g = pool_back(g) + skip_grads.pop()
    flat = []
    for gw, gb in reversed(grads):
        flat += [gw.ravel(), gb]
    return loss, np.concatenate(flat)
