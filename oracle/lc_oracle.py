"""Plain FP64 CPU reference of the learned-correction network (not in the paper).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Same definitions as the
CUDA network, written out with numpy: inputs (rho-1, u^theta, u^phi, T-1)
divided by in_scale and clamped to [-8, 8], plus cos(theta) and sin(theta) of the row;
3x3 convolutions 6 -> 32 -> 32 -> 32 -> 3 with ReLU between; padding periodic in phi
and, beyond a pole, the row on the opposite meridian (column + W/2) with the
input's velocity channels and sin(theta) negated (the pole boundary
condition of arXiv 2504.15574 Sec. 3.6 applied to moments); loss = the
sin(theta)-area-weighted mean over cells and the 3 channels of
(y - target / out_scale)^2.  Parameters are one flat FP32/FP64 vector, per layer
W[co][ci][3][3] then b[co].
"""
from __future__ import annotations

import math

import numpy as np

LAYERS = [(6, 32), (32, 32), (32, 32), (32, 3)]
NEG = [1, 2, 5]   # input channels odd across a pole: u^theta, u^phi, sin(theta)


def unflatten(p):
    out, o = [], 0
    for ci, co in LAYERS:
        w = p[o:o + co * ci * 9].reshape(co, ci, 3, 3)
        o += co * ci * 9
        b = p[o:o + co]
        o += co
        out.append((w, b))
    return out


def num_params():
    return sum(co * ci * 9 + co for ci, co in LAYERS)


def pad(x, neg):
    """x [C][H][W] -> [C][H+2][W+2]; neg: channels negated across a pole."""
    C, H, W = x.shape
    xp = np.zeros((C, H + 2, W + 2))
    xp[:, 1:-1, 1:-1] = x
    xp[:, 1:-1, 0] = x[:, :, -1]
    xp[:, 1:-1, -1] = x[:, :, 0]
    sign = np.ones(C)
    for c in neg:
        sign[c] = -1.0
    for xpc in range(W + 2):
        src = (xpc - 1 + W // 2) % W
        xp[:, 0, xpc] = sign * x[:, 0, src]
        xp[:, -1, xpc] = sign * x[:, -1, src]
    return xp


def unpad(g, neg):
    """Adjoint of pad(): g [C][H+2][W+2] -> [C][H][W]."""
    C, Hp, Wp = g.shape
    H, W = Hp - 2, Wp - 2
    x = g[:, 1:-1, 1:-1].copy()
    x[:, :, -1] += g[:, 1:-1, 0]
    x[:, :, 0] += g[:, 1:-1, -1]
    sign = np.ones(C)
    for c in neg:
        sign[c] = -1.0
    for xpc in range(W + 2):
        src = (xpc - 1 + W // 2) % W
        x[:, 0, src] += sign * g[:, 0, xpc]
        x[:, -1, src] += sign * g[:, -1, xpc]
    return x


def conv_valid(xp, w, b):
    """y[co][i][j] = b[co] + sum_{ci,dy,dx} w[co][ci][dy][dx] xp[ci][i+dy][j+dx]."""
    C, Hp, Wp = xp.shape
    H, W = Hp - 2, Wp - 2
    y = np.zeros((w.shape[0], H, W)) + b[:, None, None]
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("oc,chw->ohw", w[:, :, dy, dx], xp[:, dy:dy + H, dx:dx + W])
    return y


CLAMP = 8.0


def features(inputs, in_scale):
    """Scaled moments clamped to [-CLAMP, CLAMP], then cos(theta) and sin(theta) of the cell row."""
    rho, ut, up, T = inputs
    x = np.stack([(rho - 1.0) / in_scale[0], ut / in_scale[1], up / in_scale[2], (T - 1.0) / in_scale[3]])
    H, W = rho.shape
    th = (np.arange(H) + 0.5) * math.pi / H
    lat = np.stack([np.cos(th)[:, None] * np.ones((1, W)), np.sin(th)[:, None] * np.ones((1, W))])
    return np.concatenate([np.clip(x, -CLAMP, CLAMP), lat])


def area_weights(H, W):
    th = (np.arange(H) + 0.5) * math.pi / H
    s = np.sin(th)
    w = np.repeat(s[:, None], W, axis=1)
    return w / w.sum()


def forward(params, inputs, in_scale):
    """Returns the net output [3][H][W] (scaled units) and the per-layer tensors."""
    x = features(inputs, in_scale)
    cache = []
    for l, (w, b) in enumerate(unflatten(params)):
        xp = pad(x, NEG if l == 0 else [])
        y = conv_valid(xp, w, b)
        cache.append((xp, y))
        x = np.maximum(y, 0.0) if l < len(LAYERS) - 1 else y
    return x, cache


def loss_and_grad(params, inputs, targets, in_scale, out_scale):
    """Loss and d loss / d params by explicit backpropagation."""
    y, cache = forward(params, inputs, in_scale)
    H, W = y.shape[1:]
    aw = area_weights(H, W)
    t = np.stack([targets[c] / out_scale[c] for c in range(3)])
    r = y - t
    loss = float((aw[None] * r * r).sum() / 3.0)
    g = 2.0 * aw[None] * r / 3.0
    grads = []
    layers = unflatten(params)
    for l in range(len(LAYERS) - 1, -1, -1):
        w, b = layers[l]
        xp, ypre = cache[l]
        if l < len(LAYERS) - 1:
            g = g * (ypre > 0.0)
        gw = np.zeros_like(w)
        for dy in range(3):
            for dx in range(3):
                gw[:, :, dy, dx] = np.einsum("ohw,chw->oc", g, xp[:, dy:dy + H, dx:dx + W])
        gb = g.sum(axis=(1, 2))
        grads.append((gw, gb))
        if l == 0:
            break
        gxp = np.zeros_like(xp)
        for dy in range(3):
            for dx in range(3):
                gxp[:, dy:dy + H, dx:dx + W] += np.einsum("oc,ohw->chw", w[:, :, dy, dx], g)
        g = unpad(gxp, [])
    grads = grads[::-1]
    flat = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    return loss, flat


def init_params(seed):
    """Reproduces the library's initial weights (splitmix64, He-uniform, last layer x0.1)."""
    mask = (1 << 64) - 1
    s = seed & mask
    out = []
    for l, (ci, co) in enumerate(LAYERS):
        a = (0.1 if l == len(LAYERS) - 1 else 1.0) * math.sqrt(6.0 / (9.0 * ci))
        w = np.empty(co * ci * 9)
        for q in range(w.size):
            s = (s + 0x9E3779B97F4A7C15) & mask
            z = s
            z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
            z ^= z >> 31
            w[q] = a * (2.0 * ((z >> 11) * (1.0 / 9007199254740992.0)) - 1.0)
        out.append(w.astype(np.float32).astype(np.float64))
        out.append(np.zeros(co))
    return np.concatenate(out)
