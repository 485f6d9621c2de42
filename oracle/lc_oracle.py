"""Plain FP64 CPU reference of the learned-correction network (not in the paper).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Same definitions as the
CUDA network, written out with numpy: inputs (rho-1, u^theta, u^phi, T-1) and
undivided 4th / 6th differences of the moments along theta and phi, divided by
in_scale and clamped to [-8, 8], plus cos(theta) and sin(theta) of the row;
3x3 convolutions 16 -> 32 -> 32 -> 32 -> 3 with ReLU between; padding (and the
differences' halo) periodic in phi and, beyond a pole, the row on the opposite
meridian (column + W/2) with velocity channels and sin(theta) negated (the pole boundary
condition of arXiv 2504.15574 Sec. 3.6 applied to moments); loss = the
sin(theta)-area-weighted mean over cells and the 3 channels of
(y - target / out_scale)^2.  Parameters are one flat FP32/FP64 vector, per layer
W[co][ci][3][3] then b[co].
"""
from __future__ import annotations

import math

import numpy as np

LAYERS = [(16, 32), (32, 32), (32, 32), (32, 3)]
# input channels odd across a pole: u^theta, u^phi, sin(theta) and the velocity differences
NEG = [1, 2, 5] + list(range(8, 16))


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


def extend(a, odd, halo=3):
    """a [H][W] -> [H+2 halo][W+2 halo]: columns wrap; a row beyond a pole is the
    mirrored row on the opposite meridian, negated for a velocity component."""
    H, W = a.shape
    sgn = -1.0 if odd else 1.0
    rows = []
    for r in range(-halo, H + halo):
        if r < 0:
            rows.append(sgn * np.roll(a[-1 - r], -(W // 2)))
        elif r >= H:
            rows.append(sgn * np.roll(a[2 * H - 1 - r], -(W // 2)))
        else:
            rows.append(a[r])
    e = np.array(rows)
    return np.concatenate([e[:, W - halo:], e, e[:, :halo]], axis=1)


D4 = [1.0, -4.0, 6.0, -4.0, 1.0]
D6 = [1.0, -6.0, 15.0, -20.0, 15.0, -6.0, 1.0]


def difference(a, odd, stencil, axis):
    """Undivided difference with the given stencil along theta (axis 0) or phi (axis 1)."""
    H, W = a.shape
    e = extend(a, odd)
    h = len(stencil) // 2
    out = np.zeros((H, W))
    for m, w in enumerate(stencil):
        o = 3 + m - h
        out += w * (e[o:o + H, 3:3 + W] if axis == 0 else e[3:3 + H, o:o + W])
    return out


def features(inputs, in_scale):
    """The 16 input channels: rho-1, u^theta, u^phi, T-1, then cos(theta), sin(theta),
    then d6_theta rho, d6_phi rho, d6_theta u^theta, d6_phi u^theta, d6_theta u^phi,
    d6_phi u^phi, d4_theta u^theta, d4_phi u^theta, d4_theta u^phi, d4_phi u^phi.  The 14
    data channels are divided by in_scale and clamped to [-CLAMP, CLAMP]."""
    rho, ut, up, T = inputs
    H, W = rho.shape
    data = [rho - 1.0, ut, up, T - 1.0,
            difference(rho, False, D6, 0), difference(rho, False, D6, 1),
            difference(ut, True, D6, 0), difference(ut, True, D6, 1),
            difference(up, True, D6, 0), difference(up, True, D6, 1),
            difference(ut, True, D4, 0), difference(ut, True, D4, 1),
            difference(up, True, D4, 0), difference(up, True, D4, 1)]
    x = np.clip(np.stack([d / s for d, s in zip(data, in_scale)]), -CLAMP, CLAMP)
    th = (np.arange(H) + 0.5) * math.pi / H
    lat = np.stack([np.cos(th)[:, None] * np.ones((1, W)), np.sin(th)[:, None] * np.ones((1, W))])
    return np.concatenate([x[:4], lat, x[4:]])


def area_weights(H, W):
    th = (np.arange(H) + 0.5) * math.pi / H
    s = np.sin(th)
    w = np.repeat(s[:, None], W, axis=1)
    return w / w.sum()


def forward(params, inputs, in_scale, quantize=None):
    """Returns the net output [3][H][W] (scaled units) and the per-layer tensors.
    quantize (optional) maps the input features to a storage precision (e.g. BF16)."""
    x = features(inputs, in_scale)
    if quantize is not None:
        x = quantize(x)
    cache = []
    for l, (w, b) in enumerate(unflatten(params)):
        xp = pad(x, NEG if l == 0 else [])
        y = conv_valid(xp, w, b)
        cache.append((xp, y))
        x = np.maximum(y, 0.0) if l < len(LAYERS) - 1 else y
    return x, cache


def loss_and_grad(params, inputs, targets, in_scale, out_scale, quantize=None):
    """Loss and d loss / d params by explicit backpropagation."""
    y, cache = forward(params, inputs, in_scale, quantize)
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
