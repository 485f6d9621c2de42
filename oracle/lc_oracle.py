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

Output forms.  "direct": the three outputs are (drho, du^theta, du^phi) / out_scale.
"stream": output 0 times out_scale[0] is a stream function psi on the cell grid and
the correction is its curl, du = (d_phi psi / (R sin theta), -d_theta psi / R), in
centred differences with psi continued across a pole as a scalar (the row on the
opposite meridian); drho = 0.  The discrete velocity has zero centred divergence, so
the correction moves the vorticity without launching sound waves.  Its loss is the
sin(theta)-area-weighted mean over cells and the 2 velocity channels of
((du - target) / out_scale)^2.
"vorticity": output 0 times out_scale[0] is a vorticity correction w; psi solves the
cell-centred finite-volume Poisson equation L psi = w - (area mean of w) on the sphere
(no flux through the pole faces, whose sine is 0), and du is the curl of psi as in the
stream form (same loss).  The network stays local; the solve makes psi the integral.
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


def stream_velocity(psi, R=1.0):
    """The curl of a stream function psi [H][W] on the cell grid: (du^theta, du^phi) =
    (d_phi psi / (R sin theta), -d_theta psi / R) with centred differences; beyond a pole
    psi is the row on the opposite meridian (a scalar: no sign change)."""
    H, W = psi.shape
    dth, dph = math.pi / H, 2.0 * math.pi / W
    sin_t = np.sin((np.arange(H) + 0.5) * dth)
    e = pad(psi[None], [])[0]
    ut = (e[1:-1, 2:] - e[1:-1, :-2]) / (2.0 * R * dph * sin_t[:, None])
    up = -(e[2:, 1:-1] - e[:-2, 1:-1]) / (2.0 * R * dth)
    return ut, up


def stream_velocity_adjoint(gt, gp, R=1.0):
    """The gradient with respect to psi of sum(gt du^theta + gp du^phi), du = stream_velocity(psi)."""
    H, W = gt.shape
    dth, dph = math.pi / H, 2.0 * math.pi / W
    sin_t = np.sin((np.arange(H) + 0.5) * dth)
    ge = np.zeros((H + 2, W + 2))
    a = gt / (2.0 * R * dph * sin_t[:, None])
    ge[1:-1, 2:] += a
    ge[1:-1, :-2] -= a
    b = gp / (2.0 * R * dth)
    ge[2:, 1:-1] -= b
    ge[:-2, 1:-1] += b
    return unpad(ge[None], [])[0]


def laplacian_matrix(H, W, R=1.0):
    """The cell-centred finite-volume Laplacian on the sphere as a dense [H W][H W] matrix (cell
    (i, j) at row i W + j): (L psi)_ij = (s_{i+1/2} (psi_{i+1,j} - psi_ij) - s_{i-1/2} (psi_ij -
    psi_{i-1,j})) / (R^2 s_i dth^2) + (psi_{i,j+1} - 2 psi_ij + psi_{i,j-1}) / (R^2 s_i^2 dph^2),
    s at cell centres and at the faces theta = i dth; the pole faces have s = 0 (no flux), the
    columns wrap."""
    dth, dph = math.pi / H, 2.0 * math.pi / W
    sc = np.sin((np.arange(H) + 0.5) * dth)
    sf = np.sin(np.arange(H + 1) * dth)
    sf[0] = sf[H] = 0.0
    A = np.zeros((H * W, H * W))
    for i in range(H):
        for j in range(W):
            r = i * W + j
            kt = 1.0 / (R * R * sc[i] * dth * dth)
            kp = 1.0 / (R * R * sc[i] * sc[i] * dph * dph)
            if i > 0:
                A[r, (i - 1) * W + j] += kt * sf[i]
                A[r, r] -= kt * sf[i]
            if i < H - 1:
                A[r, (i + 1) * W + j] += kt * sf[i + 1]
                A[r, r] -= kt * sf[i + 1]
            A[r, i * W + (j + 1) % W] += kp
            A[r, i * W + (j - 1) % W] += kp
            A[r, r] -= 2.0 * kp
    return A


def area_mean_free(w):
    """w minus its sin(theta)-area-weighted mean."""
    H, W = w.shape
    sc = np.sin((np.arange(H) + 0.5) * math.pi / H)[:, None] * np.ones((1, W))
    return w - (sc * w).sum() / sc.sum()


def poisson(w, R=1.0):
    """A solution psi [H][W] of L psi = w - (area mean of w); its constant is irrelevant to the
    curl (the least-squares solution of the singular dense system)."""
    H, W = w.shape
    rhs = area_mean_free(w).ravel()
    psi = np.linalg.lstsq(laplacian_matrix(H, W, R), rhs, rcond=None)[0]
    return psi.reshape(H, W)


def vorticity_velocity(w, R=1.0):
    """du of the vorticity form: the curl of the Poisson solution of the vorticity correction w."""
    return stream_velocity(poisson(w, R), R)


def vorticity_velocity_adjoint(gt, gp, R=1.0):
    """The gradient with respect to w of sum(gt du^theta + gp du^phi), du = vorticity_velocity(w).
    With S = diag(sin theta), S L is symmetric, so the adjoint of the solve is S P S^-1 on the
    gradients the curl's adjoint leaves (which sum to zero); the mean removal's adjoint
    subtracts S times their sum over the sum of S."""
    H, W = gt.shape
    sc = np.sin((np.arange(H) + 0.5) * math.pi / H)[:, None] * np.ones((1, W))
    h = stream_velocity_adjoint(gt, gp, R)
    v = sc * poisson(h / sc, R)
    return v - sc * v.sum() / sc.sum()


def outputs(y, out_scale, form="direct", R=1.0):
    """The correction (drho, du^theta, du^phi) [3][H][W] in physical units from the net output."""
    if form == "direct":
        return np.stack([y[c] * out_scale[c] for c in range(3)])
    if form == "stream":
        ut, up = stream_velocity(y[0] * out_scale[0], R)
    else:
        ut, up = vorticity_velocity(y[0] * out_scale[0], R)
    return np.stack([np.zeros_like(ut), ut, up])


def loss_and_grad(params, inputs, targets, in_scale, out_scale, quantize=None, form="direct", R=1.0):
    """Loss and d loss / d params by explicit backpropagation."""
    y, cache = forward(params, inputs, in_scale, quantize)
    H, W = y.shape[1:]
    aw = area_weights(H, W)
    if form == "direct":
        t = np.stack([targets[c] / out_scale[c] for c in range(3)])
        r = y - t
        loss = float((aw[None] * r * r).sum() / 3.0)
        g = 2.0 * aw[None] * r / 3.0
    else:
        vel, adj = (stream_velocity, stream_velocity_adjoint) if form == "stream" else \
            (vorticity_velocity, vorticity_velocity_adjoint)
        ut, up = vel(y[0] * out_scale[0], R)
        rt = (ut - targets[1]) / out_scale[1]
        rp = (up - targets[2]) / out_scale[2]
        loss = float((aw * (rt * rt + rp * rp)).sum() / 2.0)
        g = np.zeros_like(y)
        g[0] = out_scale[0] * adj(aw * rt / out_scale[1], aw * rp / out_scale[2], R)
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
