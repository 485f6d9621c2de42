"""Brute force: an independent, slow transcription of one SSP-RK3 step of the
vLBM (arXiv 2504.15574 Sec. 3) in 30-digit arithmetic (mpmath), on grids small
enough to exercise every ghost path (both poles, the phi seam, N_phi = 1),
compared with the FP64 oracle.

The transcription builds explicit ghost-extended arrays (rows -3..N_theta+2 and
columns -3..N_phi+2) from Eqs. (bcs_phi) and (bcs_theta) instead of mapping
indices per access, so that an index slip in either implementation shows up.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2504_15574_gb300 import inputs

mp = pytest.importorskip("mpmath")


def _tables():
    mp.mp.dps = 30
    s6 = mp.sqrt(6)
    v = [-mp.sqrt(3 + s6), -mp.sqrt(3 - s6), mp.sqrt(3 - s6), mp.sqrt(3 + s6)]
    He = [lambda x: mp.mpf(1), lambda x: x, lambda x: x**2 - 1, lambda x: x**3 - 3 * x,
          lambda x: x**4 - 6 * x**2 + 3, lambda x: x**5 - 10 * x**3 + 15 * x]
    w = [mp.mpf(24) / He[5](x) ** 2 for x in v]
    K = [[-w[k] * mp.fsum(He[l + 1](v[k]) * He[l](v[kp]) / mp.factorial(l) for l in range(4))
          for kp in range(4)] for k in range(4)]
    Kt = [[-w[k] * mp.fsum(He[l + 1](v[k]) * (He[l + 1](v[kp]) + (l * He[l - 1](v[kp]) if l else 0))
                            / mp.factorial(l) for l in range(4)) for kp in range(4)] for k in range(4)]
    return v, w, K, Kt


def _weno(a, b, c, d, e, eps):
    p = [(2 * a - 7 * b + 11 * c) / 6, (-b + 5 * c + 2 * d) / 6, (2 * c + 5 * d - e) / 6]
    s = [mp.mpf(13) / 12 * (a - 2 * b + c) ** 2 + (a - 4 * b + 3 * c) ** 2 / 4,
         mp.mpf(13) / 12 * (b - 2 * c + d) ** 2 + (b - d) ** 2 / 4,
         mp.mpf(13) / 12 * (c - 2 * d + e) ** 2 + (3 * c - 4 * d + e) ** 2 / 4]
    wt = [mp.mpf(dl) / 10 / (si + eps) ** 2 for dl, si in zip((1, 6, 3), s)]
    return mp.fsum(wi * pi for wi, pi in zip(wt, p)) / mp.fsum(wt)


def _L(f, nt, np_, tau, eps, T):
    v, w, K, Kt = T
    R = mp.mpf(1)
    dth = mp.pi / nt
    dph = 2 * mp.pi / np_
    # sin/cos at cell centres: north half computed, mirrored (reading R19)
    sn = [None] * nt
    cs = [None] * nt
    for i in range(nt):
        m = nt - 1 - i
        if i <= m:
            sn[i] = mp.sin((i + mp.mpf(1) / 2) * dth)
            cs[i] = mp.mpf(0) if i == m else mp.cos((i + mp.mpf(1) / 2) * dth)
        else:
            sn[i] = sn[m]
            cs[i] = -cs[m]
    out = [[[None] * np_ for _ in range(nt)] for _ in range(16)]
    for k in range(16):
        a, b = divmod(k, 4)
        kbar = 4 * (3 - a) + (3 - b)
        # theta-extended nodal g = sin(theta) f, rows -3 .. nt+2 stored at offset 3
        G = [[None] * np_ for _ in range(nt + 6)]
        for r in range(-3, nt + 3):
            for j in range(np_):
                if 0 <= r < nt:
                    G[r + 3][j] = sn[r] * f[k][r][j]
                else:
                    jj = (j + np_ // 2) % np_
                    rr = -1 - r if r < 0 else 2 * nt - 1 - r
                    G[r + 3][j] = -sn[rr] * f[kbar][rr][jj]
        # phi-extended f, columns -3 .. np+2 at offset 3
        Fx = [[f[k][i][(c - 3) % np_] for c in range(np_ + 6)] for i in range(nt)]
        for i in range(nt):
            for j in range(np_):
                def th_flux(iface):  # interface between rows iface-1 and iface
                    x = [G[iface + o + 3][j] for o in (-3, -2, -1, 0, 1, 2)]
                    if v[a] > 0:
                        return v[a] * _weno(x[0], x[1], x[2], x[3], x[4], eps)
                    return v[a] * _weno(x[5], x[4], x[3], x[2], x[1], eps)

                def ph_flux(iface):
                    x = [Fx[i][iface + o + 3] for o in (-3, -2, -1, 0, 1, 2)]
                    if v[b] > 0:
                        return v[b] * _weno(x[0], x[1], x[2], x[3], x[4], eps)
                    return v[b] * _weno(x[5], x[4], x[3], x[2], x[1], eps)

                adv = -(th_flux(i + 1) - th_flux(i)) / (R * sn[i] * dth) \
                    - (ph_flux(j + 1) - ph_flux(j)) / (R * sn[i] * dph)
                cell = [f[kk][i][j] for kk in range(16)]
                n = mp.fsum(cell)
                ut = mp.fsum(cell[kk] * v[kk // 4] for kk in range(16)) / n
                up = mp.fsum(cell[kk] * v[kk % 4] for kk in range(16)) / n
                xi = v[a] * ut + v[b] * up
                u2 = ut * ut + up * up
                feq = n * w[a] * w[b] * (1 + xi + (xi * xi - u2) / 2 + xi * (xi * xi - 3 * u2) / 6)
                dfdv = mp.fsum(K[a][m] * cell[4 * m + b] for m in range(4))
                dfvdv = mp.fsum(Kt[b][m] * cell[4 * a + m] for m in range(4))
                force = cs[i] / (R * sn[i]) * (v[b] ** 2 * dfdv - v[a] * dfvdv)
                out[k][i][j] = adv - force - (f[k][i][j] - feq) / tau
    return out


def _rk3(f0, nt, np_, tau, dt, eps):
    T = _tables()
    tau, dt, eps = mp.mpf(tau), mp.mpf(dt), mp.mpf(eps)
    comb = lambda A, B, ca, cb: [[[ca * A[k][i][j] + cb * B[k][i][j] for j in range(np_)]
                                  for i in range(nt)] for k in range(16)]
    L0 = _L(f0, nt, np_, tau, eps, T)
    f1 = comb(f0, L0, 1, dt)
    L1 = _L(f1, nt, np_, tau, eps, T)
    f2 = comb(comb(f0, f1, mp.mpf(3) / 4, mp.mpf(1) / 4), L1, 1, dt / 4)
    L2 = _L(f2, nt, np_, tau, eps, T)
    return comb(comb(f0, f2, mp.mpf(1) / 3, mp.mpf(2) / 3), L2, 1, 2 * dt / 3)


def _state(nt, np_, seed, amp):
    rho, ut, up, _ = inputs.gaussian_vortices(nt, np_, run=seed, umax=0.2)
    o = oracle.Oracle(nt, np_, tau=0.05, dt=1e-3)
    o.init_moments(rho, ut, up)
    f = o.get_populations()
    return f * (1.0 + amp * inputs.SplitMix64(seed).normal_array(f.shape))


@pytest.mark.parametrize("nt,np_,amp,eps", [(6, 4, 0.02, 1e-6), (7, 2, 0.3, 1e-6), (6, 1, 0.05, 1e-6),
                                            (8, 6, 0.5, 1e-3)])
def test_one_step_matches_30_digit_transcription(nt, np_, amp, eps):
    tau, dt = 0.05, 2e-3
    f = _state(nt, np_, seed=nt * 10 + np_, amp=amp)
    o = oracle.Oracle(nt, np_, tau=tau, dt=dt, eps=eps)
    o.set_populations(f)
    o.step(1)
    got = o.get_populations()
    fm = [[[mp.mpf(float(f[k, i, j])) for j in range(np_)] for i in range(nt)] for k in range(16)]
    ref = _rk3(fm, nt, np_, tau, dt, eps)
    ref = np.array([[[float(ref[k][i][j]) for j in range(np_)] for i in range(nt)] for k in range(16)])
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < 1e-13, err
