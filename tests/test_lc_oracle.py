"""Pins of the CPU reference of the learned-correction network (FP64):
the padding's adjoint, the pole reflection, and backpropagation against
central finite differences."""
import numpy as np
import pytest

from oracle import lc_oracle as L
from paper_2504_15574_gb300 import inputs


def test_unpad_is_the_adjoint_of_pad():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(5, 6, 8))
    y = rng.normal(size=(5, 8, 10))
    for neg in ([], [1, 2]):
        assert np.isclose((L.pad(x, neg) * y).sum(), (x * L.unpad(y, neg)).sum(), rtol=1e-13)


def test_pole_ghost_row_is_the_opposite_meridian_with_vectors_negated():
    x = np.arange(3 * 4 * 8, dtype=float).reshape(3, 4, 8)
    xp = L.pad(x, [1])
    # ghost of column q (padded q+1) is row 0 at column q + W/2
    for q in range(8):
        assert xp[0, 0, q + 1] == x[0, 0, (q + 4) % 8]
        assert xp[1, 0, q + 1] == -x[1, 0, (q + 4) % 8]
        assert xp[2, -1, q + 1] == x[2, -1, (q + 4) % 8]
    assert np.array_equal(xp[:, 1:-1, 0], x[:, :, -1]) and np.array_equal(xp[:, 1:-1, -1], x[:, :, 0])


def _sample(H, W, seed):
    rho, ut, up, _ = inputs.gaussian_vortices(H, W, run=seed, umax=0.05)
    T = 1.0 + 0.01 * np.cos(np.arange(H))[:, None] * np.ones((1, W))
    x = np.stack([rho + 1e-3 * np.sin(np.arange(W))[None, :], ut, up, T])
    t = 1e-4 * inputs.SplitMix64(seed).normal_array((3, H, W))
    return x, t


def test_backprop_matches_finite_differences():
    H, W = 6, 8
    x, t = _sample(H, W, 3)
    p = L.init_params(7)
    p[-3:] = [0.01, -0.02, 0.03]
    ins, outs = [1e-3, 2e-2, 2e-2, 1e-2] + [1e-3] * 10, [1e-4, 1e-4, 1e-4]
    loss, g = L.loss_and_grad(p, x, t, ins, outs)
    rng = np.random.default_rng(1)
    idx = rng.choice(p.size, 40, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        lp, _ = L.loss_and_grad(p + e, x, t, ins, outs)
        lm, _ = L.loss_and_grad(p - e, x, t, ins, outs)
        fd = (lp - lm) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9 * max(1.0, abs(loss)))


def test_parameter_count():
    assert L.num_params() == 32 * 16 * 9 + 32 + 2 * (32 * 32 * 9 + 32) + 3 * 32 * 9 + 3


def test_phi_differences_of_a_fourier_mode_are_powers_of_the_second_difference():
    # the undivided second difference of cos(k phi) on a periodic grid is (2 cos(k dphi) - 2) cos(k phi)
    H, W, k = 5, 16, 3
    phi = (np.arange(W) + 0.5) * 2 * np.pi / W
    a = np.cos(k * phi)[None, :] * np.ones((H, 1))
    lam = 2 * np.cos(k * 2 * np.pi / W) - 2
    assert np.allclose(L.difference(a, False, L.D4, 1), lam ** 2 * a, atol=1e-12)
    assert np.allclose(L.difference(a, False, L.D6, 1), lam ** 3 * a, atol=1e-12)
    # a row-independent even mode continues unchanged across a pole: no theta difference
    a2 = np.cos(2 * phi)[None, :] * np.ones((H, 1))
    assert np.allclose(L.difference(a2, False, L.D6, 0), 0.0, atol=1e-12)


def test_theta_differences_continue_smooth_fields_across_the_poles():
    # cos(theta) and the components of a uniform Cartesian flow (u_theta = cos(theta) cos(phi),
    # u_phi = -sin(phi)) continue across a pole as the same smooth functions of the row index,
    # so their theta differences are powers of the second difference on every row
    H, W = 8, 12
    th = (np.arange(H) + 0.5) * np.pi / H
    ph = (np.arange(W) + 0.5) * 2 * np.pi / W
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    lam = 2 * np.cos(np.pi / H) - 2
    z = np.cos(TH)
    assert np.allclose(L.difference(z, False, L.D6, 0), lam ** 3 * z, atol=1e-12)
    ut, up = np.cos(TH) * np.cos(PH), -np.sin(PH)
    assert np.allclose(L.difference(ut, True, L.D4, 0), lam ** 2 * ut, atol=1e-12)
    assert np.allclose(L.difference(ut, True, L.D6, 0), lam ** 3 * ut, atol=1e-12)
    assert np.allclose(L.difference(up, True, L.D6, 0), 0.0, atol=1e-12)
    # the wrong sign rule (a velocity treated as a scalar) breaks it at the pole rows
    assert not np.allclose(L.difference(ut, False, L.D6, 0), lam ** 3 * ut, atol=1e-6)


# ---- the stream-function output form -------------------------------------------------------

def _grid(H, W):
    th = (np.arange(H) + 0.5) * np.pi / H
    ph = (np.arange(W) + 0.5) * 2 * np.pi / W
    return np.meshgrid(th, ph, indexing="ij"), np.pi / H, 2 * np.pi / W


@pytest.mark.parametrize("R", [1.0, 2.5])
def test_stream_velocity_of_rotations_is_their_centred_difference_in_closed_form(R):
    # psi = cos(theta): solid rotation about the axis, du^phi = sin(theta) sin(dth)/dth / R on
    # every row (cos is even, so the pole continuation is cos itself); psi = sin(theta) cos(phi):
    # rotation about a horizontal axis, odd across a pole exactly like its opposite-meridian image
    H, W = 10, 16
    (TH, PH), dth, dph = _grid(H, W)
    ut, up = L.stream_velocity(np.cos(TH), R)
    assert np.allclose(ut, 0.0, atol=1e-14)
    assert np.allclose(up, np.sin(TH) * np.sin(dth) / dth / R, rtol=1e-12, atol=0)
    ut, up = L.stream_velocity(np.sin(TH) * np.cos(PH), R)
    assert np.allclose(ut, -np.sin(PH) * np.sin(dph) / dph / R, rtol=1e-12, atol=1e-15)
    assert np.allclose(up, -np.cos(TH) * np.cos(PH) * np.sin(dth) / dth / R, rtol=1e-12, atol=1e-15)


def test_stream_velocity_has_zero_centred_divergence_including_the_pole_rows():
    # div u = (d_theta (sin u^theta) + d_phi u^phi) / (R sin theta) in centred differences, the
    # velocity continued across a pole as a vector (opposite meridian, components negated)
    H, W, R = 8, 12, 1.7
    rng = np.random.default_rng(3)
    psi = rng.normal(size=(H, W))
    ut, up = L.stream_velocity(psi, R)
    (TH, _), dth, dph = _grid(H, W)
    st = np.sin(TH[:, 0])
    ute = L.pad(ut[None], [0])[0]
    upe = L.pad(up[None], [0])[0]
    ste = np.concatenate([[-st[0]], st, [-st[-1]]])   # sin theta at the ghost rows: negative
    flux = ste[:, None] * ute
    div = ((flux[2:, 1:-1] - flux[:-2, 1:-1]) / (2 * dth) + (upe[1:-1, 2:] - upe[1:-1, :-2]) / (2 * dph)) / (R * st[:, None])
    assert np.abs(div).max() <= 1e-12 * np.abs(ut).max()
    # a velocity that is not a curl (du^theta = cos(theta)) has a divergence there
    flux = ste[:, None] * L.pad(np.cos(TH)[None], [0])[0]
    assert np.abs((flux[2:, 1:-1] - flux[:-2, 1:-1])).max() > 0.1


def test_stream_velocity_adjoint_is_the_transpose():
    H, W, R = 7, 10, 1.3
    rng = np.random.default_rng(4)
    psi, gt, gp = rng.normal(size=(3, H, W))
    ut, up = L.stream_velocity(psi, R)
    lhs = (gt * ut + gp * up).sum()
    rhs = (psi * L.stream_velocity_adjoint(gt, gp, R)).sum()
    assert lhs == pytest.approx(rhs, rel=1e-13)


def test_stream_form_backprop_matches_finite_differences():
    H, W = 6, 8
    x, t = _sample(H, W, 5)
    p = L.init_params(9)
    p[-3:] = [0.02, 0.0, 0.0]
    ins, outs = [1e-3, 2e-2, 2e-2, 1e-2] + [1e-3] * 10, [1e-5, 1e-4, 1e-4]
    loss, g = L.loss_and_grad(p, x, t, ins, outs, form="stream", R=1.5)
    # outputs 1 and 2 do not enter the stream form: their weights get no gradient
    nw3 = 3 * 32 * 9
    w3 = g[-(nw3 + 3):-3].reshape(3, 32, 3, 3)
    assert np.all(w3[1:] == 0.0) and np.all(g[-2:] == 0.0) and np.abs(w3[0]).max() > 0
    rng = np.random.default_rng(2)
    idx = rng.choice(p.size, 40, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        lp, _ = L.loss_and_grad(p + e, x, t, ins, outs, form="stream", R=1.5)
        lm, _ = L.loss_and_grad(p - e, x, t, ins, outs, form="stream", R=1.5)
        fd = (lp - lm) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9 * max(1.0, abs(loss)))


# ---- the vorticity output form: finite-volume Poisson solve on the sphere --------------------

def _cells(H, W):
    (TH, PH), _, _ = _grid(H, W)
    return TH, PH


def test_laplacian_is_symmetric_in_the_area_weighted_product_with_constants_as_null_space():
    H, W, R = 6, 8, 1.4
    A = L.laplacian_matrix(H, W, R)
    s = np.repeat(np.sin((np.arange(H) + 0.5) * np.pi / H), W)
    SA = s[:, None] * A
    assert np.allclose(SA, SA.T, atol=1e-12 * np.abs(SA).max())
    assert np.abs(A @ np.ones(H * W)).max() <= 1e-12 * np.abs(A).max()
    assert np.linalg.matrix_rank(A) == H * W - 1


@pytest.mark.parametrize("R", [1.0, 2.0])
def test_laplacian_of_spherical_harmonics_converges_at_second_order(R):
    # Y_1^0 = cos(theta) and Y_2^1 = sin(theta) cos(theta) cos(phi) are eigenfunctions of the
    # Laplacian with -l (l + 1) / R^2; the area-weighted L2 error of the discrete operator falls
    # by ~4 per halving of the spacing
    errs = []
    for H in (16, 32, 64):
        W = 2 * H
        TH, PH = _cells(H, W)
        A = L.laplacian_matrix(H, W, R) if H <= 32 else None
        e = []
        for f, lam in ((np.cos(TH), -2.0), (np.sin(TH) * np.cos(TH) * np.cos(PH), -6.0)):
            if A is not None:
                lf = (A @ f.ravel()).reshape(H, W)
            else:   # the same stencil written out for the largest grid (a dense matrix is 67 MB)
                dth, dph = np.pi / H, 2 * np.pi / W
                sc = np.sin(TH[:, 0])
                sf = np.sin(np.arange(H + 1) * dth)
                sf[0] = sf[H] = 0.0
                fl = np.zeros((H + 1, W))
                fl[1:H] = sf[1:H, None] * (f[1:] - f[:-1])
                lf = (fl[1:] - fl[:-1]) / (R * R * sc[:, None] * dth * dth) + \
                    (np.roll(f, -1, 1) - 2 * f + np.roll(f, 1, 1)) / (R * R * sc[:, None] ** 2 * dph * dph)
            w = np.sin(TH)
            ref = lam / R ** 2 * f
            e.append(np.sqrt((w * (lf - ref) ** 2).sum() / (w * ref ** 2).sum()))
        errs.append(e)
    errs = np.array(errs)
    order = np.log2(errs[:-1] / errs[1:])
    assert np.all(order > 1.8), order
    # (a flux through the pole faces, e.g. to a ghost row across the pole, stops the convergence:
    # order ~0 with a face sine of sin(dth/4))
    assert errs[-1].max() < 2e-3


def test_poisson_solves_the_mean_free_equation_and_recovers_a_harmonic():
    H, W, R = 8, 12, 1.3
    rng = np.random.default_rng(6)
    w = rng.normal(size=(H, W))
    psi = L.poisson(w, R)
    A = L.laplacian_matrix(H, W, R)
    res = (A @ psi.ravel()).reshape(H, W) - L.area_mean_free(w)
    assert np.abs(res).max() <= 1e-10 * np.abs(w).max()
    # psi = Y_2^1 is the solution for w = L Y_2^1 (up to a constant)
    TH, PH = _cells(H, W)
    y21 = np.sin(TH) * np.cos(TH) * np.cos(PH)
    got = L.poisson((A @ y21.ravel()).reshape(H, W), R)
    d = got - y21
    assert np.abs(d - d.mean()).max() <= 1e-10


def test_vorticity_velocity_adjoint_is_the_transpose():
    H, W, R = 6, 10, 0.9
    rng = np.random.default_rng(7)
    w, gt, gp = rng.normal(size=(3, H, W))
    ut, up = L.vorticity_velocity(w, R)
    lhs = (gt * ut + gp * up).sum()
    rhs = (w * L.vorticity_velocity_adjoint(gt, gp, R)).sum()
    assert lhs == pytest.approx(rhs, rel=1e-10)
    # the adjoint of the mean removal: a vorticity that is a multiple of 1 moves nothing
    ut1, up1 = L.vorticity_velocity(np.full((H, W), 3.0), R)
    assert np.abs(ut1).max() < 1e-12 and np.abs(up1).max() < 1e-12


def test_vorticity_form_backprop_matches_finite_differences():
    H, W = 6, 8
    x, t = _sample(H, W, 6)
    p = L.init_params(11)
    p[-3:] = [0.02, 0.0, 0.0]
    ins, outs = [1e-3, 2e-2, 2e-2, 1e-2] + [1e-3] * 10, [1e-3, 1e-4, 1e-4]
    loss, g = L.loss_and_grad(p, x, t, ins, outs, form="vorticity", R=1.2)
    rng = np.random.default_rng(3)
    idx = rng.choice(p.size - 3, 30, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        lp, _ = L.loss_and_grad(p + e, x, t, ins, outs, form="vorticity", R=1.2)
        lm, _ = L.loss_and_grad(p - e, x, t, ins, outs, form="vorticity", R=1.2)
        fd = (lp - lm) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9 * max(1.0, abs(loss)))
