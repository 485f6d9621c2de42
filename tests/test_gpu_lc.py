"""The learned-correction network on the GPU (BF16 tensor-core kernels, FP32
accumulation) against the FP64 CPU reference: forward outputs, loss and every
parameter gradient; phi-rotation equivariance; a training step lowers the loss;
applying the correction keeps the solver's mass."""
import numpy as np
import pytest

from oracle import lc_oracle as L
from parity import require_gpu
from paper_2504_15574_gb300 import inputs

pytestmark = pytest.mark.gpu

IN_SCALE = (1e-3, 2e-2, 2e-2, 1e-2)
OUT_SCALE = (1e-4, 1e-4, 1e-4)


@pytest.fixture(scope="module")
def V():
    require_gpu()
    from paper_2504_15574_gb300 import build, vlbm
    build.build()
    vlbm.load()
    return vlbm


def _sample(H, W, seed):
    rho, ut, up, _ = inputs.gaussian_vortices(H, W, run=seed, umax=0.05)
    T = 1.0 + 0.01 * np.cos(np.arange(H))[:, None] * np.ones((1, W))
    x = np.stack([rho + 1e-3 * np.sin(np.arange(W) * 0.3)[None, :], ut, up, T])
    t = 1e-4 * np.tanh(inputs.SplitMix64(seed).normal_array((3, H, W)))
    return x, t


def _bf16(a):
    """Round to bfloat16 (nearest even), as the kernels store weights."""
    a = np.asarray(a, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("H,W", [(16, 32), (24, 64)])
def test_forward_and_gradients_match_fp64_reference(V, H, W):
    net = V.LearnedCorrection(H, W, seed=5, in_scale=IN_SCALE, out_scale=OUT_SCALE)
    p = net.get_weights().astype(np.float64)
    p[-3:] = [0.3, -0.2, 0.1]                       # non-zero output biases
    net.set_weights(p)
    x, t = _sample(H, W, 11)
    # the reference sees the weights the kernels see (bf16), in FP64 arithmetic
    pw = p.copy()
    o = 0
    for ci, co in L.LAYERS:
        pw[o:o + co * ci * 9] = _bf16(p[o:o + co * ci * 9])
        o += co * ci * 9 + co
    y_ref, _ = L.forward(pw, x, IN_SCALE)
    y = net.predict(x) / np.asarray(OUT_SCALE)[:, None, None]
    scale = np.abs(y_ref).max()
    assert np.abs(y - y_ref).max() <= 3e-2 * scale, np.abs(y - y_ref).max() / scale
    loss, g = net.gradients(x, t)
    loss_ref, g_ref = L.loss_and_grad(pw, x, t, IN_SCALE, OUT_SCALE)
    assert loss == pytest.approx(loss_ref, rel=3e-2)
    # per layer: weights and biases, relative to the largest entry of that block
    o = 0
    for ci, co in L.LAYERS:
        for n in (co * ci * 9, co):
            a, b = g[o:o + n], g_ref[o:o + n]
            assert np.abs(a - b).max() <= 5e-2 * np.abs(b).max(), (o, np.abs(a - b).max() / np.abs(b).max())
            o += n


def test_phi_rotation_equivariance_is_bitwise(V):
    H, W, r = 16, 32, 8
    net = V.LearnedCorrection(H, W, seed=2, in_scale=IN_SCALE, out_scale=OUT_SCALE)
    x, _ = _sample(H, W, 4)
    y0 = net.predict(x)
    y1 = net.predict(np.roll(x, r, axis=2))
    assert np.array_equal(np.roll(y0, r, axis=2), y1)


def test_training_lowers_the_loss(V):
    H, W = 16, 32
    net = V.LearnedCorrection(H, W, seed=3, in_scale=IN_SCALE, out_scale=OUT_SCALE)
    x, _ = _sample(H, W, 9)
    # a learnable target: a smooth function of the inputs
    t = np.stack([1e-4 * np.tanh((x[0] - 1.0) / 1e-3), 5e-5 * np.tanh(x[1] / 2e-2), -5e-5 * np.tanh(x[2] / 2e-2)])
    losses = [net.train_step(x, t, 3e-3) for _ in range(150)]
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])


def test_apply_keeps_mass_and_moves_the_moments(V):
    H, W = 16, 32
    net = V.LearnedCorrection(H, W, seed=4, in_scale=IN_SCALE, out_scale=OUT_SCALE)
    p = net.get_weights()
    p[-3:] = [1.0, 0.5, -0.5]
    net.set_weights(p)
    s = V.Solver(H, W, 2e-3, 1e-4, precision="fp32")
    s.init_moments(*inputs.gaussian_vortices(H, W, run=6))
    m0 = s.diagnostics()["mass"]
    r0, ut0, up0 = s.moments()
    net.apply(s)
    m1 = s.diagnostics()["mass"]
    r1, ut1, up1 = s.moments()
    assert abs(m1 - m0) < 1e-6 * m0
    assert np.abs(ut1 - ut0).max() > 1e-6 and np.abs(r1 - r0).max() > 1e-7


def test_trained_correction_beats_the_plain_coarse_run_on_held_out_seeds(V):
    """Small learned-coarse experiment (coarse 32 x 64 from fine 128 x 256): after
    training on one-step gaps, the corrected coarse rollout is closer to the
    downsampled fine run than the plain coarse rollout, in vorticity and density."""
    from paper_2504_15574_gb300 import learned
    setup = learned.Setup(coarse=(32, 64))
    X, Y = learned.make_samples(setup, list(range(1000, 1008)), 32, spinup=10)
    net, _ = learned.train(setup, X, Y, epochs=4)
    res = learned.evaluate(setup, net, [5000, 5001], 30)
    assert np.isfinite(res["vort_err_learned"])
    assert res["vort_err_learned"] < 0.8 * res["vort_err_plain"], res
    assert res["rho_err_learned"] < res["rho_err_plain"], res
