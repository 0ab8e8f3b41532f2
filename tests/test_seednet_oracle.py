"""Pins of the seed-network oracle (oracle/seednet.py), CPU only: bfloat16
rounding on known values, the input features on constructed frames (constant
frames, one pixel, known temporal vectors), the convolution against explicit
loops, the backward pass against central finite differences, the pooled Huber
loss against its closed form, and the Adam update against closed forms."""
import numpy as np
import pytest

from oracle import seednet as SN


def test_bf16_rounding_known_values():
    one = 1.0
    assert SN.bf16(one + 2.0 ** -8) == one                     # halfway, ties to even (down)
    assert SN.bf16(one + 3 * 2.0 ** -8) == one + 2.0 ** -6     # halfway, ties to even (up)
    assert SN.bf16(one + 2.0 ** -7) == one + 2.0 ** -7         # representable
    assert SN.bf16(one + 1.1 * 2.0 ** -8) == one + 2.0 ** -7   # above halfway
    assert SN.bf16(-3.0) == -3.0 and SN.bf16(0.0) == 0.0


def test_conv3x3_against_loops():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 5, 7, 3))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = SN.conv3x3(x, w, b)
    for n in range(2):
        for i in range(5):
            for j in range(7):
                for o in range(4):
                    s = b[o]
                    for dy in range(3):
                        for dx in range(3):
                            ii, jj = i + dy - 1, j + dx - 1
                            if 0 <= ii < 5 and 0 <= jj < 7:
                                s += (x[n, ii, jj] * w[o, dy, dx]).sum()
                    assert y[n, i, j, o] == pytest.approx(s, abs=1e-12)


def _loss(params, x, labels, mask):
    acts = SN.forward(x, params, round_bf16=False)
    return SN.loss_and_grad(acts[-1], labels, mask)[0]


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    params = SN.init_params(3)
    params = [(w, rng.normal(0, 0.05, b.shape)) for w, b in params]
    x = rng.normal(0, 0.5, (1, 8, 8, 16))
    labels = rng.normal(0, 3, (1, 4, 2))
    mask = np.array([[1, 1, 0, 1]], np.uint8)
    acts = SN.forward(x, params, round_bf16=False)
    _, d = SN.loss_and_grad(acts[-1], labels, mask)
    grads = SN.backward(acts, params, d, round_bf16=False)
    eps = 1e-6
    for li in (0, 2, 4):
        w, b = params[li]
        for idx in [(0, 1, 1, 0), (1, 0, 2, 3), (0, 2, 0, 5)]:
            pp = [(ww.copy(), bb.copy()) for ww, bb in params]
            pp[li][0][idx] += eps
            lp = _loss(pp, x, labels, mask)
            pp[li][0][idx] -= 2 * eps
            lm = _loss(pp, x, labels, mask)
            num = (lp - lm) / (2 * eps)
            assert grads[li][0][idx] == pytest.approx(num, rel=1e-4, abs=1e-8)
        pp = [(ww.copy(), bb.copy()) for ww, bb in params]
        pp[li][1][0] += eps
        lp = _loss(pp, x, labels, mask)
        pp[li][1][0] -= 2 * eps
        lm = _loss(pp, x, labels, mask)
        assert grads[li][1][0] == pytest.approx((lp - lm) / (2 * eps), rel=1e-4, abs=1e-8)


def test_pool_and_huber_closed_form():
    out = np.zeros((1, 8, 4, 16))
    out[:, :4, :, 0] = 0.25   # MB 0: seed dx = 8 * 0.25 = 2 px
    out[:, 4:, :, 1] = -0.05  # MB 1: seed dy = -0.4 px
    seeds = SN.pool_seeds(out)
    assert np.allclose(seeds[0], [[2.0, 0.0], [0.0, -0.4]])
    labels = np.array([[[0.0, 0.0], [0.0, 0.0]]])
    loss, d = SN.loss_and_grad(out, labels, np.array([[1, 1]]))
    # MB 0: |r| = 2 > 1 -> 2 - 0.5; MB 1: 0.5 * 0.16; mean over 2 MBs
    assert loss == pytest.approx(((2 - 0.5) + 0.5 * 0.16) / 2)
    assert d[0, 0, 0, 0] == pytest.approx(1.0 / 2 * 8 / 16)      # clipped residual 1
    assert d[0, 5, 0, 1] == pytest.approx(-0.4 / 2 * 8 / 16)
    # masked MBs count neither in the loss nor in its mean: only MB 0 remains
    loss, d = SN.loss_and_grad(out, labels, np.array([[1, 0]]))
    assert loss == pytest.approx(2 - 0.5)
    assert d[0, 0, 0, 0] == pytest.approx(1.0 * 8 / 16) and d[0, 5, 0, 1] == 0.0


# ------------------------------------------------------------- features --
def test_features_of_constant_frames():
    """Channel 0 is the current cell mean /255 - 0.5, channel 1 the reference
    one, channel 2 their difference /255; nothing else without a temporal
    field."""
    H, W = 32, 48  # 8 x 12 cells, 2 x 3 MBs
    cur = np.full((H, W), 255, np.uint8)
    ref = np.zeros((H, W), np.uint8)
    x = SN.features(ref, cur, None, 1)
    assert x.shape == (8, 12, 16)
    assert np.all(x[..., 0] == 0.5) and np.all(x[..., 1] == -0.5) and np.all(x[..., 2] == 1.0)
    assert np.all(x[..., 3:] == 0.0)
    # cells of half 127, half 128 have mean 127.5: exactly zero after the offset
    mid = np.zeros((H, W), np.uint8)
    mid[:, 0::2], mid[:, 1::2] = 127, 128
    x = SN.features(ref, mid, None, 2)
    assert np.all(x[..., 0] == 0.0) and np.all(x[..., 1] == -0.5)
    assert np.all(x[..., 2] == SN.bf16(127.5 / 255.0))


def test_features_one_pixel_lands_in_its_cell():
    """A single bright pixel of the current frame raises its own 4x4 cell's
    mean by 255/16 and no other cell; the same pixel in the reference frame
    moves channel 1 and flips the sign of channel 2."""
    H, W = 32, 48
    one = np.zeros((H, W), np.uint8)
    one[13, 22] = 255  # cell (3, 5)
    zero = np.zeros_like(one)
    x = SN.features(zero, one, None, 1)
    others = np.ones((8, 12), bool)
    others[3, 5] = False
    assert x[3, 5, 0] == 1 / 16 - 0.5 and x[3, 5, 1] == -0.5 and x[3, 5, 2] == 1 / 16
    assert np.all(x[others, 0] == -0.5) and np.all(x[others, 2] == 0.0)
    x = SN.features(one, zero, None, 1)
    assert x[3, 5, 0] == -0.5 and x[3, 5, 1] == 1 / 16 - 0.5 and x[3, 5, 2] == -1 / 16
    assert np.all(x[others, 1] == -0.5)


@pytest.mark.parametrize("subpel", [1, 2])
def test_features_temporal_vector_per_mb(subpel):
    """Channels 3, 4 carry the temporal candidate of the cell's MB in pixels
    / 16 (a vector in MV units divided by 16 * subpel), on all 16 cells of
    that MB and only there."""
    H, W = 32, 48  # MB (u, v) = cells [4v, 4v + 4) x [4u, 4u + 4)
    t = np.array([[32 * (i + 1), -16 * (i + 1)] for i in range(6)], np.int16)
    x = SN.features(np.zeros((H, W), np.uint8), np.zeros((H, W), np.uint8), t, subpel)
    for mb in range(6):
        v, u = divmod(mb, 3)
        blk = x[4 * v:4 * v + 4, 4 * u:4 * u + 4]
        assert np.all(blk[..., 3] == (i := mb + 1) * 2.0 / subpel), mb
        assert np.all(blk[..., 4] == -i / subpel), mb
    assert np.all(x[..., 5:] == 0.0)


# ------------------------------------------------------------------ Adam --
def test_adam_first_step_is_a_signed_learning_rate():
    """With fresh moments the bias-corrected first step is lr * g / (|g| + eps):
    the sign of the gradient times lr, descending."""
    g = np.array([3.0, -0.25, 1e-3, 0.0], np.float32)
    p0 = np.ones(4, np.float32)
    p, m, v = SN.adam_step(p0, g, np.zeros(4), np.zeros(4), 1, 1e-2)
    want = p0 - np.float32(1e-2) * g / (np.abs(g) + np.float32(1e-8))
    assert np.allclose(p, want, rtol=0, atol=2e-7)
    assert p[0] < 1 and p[1] > 1 and p[3] == 1.0
    assert np.allclose(m, 0.1 * g, rtol=1e-6) and np.allclose(v, 1e-3 * g * g, rtol=2e-5)  # 1 - 0.999 in float32


def test_adam_constant_gradient_and_reversal():
    """Constant gradient: the bias-corrected moments equal g and g^2 at every
    step, so each step moves by lr * sign(g).  A reversal (g then -g): the
    second step's corrected first moment is -(1 - b1) g / (1 + b1) and the
    second moment g^2, so it moves back by lr / 19."""
    lr = np.float32(1e-3)
    p, m, v = np.zeros(1, np.float32), np.zeros(1), np.zeros(1)
    for t in range(1, 6):
        p, m, v = SN.adam_step(p, np.array([2.0]), m, v, t, lr)
    assert p[0] == pytest.approx(-5 * 1e-3, rel=1e-5)
    p, m, v = SN.adam_step(np.zeros(1), np.array([2.0]), np.zeros(1), np.zeros(1), 1, lr)
    p2, _, _ = SN.adam_step(p, np.array([-2.0]), m, v, 2, lr)
    assert float(p2[0] - p[0]) == pytest.approx(1e-3 / 19, rel=1e-4)
