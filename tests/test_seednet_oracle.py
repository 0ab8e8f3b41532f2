"""Pins of the seed-network oracle (oracle/seednet.py), CPU only: bfloat16
rounding on known values, the convolution against explicit loops, the
backward pass against central finite differences, and the pooled Huber loss
against its closed form."""
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
