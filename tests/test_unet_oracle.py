"""Pins of the FP64 U-Net oracle: the convolution against scipy's correlation, every
backward pass against central finite differences of the forward pass, pooling and
upsampling against hand-worked examples."""
import math

import numpy as np
import pytest
from scipy import signal

from oracle import unet_oracle as U


def test_conv3x3_matches_scipy_correlation():
    rng = np.random.Generator(np.random.PCG64(1))
    x = rng.standard_normal((3, 7, 9))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = U.conv3x3(x, W, b)
    for o in range(4):
        want = b[o] + sum(signal.correlate2d(x[c], W[o, c], mode="same", boundary="fill")
                          for c in range(3))
        assert np.allclose(y[o], want, rtol=0, atol=1e-12)


def test_conv3x3_backward_finite_differences():
    rng = np.random.Generator(np.random.PCG64(2))
    x = rng.standard_normal((2, 5, 6))
    W = rng.standard_normal((3, 2, 3, 3))
    b = rng.standard_normal(3)
    dy = rng.standard_normal((3, 5, 6))
    dx, dW, db = U.conv3x3_backward(x, W, dy)

    def L(x_, W_, b_):
        return float(np.sum(U.conv3x3(x_, W_, b_) * dy))
    h = 1e-6
    for idx in [(0, 0, 0), (1, 4, 5), (0, 2, 3)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        assert dx[idx] == pytest.approx((L(xp, W, b) - L(xm, W, b)) / (2 * h), rel=1e-7, abs=1e-8)
    for idx in [(0, 0, 0, 0), (2, 1, 2, 1), (1, 0, 1, 2)]:
        Wp, Wm = W.copy(), W.copy()
        Wp[idx] += h
        Wm[idx] -= h
        assert dW[idx] == pytest.approx((L(x, Wp, b) - L(x, Wm, b)) / (2 * h), rel=1e-7, abs=1e-8)
    assert np.allclose(db, dy.sum(axis=(1, 2)))


def test_pool_and_upsample_hand_examples():
    x = np.array([[[1.0, 5.0, 2.0, 2.0], [3.0, 4.0, 9.0, 1.0]]])
    assert np.array_equal(U.maxpool2(x), [[[5.0, 9.0]]])
    dx = U.maxpool2_backward(x, np.array([[[10.0, 20.0]]]))
    assert np.array_equal(dx, [[[0, 10.0, 0, 0], [0, 0, 20.0, 0]]])
    t = np.array([[[1.0, 1.0], [1.0, 1.0]]])                 # ties go to the first element
    assert np.array_equal(U.maxpool2_backward(t, np.array([[[7.0]]])), [[[7.0, 0], [0, 0]]])
    assert np.array_equal(U.upsample2(np.array([[[1.0, 2.0]]])), [[[1, 1, 2, 2], [1, 1, 2, 2]]])
    assert np.array_equal(U.upsample2_backward(np.ones((1, 2, 4))), [[[4.0, 4.0]]])


def test_network_gradients_finite_differences():
    params = U.init_params(3)
    rng = np.random.Generator(np.random.PCG64(4))
    x = rng.uniform(0, 1, (2, 8, 8))
    f_t = rng.uniform(0, 1, (8, 8))
    w_t = rng.uniform(0, 1, (8, 8))
    loss, grads = U.loss_and_grads(params, x, f_t, w_t)
    h = 1e-6
    checks = [(0, 0, (3, 0, 1, 1)), (1, 0, (5, 2, 0, 2)), (4, 0, (7, 11, 2, 2)), (6, 0, (1, 70, 1, 0)),
              (8, 0, (2, 40, 2, 1)), (9, 1, (3,)), (10, 0, (1, 5)), (10, 1, (0,)), (2, 1, (4,))]
    for layer, which, idx in checks:
        pp = [[a.copy() for a in l] for l in params]
        pm = [[a.copy() for a in l] for l in params]
        pp[layer][which][idx] += h
        pm[layer][which][idx] -= h
        lp, _ = U.loss_and_grads(pp, x, f_t, w_t)
        lm, _ = U.loss_and_grads(pm, x, f_t, w_t)
        fd = (lp - lm) / (2 * h)
        assert grads[layer][which][idx] == pytest.approx(fd, rel=1e-5, abs=1e-9), (layer, which, idx)


def test_forward_head_hand_example():
    """All 3x3 weights zero: every convolution outputs its bias, so the last decoder layer
    is the constant relu(b9) per channel and the head is o_k = hb_k + sum_c hW[k, c] relu(b9_c).
    Chosen so that o0 = 0.3 and o1 = ln 3: f0 = 0.3 and w = sigmoid(ln 3) = 3/4 at every
    pixel; a negative bias channel is cut by the ReLU.  The loss is then a hand-computed
    mean of squares, and the served warm start max(base + 0.02 o0, 0) is clamped where the
    base is below -0.006."""
    params = U.init_params(0)
    for k in range(10):
        params[k][0] = np.zeros_like(params[k][0])
        params[k][1] = np.full_like(params[k][1], 0.5)
    params[9][1] = np.zeros(16)
    params[9][1][:3] = [1.0, 2.0, -4.0]                  # relu -> 1, 2, 0
    hW = np.zeros((2, 16))
    hW[0, :3] = [0.1, 0.05, 7.0]                         # o0 = 0.1 + 0.1 + 0 + hb0
    hW[1, :3] = [0.5, 0.0, 9.0]                          # o1 = 0.5 + 0 + hb1
    params[10] = [hW, np.array([0.1, math.log(3.0) - 0.5])]
    rng = np.random.Generator(np.random.PCG64(7))
    x = rng.uniform(0, 1, (2, 8, 8))
    f0, w, cache = U.forward(params, x)
    assert np.allclose(f0, 0.3, rtol=0, atol=1e-15)
    assert np.allclose(w, 0.75, rtol=0, atol=1e-15)
    f_t = np.full((8, 8), 0.1)
    f_t[0, :] = 0.5
    w_t = np.full((8, 8), 0.25)
    loss, _ = U.loss_and_grads(params, x, f_t, w_t)
    want = (56 * 0.2 ** 2 + 8 * 0.2 ** 2) / 64 + 0.5 ** 2
    assert loss == pytest.approx(want, rel=1e-14)
    params[10][1][1] = -math.log(3.0) - 0.5              # o1 = -ln 3 -> w = 1/4
    _, w2, _ = U.forward(params, x)
    assert np.allclose(w2, 0.25, rtol=0, atol=1e-15)
    base = np.array([[0.01, -0.006, -0.01], [0.0, 0.02, -0.0061]])
    got = U.warm_start(np.full(base.shape, 0.3), base, 0.02)
    assert np.allclose(got, [[0.016, 0.0, 0.0], [0.006, 0.026, 0.0]], rtol=0, atol=1e-15)
