"""Pins for the oracle convolution network of the warm start: the 3-D
convolution against scipy's N-d correlation (zero padding), the backward
pass against central finite differences, and a network gradient against
finite differences of the squared-error loss."""
import numpy as np
import pytest
from scipy import signal

from oracle.convnet import conv3d, conv3d_backward, network_backward, network_forward


def test_conv3d_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(5, 6, 4, 3))
    w = rng.normal(size=(3, 3, 3, 2, 3))
    y = conv3d(x, w)
    for co in range(2):
        ref = sum(signal.correlate(x[..., ci], w[..., co, ci], mode="same") for ci in range(3))
        np.testing.assert_allclose(y[..., co], ref, atol=1e-12)


def test_conv3d_identity_kernel_and_shift():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(4, 4, 4, 2))
    w = np.zeros((3, 3, 3, 2, 2))
    w[1, 1, 1] = np.eye(2)
    np.testing.assert_allclose(conv3d(x, w), x, atol=0)
    w = np.zeros((3, 3, 3, 1, 2))
    w[2, 1, 1, 0, 1] = 1.0            # y[v] = x[v + (1,0,0), channel 1]
    y = conv3d(x, w)[..., 0]
    np.testing.assert_allclose(y[:-1], x[1:, :, :, 1], atol=0)
    assert not np.any(y[-1])


def test_conv3d_backward_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(4, 3, 5, 2))
    w = rng.normal(size=(3, 3, 3, 3, 2))
    dy = rng.normal(size=(4, 3, 5, 3))
    dx, dw = conv3d_backward(x, w, dy)
    f = lambda xx, ww: float(np.sum(conv3d(xx, ww) * dy))
    h = 1e-6
    for _ in range(12):
        t = tuple(rng.integers(0, n) for n in x.shape)
        xp = x.copy(); xp[t] += h
        xm = x.copy(); xm[t] -= h
        assert abs((f(xp, w) - f(xm, w)) / (2 * h) - dx[t]) < 1e-6
        t = tuple(rng.integers(0, n) for n in w.shape)
        wp = w.copy(); wp[t] += h
        wm = w.copy(); wm[t] -= h
        assert abs((f(x, wp) - f(x, wm)) / (2 * h) - dw[t]) < 1e-6


def test_network_gradient_finite_differences():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(4, 4, 3, 2))
    target = rng.normal(size=(4, 4, 3, 2))
    ws = [rng.normal(size=(3, 3, 3, 4, 2)) * 0.3, rng.normal(size=(3, 3, 3, 4, 4)) * 0.3,
          rng.normal(size=(3, 3, 3, 2, 4)) * 0.3]
    loss = lambda ww: float(np.sum((network_forward(x, ww)[-1] - target) ** 2))
    acts = network_forward(x, ws)
    grads = network_backward(acts, ws, 2 * (acts[-1] - target))
    h = 1e-6
    for l in range(3):
        for _ in range(6):
            t = tuple(rng.integers(0, n) for n in ws[l].shape)
            wp = [w.copy() for w in ws]; wp[l][t] += h
            wm = [w.copy() for w in ws]; wm[l][t] -= h
            fd = (loss(wp) - loss(wm)) / (2 * h)
            assert abs(fd - grads[l][t]) < 1e-5 * max(1.0, abs(fd)), (l, t, fd, grads[l][t])
