"""3-D convolutional network of the learned warm start, FP64 numpy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper's outlook proposes generating simulated data to train machine
learning models; the warm start maps the first back-projected gradient of a
reconstruction to a starting coefficient volume.  Definitions used here
(plain, by the formulas):

  conv(x, w)[v, co] = sum_{t in {-1,0,1}^3} sum_ci x[v + t, ci] w[t, co, ci],
      zero outside the volume ("same" padding, cross-correlation),
      x: [nx, ny, nz, Cin], w: [3, 3, 3, Cout, Cin] indexed by t + 1.
  layer l: a_l = relu(conv(a_{l-1}, w_l)) for hidden layers, the last layer
      is linear.
  backward of conv for an output gradient dy:
      dx[u, ci] = sum_t sum_co dy[u - t, co] w[t, co, ci]
      dw[t, co, ci] = sum_v dy[v, co] x[v + t, ci]
"""
from __future__ import annotations

import itertools

import numpy as np

TAPS = list(itertools.product((-1, 0, 1), repeat=3))


def _shifted(x, t):
    """s[v] = x[v + t], zero where v + t leaves the volume."""
    out = np.zeros_like(x)
    src = []
    dst = []
    for d, n in zip(t, x.shape[:3]):
        if d == 1:
            src.append(slice(1, n)); dst.append(slice(0, n - 1))
        elif d == -1:
            src.append(slice(0, n - 1)); dst.append(slice(1, n))
        else:
            src.append(slice(0, n)); dst.append(slice(0, n))
    out[tuple(dst)] = x[tuple(src)]
    return out


def conv3d(x, w):
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    y = np.zeros(x.shape[:3] + (w.shape[3],))
    for t in TAPS:
        wt = w[t[0] + 1, t[1] + 1, t[2] + 1]           # [Cout, Cin]
        y += _shifted(x, t) @ wt.T
    return y


def conv3d_backward(x, w, dy):
    """(dx, dw) of y = conv3d(x, w) for the output gradient dy."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for t in TAPS:
        wt = w[t[0] + 1, t[1] + 1, t[2] + 1]
        dx += _shifted(dy, tuple(-d for d in t)) @ wt
        xs = _shifted(x, t)
        dw[t[0] + 1, t[1] + 1, t[2] + 1] = np.einsum("xyzo,xyzi->oi", dy, xs)
    return dx, dw


def _keep(a):
    return a


def network_forward(x, weights, rnd=_keep):
    """Activations [a_0 = x, a_1, ..., a_L]; ReLU on all but the last layer.
    rnd (identity by default) is applied to the input, the weights and every
    stored hidden activation: passing a rounding to bfloat16 reproduces the
    storage precision of a mixed-precision implementation, while every sum
    is still taken in FP64."""
    acts = [rnd(np.asarray(x, dtype=np.float64))]
    for l, w in enumerate(weights):
        y = conv3d(acts[-1], rnd(w))
        if l < len(weights) - 1:
            y = rnd(np.maximum(y, 0.0))
        acts.append(y)
    return acts


def network_backward(acts, weights, dout, rnd=_keep):
    """Weight gradients of a network given its activations and dL/d(output);
    rnd is applied to the weights and to every propagated gradient."""
    grads = [None] * len(weights)
    d = rnd(np.asarray(dout, dtype=np.float64))
    for l in range(len(weights) - 1, -1, -1):
        if l < len(weights) - 1:
            d = d * (acts[l + 1] > 0)
        dx, dw = conv3d_backward(acts[l], rnd(weights[l]), d)
        grads[l] = dw
        d = rnd(dx)
    return grads
