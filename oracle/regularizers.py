"""Regularisers of the loss function (Section "Optimization"), FP64 numpy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper lists, among the Regularizer classes, the squared L2 norm of the
tensor field (L2Norm) and the Huber norm of the spatial gradient of each
basis-set mode (TotalVariation).  It gives no formulas; the readings are:

  L2(c)  = sum_{x,i} c_{x,i}^2,                   grad = 2 c
  TV(c)  = sum_{x,i} H_delta(|g_i(x)|),
           g_i(x)_d = c_i(x + e_d) - c_i(x) for x_d + 1 < N_d, else 0
           (forward differences, Neumann boundary), |.| the Euclidean norm
           over the three directions d, and the Huber function
           H_delta(t) = t^2 / (2 delta) for t <= delta, t - delta/2 otherwise.

The gradient of TV is written out from the definition:
  dTV/dc_i(y) = sum_d w_i(y - e_d) g_i(y - e_d)_d  [y_d >= 1]
                - sum_d w_i(y) g_i(y)_d,
  w = H'(t)/t = 1/delta for t <= delta, 1/t otherwise.
"""
from __future__ import annotations

import numpy as np


def l2_norm(c):
    c = np.asarray(c, dtype=np.float64)
    return float(np.sum(c * c)), 2.0 * c


def forward_differences(c):
    """g[..., d, i]: forward differences along x, y, z (zero on the last slice)."""
    c = np.asarray(c, dtype=np.float64)
    g = np.zeros(c.shape[:3] + (3,) + c.shape[3:])
    g[:-1, :, :, 0] = c[1:] - c[:-1]
    g[:, :-1, :, 1] = c[:, 1:] - c[:, :-1]
    g[:, :, :-1, 2] = c[:, :, 1:] - c[:, :, :-1]
    return g


def huber(t, delta):
    t = np.asarray(t, dtype=np.float64)
    return np.where(t <= delta, t * t / (2.0 * delta), t - 0.5 * delta)


def tv_huber(c, delta):
    """(value, gradient) of the Huber total variation of every channel."""
    c = np.asarray(c, dtype=np.float64)
    g = forward_differences(c)                      # [nx, ny, nz, 3, K]
    t = np.sqrt(np.sum(g * g, axis=3))              # [nx, ny, nz, K]
    value = float(np.sum(huber(t, delta)))
    w = np.where(t <= delta, 1.0 / delta, 1.0 / np.maximum(t, 1e-300))
    wg = w[:, :, :, None, :] * g                    # w g, per direction
    grad = -np.sum(wg, axis=3)
    grad[1:] += wg[:-1, :, :, 0]
    grad[:, 1:] += wg[:, :-1, :, 1]
    grad[:, :, 1:] += wg[:, :, :-1, 2]
    return value, grad
