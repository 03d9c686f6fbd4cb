"""Pins for the oracle regularisers (Section "Optimization": L2Norm and the
Huber total variation of every basis mode): closed forms on constant fields
and linear ramps, the two branches of the Huber function, and central finite
differences of the value against the written-out gradient."""
import numpy as np
import pytest

from oracle.regularizers import huber, l2_norm, tv_huber


def test_l2_norm_closed_form():
    c = np.arange(24, dtype=np.float64).reshape(2, 3, 2, 2)
    v, g = l2_norm(c)
    assert v == float(sum(k * k for k in range(24)))
    np.testing.assert_array_equal(g, 2 * c)


def test_huber_branches_and_continuity():
    d = 0.3
    assert huber(0.0, d) == 0.0
    assert abs(huber(d, d) - d / 2) < 1e-16          # both branches meet at t = delta
    assert abs(huber(1.0, d) - (1.0 - d / 2)) < 1e-16
    assert abs(huber(0.1, d) - 0.01 / (2 * d)) < 1e-16


def test_constant_field_has_zero_tv_and_gradient():
    c = np.full((4, 5, 3, 2), 1.7)
    v, g = tv_huber(c, 1e-2)
    assert v == 0.0 and not np.any(g)


@pytest.mark.parametrize("slope,delta", [(0.5, 1e-2), (1e-3, 1e-2)])
def test_linear_ramp_closed_form(slope, delta):
    # c = slope * x: |grad| = |slope| on every voxel with x < nx-1, 0 on the last slice
    nx, ny, nz = 6, 4, 3
    x = np.arange(nx, dtype=np.float64)[:, None, None, None]
    c = np.broadcast_to(slope * x, (nx, ny, nz, 1)).copy()
    v, _ = tv_huber(c, delta)
    per = (abs(slope) - delta / 2) if abs(slope) > delta else slope * slope / (2 * delta)
    assert abs(v - (nx - 1) * ny * nz * per) < 1e-12


def test_isotropic_norm_over_directions():
    # one voxel with differences (3, 4, 0) along x, y: |g| = 5
    c = np.zeros((2, 2, 1, 1))
    c[1, 0, 0, 0] = 3.0
    c[0, 1, 0, 0] = 4.0
    v, _ = tv_huber(c, 0.5)
    # voxel (0,0): g = (3, 4, 0) -> 5 - 0.25; voxel (1,0): g = (0, -3, 0) -> 3 - 0.25;
    # voxel (0,1): g = (-4, 0, 0) -> 4 - 0.25; voxel (1,1): g = 0
    assert abs(v - (4.75 + 2.75 + 3.75)) < 1e-14


@pytest.mark.parametrize("delta", [1e-2, 0.3, 5.0])
def test_tv_gradient_central_differences(delta):
    rng = np.random.default_rng(0)
    c = rng.normal(size=(4, 5, 3, 2)) * 0.2
    _, g = tv_huber(c, delta)
    h = 1e-6
    for _ in range(30):
        t = tuple(rng.integers(0, n) for n in c.shape)
        cp = c.copy(); cp[t] += h
        cm = c.copy(); cm[t] -= h
        fd = (tv_huber(cp, delta)[0] - tv_huber(cm, delta)[0]) / (2 * h)
        assert abs(fd - g[t]) < 1e-6 * max(1.0, abs(g[t])), (t, fd, g[t])
