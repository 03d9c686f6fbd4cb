"""Pins for the oracle's residual, loss and gradient (Eq. residual; Eq.
opt_prob_general_form with a = 2 and per-datum weights).

The gradient is checked by central finite differences of the loss, the
noise-free truth gives zero loss and gradient, and zero weights zero both.
"""
import numpy as np
import pytest

import oracle
from paper_2504_16446_gb300 import synth
from conftest import oracle_geometry


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_central_differences(seed):
    st = synth.small_setup(n=(6, 7, 6), nj=8, nk=8, ell_max=2, n_proj=5, n_seg=4, seed=seed)
    g = oracle_geometry(st)
    B = oracle.basis_matrix(g)
    c = synth.random_volume(st, seed)
    I = synth.random_data(st, seed + 1)
    W = synth.random_weights(st, seed + 2)
    loss, grad = oracle.gradient_residual(g, c, I, W, B)
    rng = np.random.default_rng(seed)
    idx = [tuple(rng.integers(0, n) for n in st.volume_shape) for _ in range(25)]
    h = 1e-4
    for t in idx:
        cp = c.copy(); cp[t] += h
        cm = c.copy(); cm[t] -= h
        fd = (oracle.gradient_residual(g, cp, I, W, B, want_grad=False)[0]
              - oracle.gradient_residual(g, cm, I, W, B, want_grad=False)[0]) / (2 * h)
        # the loss is quadratic: central differences are exact up to rounding
        assert abs(fd - grad[t]) <= 1e-7 * max(1.0, np.abs(grad).max()), (t, fd, grad[t])


def test_loss_is_weighted_sum_of_squares():
    st = synth.small_setup(n=(5, 5, 5), n_proj=3, seed=4)
    g = oracle_geometry(st)
    c = synth.random_volume(st, 0)
    I = synth.random_data(st, 1)
    W = synth.random_weights(st, 2)
    r = oracle.forward(g, c) - I
    loss, grad = oracle.gradient_residual(g, c, I, W)
    assert abs(loss - np.sum(W * r * r)) < 1e-11 * loss
    np.testing.assert_allclose(grad, 2 * oracle.adjoint(g, W * r), atol=1e-12)
    loss1, _ = oracle.gradient_residual(g, c, I, None)
    assert abs(loss1 - np.sum(r * r)) < 1e-11 * loss1


def test_noise_free_truth_is_a_stationary_point():
    st = synth.small_setup(n=(6, 6, 6), ell_max=4, n_proj=4, seed=5)
    g = oracle_geometry(st)
    c = synth.random_volume(st, 3)
    I = oracle.forward(g, c)
    loss, grad = oracle.gradient_residual(g, c, I)
    assert loss < 1e-24
    assert np.abs(grad).max() < 1e-12


def test_zero_weights_zero_everything():
    st = synth.small_setup(n=(4, 4, 4), n_proj=2, seed=6)
    g = oracle_geometry(st)
    loss, grad = oracle.gradient_residual(g, synth.random_volume(st, 0), synth.random_data(st, 1),
                                          np.zeros(st.data_shape))
    assert loss == 0.0 and not np.any(grad)
