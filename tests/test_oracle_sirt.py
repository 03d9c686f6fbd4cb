"""Pins for the oracle's SIRT weights and MITRA iteration (Section "Standard
reconstruction pipelines"): row and column sums of |A| against brute force on
the dense system matrix, an axis-aligned closed form, the Cauchy-Schwarz
(Schur) bound on the preconditioned operator, the classical SIRT update
written with dense matrices, and descent / acceleration on consistent data."""
import numpy as np
import pytest

import oracle
from paper_2504_16446_gb300 import synth
from conftest import oracle_geometry


def _dense(g, B):
    nv = int(np.prod(g.volume_shape))
    A = np.zeros((int(np.prod(g.data_shape)), nv))
    for col in range(nv):
        e = np.zeros(nv)
        e[col] = 1.0
        A[:, col] = oracle.forward(g, e.reshape(g.volume_shape), B).ravel()
    return A


@pytest.fixture(scope="module")
def small():
    st = synth.small_setup(n=(3, 4, 3), nj=4, nk=5, ell_max=2, n_proj=3, n_seg=3, seed=21)
    g = oracle_geometry(st)
    B = oracle.basis_matrix(g)
    return st, g, B, _dense(g, B)


def test_weights_are_inverse_abs_row_and_column_sums(small):
    st, g, B, A = small
    rho = np.abs(A).sum(axis=1)
    kappa = np.abs(A).sum(axis=0)
    R, D = oracle.sirt_weights(g, None, B)
    R, D = R.ravel(), D.ravel()
    hit = R > 0
    assert hit.sum() > 0.3 * R.size and (~hit).sum() > 0
    np.testing.assert_allclose(R[hit] * rho[hit], 1.0, rtol=1e-12)
    assert np.all(rho[~hit] < 1e-6 * g.a * np.abs(B).sum(axis=2).max())
    seen = D > 0
    assert seen.sum() > 0.5 * D.size
    np.testing.assert_allclose(D[seen] * kappa[seen], 1.0, rtol=1e-12)
    assert np.all(kappa[~seen] <= 1e-6 * g.a * oracle.sirt.Y00)
    # data weights scale the row weights
    W = np.random.default_rng(0).uniform(0.0, 1.0, g.data_shape)
    RW, DW = oracle.sirt_weights(g, W, B)
    np.testing.assert_allclose(RW.ravel(), W.ravel() * R, rtol=1e-15, atol=0)
    np.testing.assert_array_equal(DW.ravel(), D)


def test_axis_aligned_closed_form():
    # p = +z through voxel centres (a = b, no offsets): every ray crosses n
    # voxels at weight a, every voxel is crossed by exactly one ray
    n, a = 5, 0.5
    st = synth.small_setup(n=(n, n, n), nj=n, nk=n, ell_max=2, n_proj=1, n_seg=4, offsets=False, a=a, b=a)
    st.inner_angle[:] = 0.0
    st.outer_angle[:] = 0.0
    g = oracle_geometry(st)
    B = oracle.basis_matrix(g)
    R, D = oracle.sirt_weights(g, None, B)
    row = np.abs(B[0]).sum(axis=1)                       # [C]
    np.testing.assert_allclose(R[0], np.broadcast_to(1.0 / (n * a * row), R[0].shape), rtol=1e-13)
    col = np.abs(B[0]).sum(axis=0)                       # [K]
    blind = col < 1e-9                                   # Y_2,+-1 vanish on the equator q . z = 0
    assert blind.sum() == 2
    np.testing.assert_allclose(D[..., ~blind], np.broadcast_to(1.0 / (a * col[~blind]), D[..., ~blind].shape),
                               rtol=1e-13)
    assert not np.any(D[..., blind])


@pytest.mark.parametrize("weighted", [False, True])
def test_preconditioned_operator_norm_at_most_one(small, weighted):
    st, g, B, A = small
    W = np.random.default_rng(1).uniform(0.0, 1.0, g.data_shape) if weighted else None
    R, D = oracle.sirt_weights(g, W, B)
    M = np.sqrt(R.ravel())[:, None] * A * np.sqrt(D.ravel())[None, :]
    s = np.linalg.norm(M, 2)
    assert 0.2 < s <= 1.0 + 1e-12


def test_first_steps_are_the_dense_updates(small):
    st, g, B, A = small
    rng = np.random.default_rng(2)
    I = rng.normal(size=g.data_shape)
    c0 = rng.normal(size=g.volume_shape)
    R, D = oracle.sirt_weights(g, None, B)
    r, d, b = R.ravel(), D.ravel(), I.ravel()

    def sirt(x, eta):
        return x + eta * d * (A.T @ (r * (b - A @ x)))

    m = oracle.MITRA(g, c0, I, eta=1.0, momentum=0.0, B=B)
    L = m.step()
    x1 = sirt(c0.ravel(), 1.0)
    np.testing.assert_allclose(m.x.ravel(), x1, rtol=1e-11, atol=1e-12)
    assert L == pytest.approx(float(np.sum(r * (A @ c0.ravel() - b) ** 2)), rel=1e-12)
    # Nesterov schedule: mu_1 = 0, mu_2 = 1/4, mu_3 = 2/5
    m = oracle.MITRA(g, c0, I, eta=0.7, momentum=-1.0, B=B)
    x_prev, x = c0.ravel(), c0.ravel()
    for t in (1, 2, 3):
        m.step()
        y = x + (t - 1.0) / (t + 2.0) * (x - x_prev)
        x_prev, x = x, sirt(y, 0.7)
        np.testing.assert_allclose(m.x.ravel(), x, rtol=1e-11, atol=1e-12)


def test_descent_and_acceleration_on_consistent_data():
    st = synth.small_setup(n=(6, 5, 6), nj=7, nk=7, ell_max=2, n_proj=8, n_seg=4, seed=22)
    g = oracle_geometry(st)
    B = oracle.basis_matrix(g)
    c_true = np.random.default_rng(3).normal(size=g.volume_shape)
    I = oracle.forward(g, c_true, B)
    R, _ = oracle.sirt_weights(g, None, B)
    zero = np.zeros(g.volume_shape)
    L0 = oracle.gradient_residual(g, zero, I, R, B, want_grad=False)[0]
    plain = oracle.MITRA(g, zero, I, eta=1.0, momentum=0.0, B=B)
    losses = [plain.step() for _ in range(40)]
    assert losses[0] == pytest.approx(L0, rel=1e-12)
    assert all(b <= a * (1 + 1e-12) for a, b in zip(losses, losses[1:]))
    fast = oracle.MITRA(g, zero, I, eta=1.0, momentum=-1.0, B=B)
    for _ in range(40):
        fast.step()
    Lp = oracle.gradient_residual(g, plain.x, I, R, B, want_grad=False)[0]
    Lf = oracle.gradient_residual(g, fast.x, I, R, B, want_grad=False)[0]
    assert Lp < 0.2 * L0
    assert Lf < 0.5 * Lp
