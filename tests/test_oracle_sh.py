"""Pins for the oracle's real spherical harmonics and quadrature.

Section "Basis sets" (SH) defines the basis only by its band limit; the
reading used here is the orthonormal real SH with even l, no Condon-Shortley
phase, polar axis +z.  Every check below comes from outside the oracle:
exact product quadrature (numpy's Gauss-Legendre), the addition theorem
(scipy's Legendre polynomials), scipy's complex SH, and textbook Cartesian
forms.
"""
import math

import numpy as np
import pytest
import scipy.special as sp

import oracle


def _dirs(theta, phi):
    return np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], -1)


@pytest.mark.parametrize("L", [0, 2, 4, 8, 12])
def test_orthonormal_by_exact_quadrature(L):
    # Products of two degree-<=L SH are degree <= 2L: (L+1) Gauss-Legendre
    # nodes in cos(theta) and 2L+1 equispaced phi integrate them exactly.
    x, w = np.polynomial.legendre.leggauss(L + 1)
    M = 2 * L + 1
    phi = 2 * np.pi * np.arange(M) / M
    T, P = np.meshgrid(np.arccos(x), phi, indexing="ij")
    Wt = (w[:, None] * np.full(M, 2 * np.pi / M)[None, :]).ravel()
    Y = oracle.sh_eval(L, _dirs(T, P).reshape(-1, 3))
    G = Y.T @ (Wt[:, None] * Y)
    assert G.shape == (oracle.num_coeffs(L),) * 2
    np.testing.assert_allclose(G, np.eye(G.shape[0]), atol=1e-13)


@pytest.mark.parametrize("L", [2, 6, 10])
def test_addition_theorem(L):
    rng = np.random.default_rng(1)
    u = rng.normal(size=(20, 3)); u /= np.linalg.norm(u, axis=1, keepdims=True)
    v = rng.normal(size=(20, 3)); v /= np.linalg.norm(v, axis=1, keepdims=True)
    Yu, Yv = oracle.sh_eval(L, u), oracle.sh_eval(L, v)
    i = 0
    for l in range(0, L + 1, 2):
        n = 2 * l + 1
        lhs = np.sum(Yu[:, i:i + n] * Yv[:, i:i + n], axis=1)
        rhs = n / (4 * np.pi) * sp.eval_legendre(l, np.sum(u * v, axis=1))
        np.testing.assert_allclose(lhs, rhs, atol=1e-13)
        i += n


def test_matches_scipy_complex_sh():
    # Real SH without Condon-Shortley phase from scipy's complex SH (which
    # carries the (-1)^m phase): m>0 -> sqrt2 (-1)^m Re Y_l^m, m<0 -> sqrt2 (-1)^m Im Y_l^|m|.
    L = 8
    rng = np.random.default_rng(2)
    th = np.arccos(rng.uniform(-1, 1, 50))
    ph = rng.uniform(0, 2 * np.pi, 50)
    Y = oracle.sh_eval(L, _dirs(th, ph))
    i = 0
    for l in range(0, L + 1, 2):
        for m in range(-l, l + 1):
            am = abs(m)
            z = sp.sph_harm_y(l, am, th, ph)
            if m == 0:
                ref = z.real
            elif m > 0:
                ref = math.sqrt(2) * (-1) ** am * z.real
            else:
                ref = math.sqrt(2) * (-1) ** am * z.imag
            np.testing.assert_allclose(Y[:, i], ref, atol=1e-13, err_msg=f"l={l} m={m}")
            i += 1


def test_textbook_cartesian_forms():
    rng = np.random.default_rng(3)
    d = rng.normal(size=(30, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
    x, y, z = d.T
    Y = oracle.sh_eval(4, d)
    pi = np.pi
    np.testing.assert_allclose(Y[:, 0], 1 / math.sqrt(4 * pi), atol=1e-15)
    # l = 2, m = -2..2 (index 1..5)
    np.testing.assert_allclose(Y[:, 1], math.sqrt(15 / (4 * pi)) * x * y, atol=1e-14)
    np.testing.assert_allclose(Y[:, 2], math.sqrt(15 / (4 * pi)) * y * z, atol=1e-14)
    np.testing.assert_allclose(Y[:, 3], math.sqrt(5 / (16 * pi)) * (3 * z * z - 1), atol=1e-14)
    np.testing.assert_allclose(Y[:, 4], math.sqrt(15 / (4 * pi)) * x * z, atol=1e-14)
    np.testing.assert_allclose(Y[:, 5], math.sqrt(15 / (16 * pi)) * (x * x - y * y), atol=1e-14)
    # l = 4, m = 0 (index 6 + 4)
    np.testing.assert_allclose(Y[:, 10], 3 / 16 * math.sqrt(1 / pi) * (35 * z**4 - 30 * z**2 + 3), atol=1e-14)


def test_poles_are_finite_and_zonal():
    Y = oracle.sh_eval(6, np.array([[0, 0, 1.0], [0, 0, -1.0]]))
    assert np.all(np.isfinite(Y))
    i = 0
    for l in range(0, 7, 2):
        for m in range(-l, l + 1):
            if m != 0:
                assert abs(Y[0, i]) < 1e-15 and abs(Y[1, i]) < 1e-15
            else:
                np.testing.assert_allclose(Y[:, i], math.sqrt((2 * l + 1) / (4 * math.pi)), atol=1e-14)
            i += 1


@pytest.mark.parametrize("n", [1, 2, 5, 32, 64])
def test_gauss_legendre_matches_numpy(n):
    x, w = oracle.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    o = np.argsort(x)
    np.testing.assert_allclose(x[o], xr, atol=1e-14)
    np.testing.assert_allclose(w[o], wr, atol=1e-14)


def test_zonal_to_sh_is_the_rotated_zonal_function():
    # f(q) = sum_l a_l sqrt((2l+1)/4pi) P_l(q.n) evaluated directly (scipy
    # Legendre) must equal sum_i c_i Y_i(q) with c from the addition theorem.
    L = 6
    rng = np.random.default_rng(4)
    n = rng.normal(size=(5, 3)); n /= np.linalg.norm(n, axis=1, keepdims=True)
    a = rng.uniform(0, 1, (5, L // 2 + 1))
    c = oracle.zonal_to_sh(L, n, a)
    q = rng.normal(size=(40, 3)); q /= np.linalg.norm(q, axis=1, keepdims=True)
    Yq = oracle.sh_eval(L, q)
    for t in range(5):
        direct = sum(a[t, li] * math.sqrt((2 * l + 1) / (4 * math.pi)) * sp.eval_legendre(l, q @ n[t])
                     for li, l in enumerate(range(0, L + 1, 2)))
        np.testing.assert_allclose(Yq @ c[t], direct, atol=1e-13)
