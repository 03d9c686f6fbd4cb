"""Pins for the oracle's geometry and basis matrix, Eq. (projection_matrix).

The rotation is checked against scipy's rotation vectors (right-handed); the
basis matrix against a closed form: on any circle of directions q(phi) an
SH of degree l is a trigonometric polynomial of degree <= l in phi, so 2L+1
equispaced samples give its Fourier coefficients exactly and the segment mean
integrates in closed form.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2504_16446_gb300 import synth
from conftest import oracle_geometry

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_standard_frame_matches_paper_table():
    with open(os.path.join(GOLDEN, "standard_geometry.json")) as f:
        gold = json.load(f)
    names = dict(p="p_direction_0", j="j_direction_0", k="k_direction_0",
                 q0="detector_direction_origin", q90="detector_direction_positive_90",
                 alpha_axis="inner_axis", beta_axis="outer_axis")
    for ours, theirs in names.items():
        assert tuple(oracle.STANDARD_FRAME[ours]) == tuple(gold[theirs])


def test_rotation_is_right_handed_rodrigues():
    rng = np.random.default_rng(0)
    for _ in range(10):
        ax = rng.normal(size=3); ax /= np.linalg.norm(ax)
        t = rng.uniform(-4, 4)
        np.testing.assert_allclose(oracle.rotation(ax, t),
                                   Rotation.from_rotvec(ax * t).as_matrix(), atol=1e-14)


def _scipy_Rs(alpha, beta, frame=oracle.STANDARD_FRAME):
    Ra = Rotation.from_rotvec(np.asarray(frame["alpha_axis"]) * alpha).as_matrix()
    Rb = Rotation.from_rotvec(np.asarray(frame["beta_axis"]) * beta).as_matrix()
    return Rb @ Ra


def test_projection_frame_is_RsT_applied_to_lab_vectors():
    st = synth.small_setup(n_proj=6, seed=3)
    g = oracle_geometry(st)
    for s in range(st.S):
        R = _scipy_Rs(st.inner_angle[s], st.outer_angle[s])
        F = oracle.projection_frame(g, s)
        for key in ("p", "j", "k", "q0", "q90"):
            np.testing.assert_allclose(F[key], R.T @ np.asarray(oracle.STANDARD_FRAME[key]), atol=1e-14)


def _closed_form_B(st, s, ell_max):
    """Segment means of Y_i(R_s^T q(phi)) by exact Fourier integration."""
    L = ell_max
    M = 2 * L + 1
    R = _scipy_Rs(st.inner_angle[s], st.outer_angle[s])
    fr = oracle.STANDARD_FRAME
    th = 0.5 * st.two_theta
    phi = 2 * np.pi * np.arange(M) / M
    q = (math.cos(th) * (np.cos(phi)[:, None] * np.asarray(fr["q0"]) + np.sin(phi)[:, None] * np.asarray(fr["q90"]))
         - math.sin(th) * np.asarray(fr["p"]))
    Y = oracle.sh_eval(L, q @ R)           # rows: R^T q
    coef = np.fft.fft(Y, axis=0) / M        # f(phi) = sum_n coef[n] e^{i n phi}
    freqs = np.fft.fftfreq(M, d=1.0 / M)
    out = np.zeros((st.C, Y.shape[1]))
    for c in range(st.C):
        a0, a1 = st.seg_start[c], st.seg_end[c]
        acc = np.zeros(Y.shape[1], dtype=complex)
        for n, cf in zip(freqs, coef):
            if n == 0:
                acc += cf * (a1 - a0)
            else:
                acc += cf * (np.exp(1j * n * a1) - np.exp(1j * n * a0)) / (1j * n)
        out[c] = (acc / (a1 - a0)).real
    return out


@pytest.mark.parametrize("L,two_theta", [(2, 0.0), (4, 0.0), (8, 0.0), (6, 0.4)])
def test_basis_matrix_closed_form(L, two_theta):
    st = synth.small_setup(ell_max=L, n_proj=5, n_seg=7, seed=L, two_theta=two_theta)
    # uneven segments, including one wider than pi/2
    st.seg_start = np.array([0.0, 0.3, 0.5, 1.2, 2.9, 3.0, 4.0])
    st.seg_end = np.array([0.3, 0.5, 1.2, 2.9, 3.0, 4.0, 6.2])
    B = oracle.basis_matrix(oracle_geometry(st), 32)
    for s in range(st.S):
        np.testing.assert_allclose(B[s], _closed_form_B(st, s, L), atol=1e-14)


def test_basis_matrix_isotropic_and_row_sums():
    st = synth.workload("cyl16")
    B = oracle.basis_matrix(oracle_geometry(st))
    np.testing.assert_allclose(B[:, :, 0], 1 / math.sqrt(4 * math.pi), atol=1e-15)
    # segments tile [0, pi): sum_c dphi_c B[s,c,0] = pi Y_00 for every s
    dphi = st.seg_end - st.seg_start
    np.testing.assert_allclose(B[:, :, 0] @ dphi, math.pi / math.sqrt(4 * math.pi), atol=1e-14)


def test_main_axis_tie_break():
    assert oracle.main_axis([0.5, 0.5, 0.1]) == 0
    s = math.sqrt(0.5)
    assert oracle.main_axis([0.1, -s, s * (1 + 1e-15)]) == 1
    assert oracle.main_axis([0.0, 0.2, -0.9]) == 2
