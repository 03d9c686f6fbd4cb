"""Pins for the oracle's John transform (Joseph's method) and forward model.

Checks: exact chord lengths through a uniform cube, brute-force single-voxel
footprints (each ray intersected with the voxel's own plane, no plane march),
the 90-degree-rotation symmetry of the voxel grid, the isotropic (l = 0)
special case of Eq. (forward_model), and the adjoint identity / dense
transpose.  Geometry references are built with scipy rotations.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2504_16446_gb300 import synth
from conftest import oracle_geometry

FR = {k: np.asarray(v) for k, v in oracle.STANDARD_FRAME.items()}


def _ray_frame(st, s):
    Ra = Rotation.from_rotvec(FR["alpha_axis"] * st.inner_angle[s]).as_matrix()
    Rb = Rotation.from_rotvec(FR["beta_axis"] * st.outer_angle[s]).as_matrix()
    R = Rb @ Ra
    return R.T @ FR["p"], R.T @ FR["j"], R.T @ FR["k"]


def _ray_point(st, s, j, k, js, ks):
    tj = st.b * (j - 0.5 * (st.nj - 1) - st.j_offset[s])
    tk = st.b * (k - 0.5 * (st.nk - 1) - st.k_offset[s])
    return tj * js + tk * ks


def _transverse(st, m):
    return [t for t in range(3) if t != m]


def _index_coords(st, X):
    return X / st.a + 0.5 * (np.asarray(st.shape) - 1)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_uniform_cube_gives_exact_chords(seed):
    n = 9
    st = synth.small_setup(n=(n, n, n), nj=13, nk=13, n_proj=6, seed=seed, a=1.3, b=0.7)
    Y = oracle.john_forward(oracle_geometry(st), np.ones((n, n, n, 1)))[..., 0]
    checked = 0
    for s in range(st.S):
        d, js, ks = _ray_frame(st, s)
        m = int(np.argmax(np.abs(d)))
        uv = _transverse(st, m)
        for j in range(st.nj):
            for k in range(st.nk):
                X0 = _ray_point(st, s, j, k, js, ks)
                ends = []
                for p in (0, n - 1):
                    t = (st.a * (p - 0.5 * (n - 1)) - X0[m]) / d[m]
                    ends.append(_index_coords(st, X0 + t * d)[uv])
                ends = np.array(ends)
                if np.all(ends >= 0) and np.all(ends <= n - 1):
                    assert abs(Y[s, j, k] - n * st.a / abs(d[m])) < 1e-12
                    checked += 1
                elif np.all(ends < -1.0001) or np.all(ends > n + 0.0001):
                    pass
    assert checked > 50


def test_axis_aligned_projection_is_plain_sum():
    n = 5
    st = synth.small_setup(n=(n, n, n), nj=n, nk=n, n_proj=1, offsets=False)
    st.inner_angle[:] = 0.0
    st.outer_angle[:] = 0.0
    c = np.random.default_rng(0).normal(size=(n, n, n, 2))
    Y = oracle.john_forward(oracle_geometry(st), c)
    # p = +z: ray (j, k) runs through voxels (x = k, y = j, all z)
    np.testing.assert_allclose(Y[0], np.transpose(c.sum(axis=2), (1, 0, 2)), atol=1e-13)


def test_offsets_shift_the_ray_by_a_tent_weight():
    n = 5
    st = synth.small_setup(n=(n, n, n), nj=n, nk=n, n_proj=1, offsets=False)
    st.inner_angle[:] = 0.0
    st.outer_angle[:] = 0.0
    st.j_offset[:] = 0.25
    c = np.zeros((n, n, n, 1)); c[2, 3, 1, 0] = 1.0
    Y = oracle.john_forward(oracle_geometry(st), c)[0, :, :, 0]
    # Eq. (real_space_geom): y - (n-1)/2 = j - (n-1)/2 - dj, so pixel j sees y = j - 0.25
    expect = np.zeros((n, n)); expect[3, 2] = 0.75; expect[4, 2] = 0.25
    np.testing.assert_allclose(Y, expect, atol=1e-14)


@pytest.mark.parametrize("shape,seed", [((3, 3, 3), 0), ((4, 5, 3), 1), ((5, 4, 4), 2)])
def test_single_voxel_brute_force(shape, seed):
    st = synth.small_setup(n=shape, nj=8, nk=7, n_proj=7, seed=seed, a=1.1, b=0.9)
    g = oracle_geometry(st)
    rng = np.random.default_rng(seed)
    for _ in range(4):
        v0 = np.array([rng.integers(0, shape[t]) for t in range(3)])
        c = np.zeros((*shape, 1)); c[tuple(v0)] = 1.0
        Y = oracle.john_forward(g, c)[..., 0]
        Xv = st.a * (v0 - 0.5 * (np.asarray(shape) - 1))
        for s in range(st.S):
            d, js, ks = _ray_frame(st, s)
            m = int(np.argmax(np.abs(d)))
            u, v = _transverse(st, m)
            for j in range(st.nj):
                for k in range(st.nk):
                    X0 = _ray_point(st, s, j, k, js, ks)
                    t = (Xv[m] - X0[m]) / d[m]
                    f = _index_coords(st, X0 + t * d)
                    ref = (st.a / abs(d[m])) * max(0.0, 1 - abs(f[u] - v0[u])) * max(0.0, 1 - abs(f[v] - v0[v]))
                    assert abs(Y[s, j, k] - ref) < 1e-13, (s, j, k)


@pytest.mark.parametrize("seed", [0, 1])
def test_quarter_turn_about_the_rotation_axis(seed):
    # alpha -> alpha + 90 deg rotates every ray by R_y(-90deg); the volume
    # f'(X) = f(R_y(90deg) X) = f(z, y, -x) then projects identically.
    n = 6
    st = synth.small_setup(n=(n, n, n), nj=9, nk=8, n_proj=5, seed=seed)
    c = np.random.default_rng(seed).normal(size=(n, n, n, 3))
    c_rot = c[:, :, ::-1, :].transpose(2, 1, 0, 3)
    st2 = synth.Setup(**{**st.__dict__, "inner_angle": st.inner_angle + math.pi / 2})
    Y1 = oracle.john_forward(oracle_geometry(st), c)
    Y2 = oracle.john_forward(oracle_geometry(st2), c_rot)
    np.testing.assert_allclose(Y1, Y2, atol=1e-12)


def test_isotropic_volume_gives_segment_independent_intensity():
    st = synth.small_setup(n=(5, 6, 5), ell_max=4, n_proj=4, n_seg=6, seed=5)
    g = oracle_geometry(st)
    c = np.zeros(st.volume_shape)
    c[..., 0] = np.random.default_rng(0).uniform(size=st.shape)
    I = oracle.forward(g, c)
    Y0 = oracle.john_forward(g, c[..., :1])[..., 0]
    for cc in range(st.C):
        np.testing.assert_allclose(I[..., cc], Y0 / math.sqrt(4 * math.pi), atol=1e-13)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_adjoint_identity(seed):
    st = synth.small_setup(n=(7, 6, 8), nj=9, nk=10, ell_max=4, n_proj=6, n_seg=5, seed=seed)
    g = oracle_geometry(st)
    x = synth.random_volume(st, seed)
    y = synth.random_data(st, seed + 100)
    lhs = np.vdot(oracle.forward(g, x), y)
    rhs = np.vdot(x, oracle.adjoint(g, y))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0) * 10


def test_dense_transpose_on_4cube():
    st = synth.small_setup(n=(4, 4, 4), nj=4, nk=4, ell_max=2, n_proj=3, n_seg=3, seed=9)
    g = oracle_geometry(st)
    B = oracle.basis_matrix(g)
    nv, nd = int(np.prod(st.volume_shape)), int(np.prod(st.data_shape))
    A = np.zeros((nd, nv))
    for col in range(nv):
        e = np.zeros(nv); e[col] = 1.0
        A[:, col] = oracle.forward(g, e.reshape(st.volume_shape), B).ravel()
    AT = np.zeros((nv, nd))
    for col in range(nd):
        e = np.zeros(nd); e[col] = 1.0
        AT[:, col] = oracle.adjoint(g, e.reshape(st.data_shape), B).ravel()
    np.testing.assert_allclose(A.T, AT, atol=1e-14)
    assert np.count_nonzero(np.abs(A) > 1e-12) > 0.05 * A.size
