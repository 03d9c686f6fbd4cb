"""Parity at the full workload sizes, in the launch configuration the bench
times (the whole 64^3 / l_max 4 / 120 x 64^2 x 16 problem through one handle),
and on projection subsets of the larger workloads (same kernels, fewer CTAs
along the projection axis) where the oracle would take minutes."""
import numpy as np
import pytest
import torch

import oracle
from paper_2504_16446_gb300 import synth
from paper_2504_16446_gb300 import tt
from conftest import oracle_geometry

pytestmark = pytest.mark.gpu
TOL = 1e-5


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _phantom_c(name, st):
    ph = synth.phantom(name)
    return oracle.zonal_to_sh(st.ell_max, ph.dirs.reshape(-1, 3),
                              ph.amps.reshape(-1, st.ell_max // 2 + 1)).reshape(st.volume_shape)


def test_ell64_full_gradient():
    st = synth.workload("ell64")
    g = oracle_geometry(st)
    c_true = _phantom_c("ell64", st).astype(np.float32)
    B = oracle.basis_matrix(g)
    I = synth.poisson_counts(oracle.forward(g, c_true.astype(np.float64), B), 1e4, seed=1).astype(np.float32)
    c = (0.5 * c_true + 0.1 * synth.random_volume(st, 7)).astype(np.float32)   # a generic iterate
    loss_ref, g_ref = oracle.gradient_residual(g, c.astype(np.float64), I.astype(np.float64), None, B)
    h = tt.Handle(st, "f32")
    loss, gg = h.gradient_residual(torch.as_tensor(c, device="cuda"), torch.as_tensor(I, device="cuda"))
    assert abs(loss - loss_ref) <= TOL * loss_ref
    assert rel_l2(gg.cpu().numpy(), g_ref) <= TOL
    Ip = h.project(torch.as_tensor(c_true, device="cuda")).cpu().numpy()
    assert rel_l2(Ip, oracle.forward(g, c_true.astype(np.float64), B)) <= TOL


@pytest.mark.parametrize("name,proj", [("ell128", [0, 37, 118, 239]), ("ply100", [3, 90, 177])])
def test_large_workloads_on_projection_subsets(name, proj):
    st = synth.workload(name).subset(proj)
    g = oracle_geometry(st)
    c = _phantom_c(name, st).astype(np.float32)
    I = synth.random_data(st, 3).astype(np.float32) + 1.0
    loss_ref, g_ref = oracle.gradient_residual(g, c.astype(np.float64), I.astype(np.float64))
    h = tt.Handle(st, "f32")
    loss, gg = h.gradient_residual(torch.as_tensor(c, device="cuda"), torch.as_tensor(I, device="cuda"))
    assert abs(loss - loss_ref) <= TOL * loss_ref
    assert rel_l2(gg.cpu().numpy(), g_ref) <= TOL


@pytest.mark.parametrize("name,proj", [("ell128c16", [0, 101, 239]), ("paper247_l2", [0, 123, 246]),
                                       ("paper247_l4", [7, 200]), ("paper247_l8", [50, 180])])
def test_timed_workloads_on_projection_subsets(name, proj):
    """The held-out test geometry of the warm start (128^3, l_max 4, 16
    segments: the slab-ordered forward at K = 15) and the paper dataset's
    shape (55 x 65 x 55 volume, 65 x 55 pixels, 8 segments, l_max 2 / 4 /
    8: a non-cubic volume and detector) on projection subsets, random
    iterate and data, with and without weights."""
    st = synth.workload(name).subset(proj)
    g = oracle_geometry(st)
    c = synth.random_volume(st, 41).astype(np.float32)
    I = synth.random_data(st, 42).astype(np.float32) + 1.0
    W = synth.random_weights(st, 43).astype(np.float32)
    h = tt.Handle(st, "f32")
    for Wi in (None, W):
        loss_ref, g_ref = oracle.gradient_residual(g, c.astype(np.float64), I.astype(np.float64),
                                                   None if Wi is None else Wi.astype(np.float64))
        loss, gg = h.gradient_residual(torch.as_tensor(c, device="cuda"), torch.as_tensor(I, device="cuda"),
                                       None if Wi is None else torch.as_tensor(Wi, device="cuda"))
        assert abs(loss - loss_ref) <= TOL * loss_ref
        assert rel_l2(gg.cpu().numpy(), g_ref) <= TOL


def test_ell64_adjoint_identity_fp32():
    st = synth.workload("ell64")
    h = tt.Handle(st, "f32")
    x = torch.as_tensor(synth.random_volume(st, 1, np.float32), device="cuda")
    # y = A x + noise keeps <Ax, y> away from cancellation
    y = h.project(x) + torch.as_tensor(synth.random_data(st, 2, np.float32), device="cuda")
    lhs = float(torch.sum(h.project(x).double() * y.double()))
    rhs = float(torch.sum(x.double() * h.adjoint(y).double()))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
