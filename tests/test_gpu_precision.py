"""Reduced-precision form (bfloat16 / float16 storage of the coefficient
volume the forward projector reads, float arithmetic and float
back-contracted residual, FP64 reductions) against the FP64 oracle.

Stated tolerances (relative L2 per result): bfloat16 5e-3, float16 1e-3 --
the 2-byte rounding (unit roundoff 2^-9 / 2^-12) of the stored volume bounds
them.  Results that pass through the 2-byte volume must also stay above
1e-5, which shows the 2-byte path is the one that ran; the standalone
adjoint, which never reads the volume, meets the FP32 tolerance 1e-5.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2504_16446_gb300 import synth, tt
from conftest import oracle_geometry

pytestmark = pytest.mark.gpu

TOL = {"bf16": 5e-3, "f16": 1e-3}


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _phantom(st, name):
    ph = synth.phantom(name)
    return oracle.zonal_to_sh(st.ell_max, ph.dirs.reshape(-1, 3),
                              ph.amps.reshape(-1, st.ell_max // 2 + 1)).reshape(st.volume_shape)


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_reduced_precision_on_large_workload_subset(prec):
    # 128^3, l_max 8 (K = 45), 240-projection geometry (4 projections), 8 segments
    st = synth.workload("ell128").subset([0, 57, 131, 222])
    g = oracle_geometry(st)
    c_true = _phantom(st, "ell128")
    I = synth.poisson_counts(oracle.forward(g, c_true), 1e4, seed=2)
    c = (0.6 * c_true).astype(np.float32)
    loss_ref, grad_ref = oracle.gradient_residual(g, c.astype(np.float64), I)
    h = tt.Handle(st, prec)
    cd = torch.as_tensor(c, device="cuda")
    Id = torch.as_tensor(I.astype(np.float32), device="cuda")
    proj = h.project(cd).cpu().numpy()
    e_proj = rel_l2(proj, oracle.forward(g, c.astype(np.float64)))
    loss, grad = h.gradient_residual(cd, Id)
    e_grad = rel_l2(grad.cpu().numpy(), grad_ref)
    e_loss = abs(loss - loss_ref) / loss_ref
    print(f"{prec}: projection {e_proj:.2e}, gradient {e_grad:.2e}, loss {e_loss:.2e}")
    for e in (e_proj, e_grad):
        assert 1e-5 < e <= TOL[prec]
    assert e_loss <= 10 * TOL[prec]


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_reduced_precision_small_geometries(prec):
    for kw in (dict(n=(12, 9, 10), nj=13, nk=11, ell_max=4, n_proj=9, n_seg=5, seed=1),
               dict(n=(8, 10, 6), nj=9, nk=19, ell_max=8, n_proj=3, n_seg=8, seed=3)):
        st = synth.small_setup(**kw)
        g = oracle_geometry(st)
        c = synth.random_volume(st, 1).astype(np.float32)
        R = synth.random_data(st, 2).astype(np.float32)
        h = tt.Handle(st, prec)
        e_f = rel_l2(h.project(torch.as_tensor(c, device="cuda")).cpu().numpy(), oracle.forward(g, c.astype(np.float64)))
        e_a = rel_l2(h.adjoint(torch.as_tensor(R, device="cuda")).cpu().numpy(), oracle.adjoint(g, R.astype(np.float64)))
        assert 1e-5 < e_f <= TOL[prec] and e_a <= 1e-5, (e_f, e_a)


def test_bf16_lbfgs_decreases_and_tracks_fp32():
    st = synth.small_setup(n=(10, 9, 8), nj=10, nk=10, ell_max=4, n_proj=10, n_seg=8, seed=3)
    g = oracle_geometry(st)
    I = synth.gaussian_noise(oracle.forward(g, synth.random_volume(st, 4)), 0.01, seed=5)
    Id = torch.as_tensor(I.astype(np.float32), device="cuda")
    z = torch.zeros(st.volume_shape, dtype=torch.float32, device="cuda")
    runs = {}
    for prec in ("f32", "bf16"):
        h = tt.Handle(st, prec)
        opt = tt.LBFGS(h, z, Id, None, m=10)
        losses = [opt.loss]
        for _ in range(15):
            f, _, status = opt.step()
            assert status == tt.TT_OK
            losses.append(f)
        assert all(b <= a for a, b in zip(losses, losses[1:]))
        runs[prec] = losses
    assert abs(runs["bf16"][-1] - runs["f32"][-1]) <= 0.05 * runs["f32"][0]


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_reduced_precision_on_the_warm_start_test_geometry(prec):
    """128^3, l_max 4 (K = 15), 16 segments: the geometry of the held-out
    phantoms the warm-started bfloat16 solve is timed on (3 projections),
    the first held-out phantom, a generic iterate, Poisson data."""
    st = synth.workload("ell128c16").subset([0, 101, 239])
    g = oracle_geometry(st)
    ph = synth.ellipsoid_phantom(128, 4, 6, 5000)
    c_true = oracle.zonal_to_sh(4, ph.dirs.reshape(-1, 3), ph.amps.reshape(-1, 3)).reshape(st.volume_shape)
    I = synth.poisson_counts(oracle.forward(g, c_true), 1e4, seed=3)
    c = (0.6 * c_true + 0.05 * synth.random_volume(st, 4)).astype(np.float32)
    loss_ref, grad_ref = oracle.gradient_residual(g, c.astype(np.float64), I)
    h = tt.Handle(st, prec)
    cd = torch.as_tensor(c, device="cuda")
    loss, grad = h.gradient_residual(cd, torch.as_tensor(I.astype(np.float32), device="cuda"))
    e_proj = rel_l2(h.project(cd).cpu().numpy(), oracle.forward(g, c.astype(np.float64)))
    e_grad = rel_l2(grad.cpu().numpy(), grad_ref)
    e_loss = abs(loss - loss_ref) / loss_ref
    print(f"{prec}: projection {e_proj:.2e}, gradient {e_grad:.2e}, loss {e_loss:.2e}")
    for e in (e_proj, e_grad):
        assert 1e-5 < e <= TOL[prec]
    assert e_loss <= 10 * TOL[prec]
