"""Differentiation form: regularisers and the torch.autograd front end.

- L2 and Huber-TV values and gradients (libtt kernels) against the oracle
  (FP32 relative L2 1e-5, FP64 1e-12).
- torch.autograd.gradcheck of the projector (whose backward is the
  hand-written adjoint) and of the composite loss squared + 1e-3 L2 +
  1e-2 TV on a 12^3 crop of the plywood phantom, FP64.
- The composite gradient through autograd against the oracle's, on a
  projection subset of the plywood workload (100^3, l_max 6) in FP32.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle.regularizers import l2_norm as or_l2, tv_huber as or_tv
from paper_2504_16446_gb300 import autograd as ta
from paper_2504_16446_gb300 import synth, tt
from conftest import oracle_geometry

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec,tol", [("f32", 1e-5), ("f64", 1e-12)])
@pytest.mark.parametrize("delta", [1e-2, 0.5])
def test_regularisers_match_oracle(prec, tol, delta):
    st = synth.small_setup(n=(9, 7, 11), ell_max=4, n_proj=2, seed=1)
    h = tt.Handle(st, prec)
    dt = torch.float32 if prec == "f32" else torch.float64
    c = (0.1 * synth.random_volume(st, 3)).astype(np.float32 if prec == "f32" else np.float64)
    cd = torch.as_tensor(c, device="cuda")
    v, g = h.tv_huber(cd, delta)
    rv, rg = or_tv(c.astype(np.float64), delta)
    assert abs(v - rv) <= tol * rv
    assert rel_l2(g.cpu().numpy(), rg) <= tol
    v2, g2 = h.l2_norm(cd)
    rv2, rg2 = or_l2(c.astype(np.float64))
    assert abs(v2 - rv2) <= tol * rv2
    assert rel_l2(g2.cpu().numpy(), rg2) <= tol
    assert dt == g.dtype


def test_fp32_sum_of_squares_is_accurate_to_double_rounding():
    """FP32 vectors are reduced with compensated FP32 products and sums per
    thread (Ogita-Rump-Oishi Dot2) and FP64 across threads: the sum of
    squares of a full-size FP32 volume matches the FP64 sum of the same
    float values to 1e-12, far below FP32 rounding."""
    st = synth.workload("ell64")
    h = tt.Handle(st, "f32")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    c = torch.randn(st.volume_shape, device="cuda", generator=gen) * 3.0 + 0.7
    v, _ = h.l2_norm(c, want_grad=False)
    ref = float(np.sum(c.cpu().numpy().astype(np.float64) ** 2))
    assert abs(v - ref) <= 1e-12 * ref


def _crop_setup(n=12, n_proj=6, ell_max=6):
    full = synth.workload("ply100")
    idx = np.linspace(0, full.S - 1, n_proj).round().astype(int)
    sub = full.subset(idx)
    return synth.Setup(shape=(n, n, n), nj=n, nk=n, ell_max=ell_max, inner_angle=sub.inner_angle,
                       outer_angle=sub.outer_angle, seg_start=sub.seg_start, seg_end=sub.seg_end,
                       j_offset=sub.j_offset, k_offset=sub.k_offset)


def _ply_crop_coefficients(st):
    ph = synth.plywood_phantom(100, st.ell_max, seed=3)
    n = st.shape[0]
    sl = slice(44, 44 + n)
    dirs, amps = ph.dirs[sl, sl, sl], ph.amps[sl, sl, sl]
    return oracle.zonal_to_sh(st.ell_max, dirs.reshape(-1, 3), amps.reshape(-1, st.ell_max // 2 + 1)).reshape(st.volume_shape)


def test_gradcheck_projector_fp64():
    st = synth.small_setup(n=(4, 3, 4), nj=4, nk=3, ell_max=2, n_proj=2, n_seg=3, seed=2)
    h = tt.Handle(st, "f64")
    c = torch.randn(st.volume_shape, dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda x: ta.project(h, x), (c,), eps=1e-6, atol=1e-9)


def test_gradcheck_composite_loss_on_12cube_crop_fp64():
    st = _crop_setup()
    h = tt.Handle(st, "f64")
    g_or = oracle_geometry(st)
    c_true = _ply_crop_coefficients(st)
    I = torch.as_tensor(oracle.forward(g_or, c_true), device="cuda")
    c0 = torch.as_tensor(0.7 * c_true + 0.01 * synth.random_volume(st, 5), device="cuda").requires_grad_(True)

    def loss(x):
        return ta.squared_loss(h, x, I) + 1e-3 * ta.l2_norm(h, x) + 1e-2 * ta.tv_huber(h, x, 1e-2)

    assert torch.autograd.gradcheck(loss, (c0,), eps=1e-6, atol=1e-6, rtol=1e-5, fast_mode=True)
    # and the autograd gradient equals the oracle's composite gradient
    L = loss(c0)
    L.backward()
    c_np = c0.detach().cpu().numpy()
    lr, gr = oracle.gradient_residual(g_or, c_np, I.cpu().numpy())
    l2v, l2g = or_l2(c_np)
    tvv, tvg = or_tv(c_np, 1e-2)
    ref_L = lr + 1e-3 * l2v + 1e-2 * tvv
    ref_g = gr + 1e-3 * l2g + 1e-2 * tvg
    assert abs(L.item() - ref_L) <= 1e-12 * ref_L
    assert rel_l2(c0.grad.cpu().numpy(), ref_g) <= 1e-12


def test_composite_gradient_fp32_on_plywood_workload_subset():
    st = synth.workload("ply100").subset([0, 61, 133])
    g_or = oracle_geometry(st)
    ph = synth.phantom("ply100")
    c_true = oracle.zonal_to_sh(6, ph.dirs.reshape(-1, 3), ph.amps.reshape(-1, 4)).reshape(st.volume_shape)
    I = synth.poisson_counts(oracle.forward(g_or, c_true), 5e3, seed=3).astype(np.float32)
    c = (0.5 * c_true).astype(np.float32)
    h = tt.Handle(st, "f32")
    cd = torch.as_tensor(c, device="cuda").requires_grad_(True)
    Id = torch.as_tensor(I, device="cuda")
    L = ta.squared_loss(h, cd, Id) + 1e-3 * ta.l2_norm(h, cd) + 1e-2 * ta.tv_huber(h, cd, 1e-2)
    L.backward()
    c64 = c.astype(np.float64)
    lr, gr = oracle.gradient_residual(g_or, c64, I.astype(np.float64))
    l2v, l2g = or_l2(c64)
    tvv, tvg = or_tv(c64, 1e-2)
    ref_L = lr + 1e-3 * l2v + 1e-2 * tvv
    assert abs(L.item() - ref_L) <= 1e-5 * ref_L
    assert rel_l2(cd.grad.cpu().numpy(), gr + 1e-3 * l2g + 1e-2 * tvg) <= 1e-5
