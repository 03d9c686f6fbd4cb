"""GPU parity: libtt (through its C ABI) against the FP64 oracle.

Tolerances: relative L2 <= 1e-5 for FP32 results, <= 1e-12 for the FP64
build (basis matrix 1e-13 absolute), on identical seeded inputs.  Sizes span
several CTA tiles with ragged tails (non-multiple-of-8 detector sizes,
non-cubic volumes, segment counts that are not multiples of 4, sub-pixel
offsets, tilts up to 60 degrees).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2504_16446_gb300 import synth
from paper_2504_16446_gb300 import tt
from conftest import oracle_geometry

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5
F64_TOL = 1e-12


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2504_16446_gb300 import build
    build.build()
    assert torch.cuda.is_available()


SMALL = [
    dict(n=(6, 5, 7), nj=7, nk=6, ell_max=2, n_proj=5, n_seg=4, seed=0),
    dict(n=(12, 9, 10), nj=13, nk=11, ell_max=4, n_proj=9, n_seg=5, seed=1),
    dict(n=(9, 9, 9), nj=17, nk=9, ell_max=6, n_proj=4, n_seg=3, seed=2, a=1.3, b=0.8),
    dict(n=(8, 10, 6), nj=9, nk=19, ell_max=8, n_proj=3, n_seg=8, seed=3, two_theta=0.3),
    dict(n=(5, 5, 5), nj=5, nk=5, ell_max=0, n_proj=6, n_seg=2, seed=4),
    dict(n=(7, 6, 5), nj=6, nk=7, ell_max=10, n_proj=2, n_seg=6, seed=5),
    dict(n=(5, 6, 7), nj=8, nk=8, ell_max=12, n_proj=2, n_seg=4, seed=6),
]


@pytest.mark.parametrize("kw", SMALL, ids=lambda kw: f"L{kw['ell_max']}s{kw['seed']}")
def test_basis_matrix_fp64(kw):
    st = synth.small_setup(**kw)
    h = tt.Handle(st, "f32")
    B = h.basis_matrix().cpu().numpy()
    np.testing.assert_allclose(B, oracle.basis_matrix(oracle_geometry(st)), atol=1e-13, rtol=0)


@pytest.mark.parametrize("kw", SMALL, ids=lambda kw: f"L{kw['ell_max']}s{kw['seed']}")
def test_project_fp32(kw):
    st = synth.small_setup(**kw)
    c = synth.random_volume(st, 10).astype(np.float32)
    ref = oracle.forward(oracle_geometry(st), c.astype(np.float64))
    h = tt.Handle(st, "f32")
    out = h.project(dev(c, torch.float32)).cpu().numpy()
    assert rel_l2(out, ref) <= F32_TOL


@pytest.mark.parametrize("kw", SMALL[:4], ids=lambda kw: f"L{kw['ell_max']}s{kw['seed']}")
def test_project_and_adjoint_fp64(kw):
    st = synth.small_setup(**kw)
    g = oracle_geometry(st)
    c = synth.random_volume(st, 11)
    R = synth.random_data(st, 12)
    h = tt.Handle(st, "f64")
    assert rel_l2(h.project(dev(c, torch.float64)).cpu().numpy(), oracle.forward(g, c)) <= F64_TOL
    assert rel_l2(h.adjoint(dev(R, torch.float64)).cpu().numpy(), oracle.adjoint(g, R)) <= F64_TOL


@pytest.mark.parametrize("kw", SMALL, ids=lambda kw: f"L{kw['ell_max']}s{kw['seed']}")
def test_adjoint_fp32(kw):
    st = synth.small_setup(**kw)
    R = synth.random_data(st, 13).astype(np.float32)
    ref = oracle.adjoint(oracle_geometry(st), R.astype(np.float64))
    h = tt.Handle(st, "f32")
    out = h.adjoint(dev(R, torch.float32)).cpu().numpy()
    assert rel_l2(out, ref) <= F32_TOL


@pytest.mark.parametrize("kw", SMALL, ids=lambda kw: f"L{kw['ell_max']}s{kw['seed']}")
@pytest.mark.parametrize("weights", [False, True])
def test_gradient_residual_fp32(kw, weights):
    st = synth.small_setup(**kw)
    c = synth.random_volume(st, 20).astype(np.float32)
    I = synth.random_data(st, 21).astype(np.float32)
    W = synth.random_weights(st, 22).astype(np.float32) if weights else None
    loss_ref, g_ref = oracle.gradient_residual(oracle_geometry(st), c.astype(np.float64), I.astype(np.float64),
                                               None if W is None else W.astype(np.float64))
    h = tt.Handle(st, "f32")
    loss, g = h.gradient_residual(dev(c, torch.float32), dev(I, torch.float32),
                                  None if W is None else dev(W, torch.float32))
    assert abs(loss - loss_ref) <= F32_TOL * abs(loss_ref)
    assert rel_l2(g.cpu().numpy(), g_ref) <= F32_TOL


@pytest.mark.parametrize("kw", SMALL[:5], ids=lambda kw: f"L{kw['ell_max']}s{kw['seed']}")
def test_gradient_residual_fp64(kw):
    st = synth.small_setup(**kw)
    c = synth.random_volume(st, 30)
    I = synth.random_data(st, 31)
    W = synth.random_weights(st, 32)
    loss_ref, g_ref = oracle.gradient_residual(oracle_geometry(st), c, I, W)
    h = tt.Handle(st, "f64")
    loss, g = h.gradient_residual(dev(c, torch.float64), dev(I, torch.float64), dev(W, torch.float64))
    assert abs(loss - loss_ref) <= F64_TOL * abs(loss_ref)
    assert rel_l2(g.cpu().numpy(), g_ref) <= F64_TOL


def test_early_loss_return_keeps_the_gradient_stream_ordered():
    """tt_gradient_residual returns once the adjoint has published the loss,
    with the adjoint still running.  Back-to-back evaluations of different
    volumes, each gradient consumed on the stream right away (a clone and a
    reduction) and no host synchronisation in between, give the same losses
    and gradients as evaluations separated by full synchronisations."""
    st = synth.workload("ell64")
    h = tt.Handle(st, "f32")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    cs = [torch.randn(st.volume_shape, device="cuda", generator=gen) for _ in range(4)]
    I = torch.rand(st.data_shape, device="cuda", generator=gen) * 64
    torch.cuda.synchronize()
    fast = []
    for c in cs:
        loss, g = h.gradient_residual(c, I)
        fast.append((loss, g.clone(), g.double().sum()))
    slow = []
    for c in cs:
        torch.cuda.synchronize()
        loss, g = h.gradient_residual(c, I)
        torch.cuda.synchronize()
        slow.append((loss, g))
    for (lf, gf, sf), (ls, gs) in zip(fast, slow):
        assert lf == ls
        torch.testing.assert_close(gf, gs, rtol=0, atol=0)
        assert float(sf) == float(gs.double().sum())


def test_switching_streams_orders_the_handle_behind_work_in_flight():
    """Evaluations alternate between two torch streams with no host
    synchronisation: each returns once its loss is published, its adjoint
    still running on the old stream when the next call switches the handle to
    the other stream and overwrites the handle's buffers.  tt_set_stream
    orders the new stream behind the old one, so losses and gradients equal
    those of fully synchronised evaluations bit for bit."""
    st = synth.workload("ell64")
    h = tt.Handle(st, "f32")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(9)
    cs = [torch.randn(st.volume_shape, device="cuda", generator=gen) for _ in range(6)]
    I = torch.rand(st.data_shape, device="cuda", generator=gen) * 64
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    torch.cuda.synchronize()
    fast = []
    for i, c in enumerate(cs):
        with torch.cuda.stream(streams[i % 2]):
            loss, g = h.gradient_residual(c, I)
            fast.append((loss, g.clone()))
    torch.cuda.synchronize()
    for (lf, gf), c in zip(fast, cs):
        torch.cuda.synchronize()
        ls, gs = h.gradient_residual(c, I)
        torch.cuda.synchronize()
        assert lf == ls
        torch.testing.assert_close(gf, gs, rtol=0, atol=0)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_loss_is_the_same_with_and_without_gradient(prec):
    """The loss partials are reduced by the adjoint's first CTA when a gradient
    is wanted and by a one-CTA kernel otherwise: both sum in the same fixed
    order, so the two losses agree bit for bit.  The workload's forward grid
    (64^3, 120 projections: 7680 CTAs) exercises the eight-way strided sum
    with a ragged tail."""
    st = synth.workload("ell64")
    dt = torch.float32 if prec == "f32" else torch.float64
    h = tt.Handle(st, prec)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    c = torch.randn(st.volume_shape, device="cuda", generator=gen, dtype=dt)
    I = torch.rand(st.data_shape, device="cuda", generator=gen, dtype=dt)
    L1, g = h.gradient_residual(c, I, None)
    L0, _ = h.gradient_residual(c, I, None, want_grad=False)
    assert L1 == L0
    assert torch.isfinite(g).all()


@pytest.mark.parametrize("prec,n_proj", [("f32", 300), ("f64", 200)])
def test_adjoint_over_several_parameter_blocks(prec, n_proj):
    """More projections than one adjoint launch holds in its parameter block
    (256 for FP32, 128 for FP64): the launches accumulate in the handle's
    padded gradient and the last one writes the result."""
    st = synth.small_setup(n=(7, 6, 9), nj=8, nk=7, ell_max=4, n_proj=n_proj, n_seg=5, seed=41)
    dt, tol = (torch.float32, F32_TOL) if prec == "f32" else (torch.float64, F64_TOL)
    c = synth.random_volume(st, 42)
    I = synth.random_data(st, 43)
    W = synth.random_weights(st, 44)
    loss_ref, g_ref = oracle.gradient_residual(oracle_geometry(st), c, I, W)
    h = tt.Handle(st, prec)
    loss, g = h.gradient_residual(dev(c, dt), dev(I, dt), dev(W, dt))
    assert abs(loss - loss_ref) <= tol * abs(loss_ref)
    assert rel_l2(g.cpu().numpy(), g_ref) <= tol
    R = synth.random_data(st, 45)
    assert rel_l2(h.adjoint(dev(R, dt)).cpu().numpy(), oracle.adjoint(oracle_geometry(st), R)) <= tol


def test_adjoint_identity_on_gpu_fp64():
    st = synth.small_setup(n=(14, 12, 13), nj=15, nk=17, ell_max=4, n_proj=11, n_seg=6, seed=8)
    h = tt.Handle(st, "f64")
    x = dev(synth.random_volume(st, 1), torch.float64)
    y = dev(synth.random_data(st, 2), torch.float64)
    lhs = float(torch.sum(h.project(x) * y))
    rhs = float(torch.sum(x * h.adjoint(y)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_cylinder_workload_fp64_gradient_and_data():
    # The FP64 workload: 16^3, l_max 2, 30 projections of 16x16, 8 segments,
    # cylinder phantom, data = oracle projection + 1% Gaussian noise.
    st = synth.workload("cyl16")
    g = oracle_geometry(st)
    ph = synth.phantom("cyl16")
    c_true = oracle.zonal_to_sh(2, ph.dirs.reshape(-1, 3), ph.amps.reshape(-1, 2)).reshape(st.volume_shape)
    I = synth.gaussian_noise(oracle.forward(g, c_true), 0.01, seed=0)
    h = tt.Handle(st, "f64")
    assert rel_l2(h.project(dev(c_true, torch.float64)).cpu().numpy(), oracle.forward(g, c_true)) <= F64_TOL
    c0 = np.zeros(st.volume_shape)
    for c in (c0, c_true):
        loss_ref, g_ref = oracle.gradient_residual(g, c, I)
        loss, gg = h.gradient_residual(dev(c, torch.float64), dev(I, torch.float64))
        assert abs(loss - loss_ref) <= F64_TOL * loss_ref
        assert rel_l2(gg.cpu().numpy(), g_ref) <= F64_TOL


def test_zonal_to_sh_matches_oracle():
    rng = np.random.default_rng(0)
    n = rng.normal(size=(1000, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    for L in (0, 2, 4, 8, 12):
        a = rng.uniform(0, 1, (1000, L // 2 + 1))
        ref = oracle.zonal_to_sh(L, n, a)
        out = tt.zonal_to_sh(L, dev(n, torch.float32), dev(a, torch.float32)).cpu().numpy()
        np.testing.assert_allclose(out, ref, atol=1e-5 * max(1.0, np.abs(ref).max()))   # FP32 recurrences


def test_host_entry_point_matches_device_entry_point():
    st = synth.small_setup(n=(10, 11, 9), nj=12, nk=10, ell_max=4, n_proj=7, n_seg=8, seed=9)
    c = synth.random_volume(st, 1).astype(np.float32)
    I = synth.random_data(st, 2).astype(np.float32)
    W = synth.random_weights(st, 3).astype(np.float32)
    h = tt.Handle(st, "f32")
    loss_d, g_d = h.gradient_residual(dev(c, torch.float32), dev(I, torch.float32), dev(W, torch.float32))
    loss_h, g_h = h.gradient_residual_host(c, I, W)
    assert loss_h == loss_d
    np.testing.assert_array_equal(g_h, g_d.cpu().numpy())
    # page-locked buffers: the adjoint writes the gradient straight into g_out
    pin = {k: torch.empty(v.shape, dtype=torch.float32, pin_memory=True) for k, v in (("c", c), ("I", I), ("W", W))}
    for k, v in (("c", c), ("I", I), ("W", W)):
        pin[k].numpy()[...] = v
    g_pin = torch.full(st.volume_shape, float("nan"), dtype=torch.float32, pin_memory=True)
    loss_p, g_p = h.gradient_residual_host(pin["c"].numpy(), pin["I"].numpy(), pin["W"].numpy(), g_out=g_pin.numpy())
    assert loss_p == loss_d
    np.testing.assert_array_equal(g_pin.numpy(), g_d.cpu().numpy())


def test_host_entry_point_pipelined_chunks_on_slab_ordered_forward():
    """128^3, l_max 8, 240 projections: the padded volume exceeds the size at
    which the forward switches to its slab CTA order; the host-buffer path
    runs the forward in four projection chunks overlapped with the data
    copies.  Loss and gradient equal the device path bit for bit."""
    st = synth.workload("ell128")
    h = tt.Handle(st, "f32")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(11)
    c = torch.randn(st.volume_shape, device="cuda", generator=gen)
    I = torch.rand(st.data_shape, device="cuda", generator=gen)
    W = torch.rand(st.data_shape, device="cuda", generator=gen)
    loss_d, g_d = h.gradient_residual(c, I, W)
    loss_h, g_h = h.gradient_residual_host(c.cpu().numpy(), I.cpu().numpy(), W.cpu().numpy())
    assert loss_h == loss_d
    assert np.array_equal(g_h, g_d.cpu().numpy())


def test_nonfinite_input_is_reported():
    st = synth.small_setup(seed=1)
    c = synth.random_volume(st, 1).astype(np.float32)
    c[1, 2, 3, 0] = np.nan
    h = tt.Handle(st, "f32")
    with pytest.raises(tt.TTError) as e:
        h.gradient_residual(dev(c, torch.float32), dev(synth.random_data(st, 2), torch.float32))
    assert e.value.status == tt.TT_NONFINITE


def test_precision_mismatch_and_bad_shapes_rejected():
    st = synth.small_setup(seed=2)
    h = tt.Handle(st, "f32")
    lib = tt.load()
    x = torch.zeros(st.volume_shape, dtype=torch.float64, device="cuda")
    y = torch.zeros(st.data_shape, dtype=torch.float64, device="cuda")
    assert lib.tt_project_f64(h._h, x.data_ptr(), y.data_ptr()) == tt.TT_INVALID_ARG
    x32 = torch.zeros(st.volume_shape, dtype=torch.float32, device="cuda")
    assert lib.tt_project(h._h, x32.data_ptr() + 4, y.data_ptr()) == tt.TT_INVALID_ARG   # misaligned
    assert lib.tt_project(h._h, None, y.data_ptr()) == tt.TT_INVALID_ARG
    with pytest.raises(ValueError):
        h.project(torch.zeros((3, 3, 3, 6), device="cuda"))


def test_degenerate_sizes():
    # one voxel, one pixel, one projection, one segment
    st = synth.small_setup(n=(1, 1, 1), nj=1, nk=1, ell_max=2, n_proj=1, n_seg=1, seed=3, offsets=False)
    c = synth.random_volume(st, 0).astype(np.float32)
    I = synth.random_data(st, 1).astype(np.float32)
    loss_ref, g_ref = oracle.gradient_residual(oracle_geometry(st), c.astype(np.float64), I.astype(np.float64))
    h = tt.Handle(st, "f32")
    loss, g = h.gradient_residual(dev(c, torch.float32), dev(I, torch.float32))
    assert abs(loss - loss_ref) <= F32_TOL * abs(loss_ref)
    assert rel_l2(g.cpu().numpy(), g_ref) <= F32_TOL
    # a detector that misses the volume entirely: zero projection, zero gradient
    st2 = synth.small_setup(n=(4, 4, 4), nj=3, nk=3, n_proj=2, seed=4, offsets=False)
    st2.j_offset[:] = 50.0
    h2 = tt.Handle(st2, "f32")
    I2 = dev(synth.random_data(st2, 5), torch.float32)
    loss2, g2 = h2.gradient_residual(torch.zeros(st2.volume_shape, device="cuda"), I2)
    assert float(torch.abs(h2.project(dev(synth.random_volume(st2, 1), torch.float32))).max()) == 0.0
    assert float(torch.abs(g2).max()) == 0.0
    assert abs(loss2 - float(torch.sum(I2.double() ** 2))) <= 1e-6 * loss2


@pytest.mark.parametrize("prec", ["f32", "f64", "bf16"])
def test_gradient_at_zero_without_a_volume(prec):
    """c = NULL evaluates at c = 0 without projecting a volume (the forward
    kernel marches nothing): loss sum W I^2 and gradient -2 A^T W I, bit for
    bit those of an all-zero volume, with and without weights.  With the
    staged forward kernel selected the zero volume still takes the L1
    kernel, whose gradients the staged one matches bit for bit (its loss
    partials are summed over other ray tiles, so the loss only to 1e-12)."""
    st = synth.small_setup(n=(12, 10, 11), nj=12, nk=11, ell_max=4, n_proj=9, n_seg=8, seed=17)
    dt = torch.float64 if prec == "f64" else torch.float32
    I = dev(synth.random_data(st, 18), dt)
    W = dev(synth.random_weights(st, 19), dt)
    z = torch.zeros(st.volume_shape, dtype=dt, device="cuda")
    h = tt.Handle(st, prec)
    kinds = ["l1", "staged"] if prec == "f32" else ["auto"]
    for kind in kinds:
        h.set_forward_kernel(kind)
        for Wi in (None, W):
            loss_z, g_z = h.gradient_residual(z, I, Wi)
            loss_n, g_n = h.gradient_residual(None, I, Wi)
            loss_only, _ = h.gradient_residual(None, I, Wi, want_grad=False)
            if kind == "staged":
                assert abs(loss_n - loss_z) <= 1e-12 * loss_z
            else:
                assert loss_n == loss_z
            assert loss_only == loss_n
            assert torch.equal(g_n, g_z)
            Wd = torch.ones_like(I) if Wi is None else Wi
            assert abs(loss_n - float((Wd.double() * I.double() ** 2).sum())) <= 1e-6 * loss_n


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_host_entry_point_on_two_byte_storage(prec):
    """The host-buffer entry point on a 2-byte-storage handle: the same loss
    and gradient as the device entry point, bit for bit."""
    st = synth.small_setup(n=(11, 10, 12), nj=12, nk=11, ell_max=4, n_proj=9, n_seg=8, seed=27)
    c = synth.random_volume(st, 1).astype(np.float32)
    I = synth.random_data(st, 2).astype(np.float32)
    W = synth.random_weights(st, 3).astype(np.float32)
    h = tt.Handle(st, prec)
    loss_d, g_d = h.gradient_residual(dev(c, torch.float32), dev(I, torch.float32), dev(W, torch.float32))
    loss_h, g_h = h.gradient_residual_host(c, I, W)
    assert loss_h == loss_d
    np.testing.assert_array_equal(g_h, g_d.cpu().numpy())
