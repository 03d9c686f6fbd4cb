"""The staged forward march (taps staged in shared memory by a copy warp)
against the tap-pair march that reads them from L1, and against the oracle.

Both kernels add the same FP32 products in the same order, so projections,
back-contracted residuals and gradients must agree bit for bit; the loss is
summed over ray tiles of different shapes and agrees to rounding.  The cases
cover partial ray tiles, sub-pixel offsets, tilts up to 60 degrees (every
main axis, hence both padded volume copies), pixel pitches other than the
voxel size, the bench's 64^3 geometry, and the slab-ordered 128^3 launch with
its chunked host-buffer path.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2504_16446_gb300 import synth
from paper_2504_16446_gb300 import tt
from conftest import oracle_geometry

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2504_16446_gb300 import build
    build.build()
    assert torch.cuda.is_available()


CASES = [
    dict(n=(12, 9, 10), nj=13, nk=11, ell_max=4, n_proj=9, n_seg=5, seed=1),
    dict(n=(16, 14, 15), nj=20, nk=37, ell_max=4, n_proj=12, n_seg=16, seed=7),
    dict(n=(9, 7, 11), nj=8, nk=7, ell_max=4, n_proj=10, n_seg=6, seed=8, a=1.1, b=0.9),
    dict(n=(14, 12, 13), nj=9, nk=17, ell_max=4, n_proj=8, n_seg=4, seed=9, b=1.5),
    dict(n=(5, 6, 5), nj=1, nk=1, ell_max=4, n_proj=6, n_seg=3, seed=10),
]


def _both(h, fn):
    out = {}
    for kind in ("l1", "staged"):
        h.set_forward_kernel(kind)
        out[kind] = fn()
    h.set_forward_kernel("auto")
    return out["l1"], out["staged"]


@pytest.mark.parametrize("kw", CASES, ids=lambda kw: f"s{kw['seed']}")
def test_staged_forward_equals_l1_forward_bitwise_and_matches_oracle(kw):
    st = synth.small_setup(**kw)
    c = synth.random_volume(st, 40).astype(np.float32)
    I = synth.random_data(st, 41).astype(np.float32)
    W = synth.random_weights(st, 42).astype(np.float32)
    h = tt.Handle(st, "f32")
    cd, Id, Wd = dev(c), dev(I), dev(W)
    p1, p2 = _both(h, lambda: h.project(cd).cpu().numpy())
    np.testing.assert_array_equal(p2, p1)
    (l1, g1), (l2, g2) = _both(h, lambda: h.gradient_residual(cd, Id, Wd))
    np.testing.assert_array_equal(g2.cpu().numpy(), g1.cpu().numpy())
    assert abs(l2 - l1) <= 1e-6 * abs(l1)
    g = oracle_geometry(st)
    assert rel_l2(p2, oracle.forward(g, c.astype(np.float64))) <= F32_TOL
    loss_ref, g_ref = oracle.gradient_residual(g, c.astype(np.float64), I.astype(np.float64), W.astype(np.float64))
    assert abs(l2 - loss_ref) <= F32_TOL * abs(loss_ref)
    assert rel_l2(g2.cpu().numpy(), g_ref) <= F32_TOL


@pytest.mark.parametrize("name", ["ell64", "ell128c16"])
def test_staged_forward_equals_l1_forward_on_the_workload_geometries(name):
    """ell64: the bench's geometry (20 rotations x 6 tilts, 64 x 64 rays);
    ell128c16: 128^3, where the padded volume takes the slab CTA order, and
    the host-buffer path runs the forward in projection chunks."""
    st = synth.workload(name)
    h = tt.Handle(st, "f32")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    c = torch.randn(st.volume_shape, device="cuda", generator=gen)
    I = torch.rand(st.data_shape, device="cuda", generator=gen)
    W = torch.rand(st.data_shape, device="cuda", generator=gen)
    p1, p2 = _both(h, lambda: h.project(c))
    assert torch.equal(p1, p2)
    (l1, g1), (l2, g2) = _both(h, lambda: h.gradient_residual(c, I, W))
    assert torch.equal(g1, g2)
    assert abs(l2 - l1) <= 1e-6 * abs(l1)
    if name == "ell128c16":
        h.set_forward_kernel("staged")
        lh, gh = h.gradient_residual_host(c.cpu().numpy(), I.cpu().numpy(), W.cpu().numpy())
        assert lh == l2
        assert np.array_equal(gh, g2.cpu().numpy())


def test_staged_forward_applies_to_fp32_storage_with_16_channels_only():
    st4 = synth.small_setup(ell_max=4, seed=3)
    for prec in ("f64", "bf16", "f16"):
        h = tt.Handle(st4, prec)
        with pytest.raises(tt.TTError) as e:
            h.set_forward_kernel("staged")
        assert e.value.status == tt.TT_UNSUPPORTED
        h.set_forward_kernel("l1")
        h.set_forward_kernel("auto")
    h = tt.Handle(synth.small_setup(ell_max=2, seed=3), "f32")
    with pytest.raises(tt.TTError) as e:
        h.set_forward_kernel("staged")
    assert e.value.status == tt.TT_UNSUPPORTED
    h = tt.Handle(st4, "f32")
    assert h.lib.tt_set_forward_kernel(h._h, 3) == tt.TT_INVALID_ARG
    assert h.lib.tt_set_forward_kernel(None, 0) == tt.TT_INVALID_ARG


def test_footprint_too_large_for_the_ring_is_refused():
    """Pixels of 4 voxels: a 8 x 16 ray tile's box (about 33 x 33 voxels per
    plane at these tilts) needs more than the shared memory of a CTA; the
    staged kernel is refused and the handle keeps projecting with the L1
    march."""
    st = synth.small_setup(n=(24, 24, 24), nj=12, nk=12, ell_max=4, n_proj=6, n_seg=4, seed=12, b=4.0)
    h = tt.Handle(st, "f32")
    with pytest.raises(tt.TTError) as e:
        h.set_forward_kernel("staged")
    assert e.value.status == tt.TT_UNSUPPORTED
    c = synth.random_volume(st, 1).astype(np.float32)
    out = h.project(dev(c)).cpu().numpy()
    assert rel_l2(out, oracle.forward(oracle_geometry(st), c.astype(np.float64))) <= F32_TOL
