"""GPU parity of the SIRT weights and the MITRA iteration (Section "Standard
reconstruction pipelines") against the FP64 oracle, through the C ABI.

Tolerances: relative L2 <= 1e-5 (FP32) / 1e-12 (FP64) for the row and
column sums of |A| that the weights invert (1/R, 1/D: the projector's own
outputs; an inverse amplifies the relative error of the short chords of rays
that graze the volume, so the weights themselves are not compared in L2), the
same zero pattern (rays that miss the volume, voxel channels that no ray
sees); the iterates after a few iterations within 3e-5 (FP32: each step adds
one evaluation's rounding, damped by the contraction) / 1e-11 (FP64).  The
bfloat16-storage handle stores the column sums in bfloat16 before the
adjoint: D within 1e-2.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2504_16446_gb300 import synth, tt
from conftest import oracle_geometry

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def inv(x):
    """1/x on the nonzero entries (the sums of |A| behind the weights), 0 elsewhere."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    out[x != 0] = 1.0 / x[x != 0]
    return out


def dev(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2504_16446_gb300 import build
    build.build()
    assert torch.cuda.is_available()


CASES = [
    dict(n=(6, 5, 7), nj=7, nk=6, ell_max=2, n_proj=5, n_seg=4, seed=0),
    dict(n=(12, 9, 10), nj=13, nk=11, ell_max=4, n_proj=9, n_seg=5, seed=1),
    dict(n=(9, 9, 9), nj=17, nk=9, ell_max=6, n_proj=4, n_seg=3, seed=2, a=1.3, b=0.8),
    dict(n=(8, 10, 6), nj=9, nk=19, ell_max=8, n_proj=3, n_seg=8, seed=3, two_theta=0.3),
]
PREC = {"f32": (torch.float32, 1e-5), "f64": (torch.float64, 1e-12)}


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("kw", CASES, ids=lambda kw: f"L{kw['ell_max']}s{kw['seed']}")
@pytest.mark.parametrize("weighted", [False, True])
def test_sirt_weights_match_oracle(kw, prec, weighted):
    dt, tol = PREC[prec]
    st = synth.small_setup(**kw)
    g = oracle_geometry(st)
    W = synth.random_weights(st, seed=kw["seed"] + 40) if weighted else None
    R0, D0 = oracle.sirt_weights(g, W)
    h = tt.Handle(st, prec)
    R, D = h.sirt_weights(None if W is None else dev(W, dt))
    R, D = R.cpu().numpy(), D.cpu().numpy()
    np.testing.assert_array_equal(R > 0, R0 > 0)
    np.testing.assert_array_equal(D > 0, D0 > 0)
    assert (R0 > 0).mean() > 0.2 and (D0 > 0).mean() > 0.5
    assert rel_l2(inv(R), inv(R0)) <= tol
    assert rel_l2(inv(D), inv(D0)) <= tol


def test_sirt_weights_bf16_storage():
    kw = CASES[1]
    st = synth.small_setup(**kw)
    R0, D0 = oracle.sirt_weights(oracle_geometry(st))
    R, D = tt.Handle(st, "bf16").sirt_weights()
    R, D = R.cpu().numpy(), D.cpu().numpy()
    np.testing.assert_array_equal(R > 0, R0 > 0)
    np.testing.assert_array_equal(D > 0, D0 > 0)
    assert rel_l2(inv(R), inv(R0)) <= 1e-5          # the unit volume is exact in bfloat16
    assert rel_l2(inv(D), inv(D0)) <= 1e-2


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("momentum", [0.0, -1.0, 0.5])
def test_mitra_iterates_match_oracle(prec, momentum):
    dt, _ = PREC[prec]
    tol = 3e-5 if prec == "f32" else 1e-11
    kw = CASES[1]
    st = synth.small_setup(**kw)
    g = oracle_geometry(st)
    c0 = synth.random_volume(st, seed=7) * 0.1
    I = synth.random_data(st, seed=8)
    W = synth.random_weights(st, seed=9)
    ref = oracle.MITRA(g, c0, I, W, eta=1.3, momentum=momentum)
    h = tt.Handle(st, prec)
    m = tt.MITRA(h, dev(c0, dt), dev(I, dt), dev(W, dt), eta=1.3, momentum=momentum)
    for t in range(4):
        L = m.step()
        L0 = ref.step()
        assert abs(L - L0) <= tol * abs(L0), (t, L, L0)
        x, R, D, it = m.get()
        assert it == t + 1
        assert rel_l2(x.cpu().numpy(), ref.x) <= tol, t
    assert rel_l2(inv(R.cpu().numpy()), inv(ref.R)) <= max(tol, 1e-12)
    m.close()


def test_mitra_step_without_loss_is_the_same_iteration():
    st = synth.small_setup(**CASES[0])
    c0 = torch.zeros(st.volume_shape, dtype=torch.float32, device="cuda")
    I = dev(synth.random_data(st, seed=3), torch.float32)
    h = tt.Handle(st, "f32")
    a = tt.MITRA(h, c0, I)
    b = tt.MITRA(h, c0, I)
    for _ in range(5):
        a.step()
        assert b.step(want_loss=False) is None
    torch.testing.assert_close(a.get()[0], b.get()[0], rtol=0, atol=0)


def test_mitra_rejects_unstable_parameters():
    st = synth.small_setup(**CASES[0])
    h = tt.Handle(st, "f32")
    c0 = torch.zeros(st.volume_shape, dtype=torch.float32, device="cuda")
    I = torch.zeros(st.data_shape, dtype=torch.float32, device="cuda")
    for eta, mom in ((2.0, 0.0), (0.0, 0.0), (1.0, 1.0)):
        with pytest.raises(tt.TTError):
            tt.MITRA(h, c0, I, eta=eta, momentum=mom)


def test_sirt_weights_full_size_ell64():
    """64^3, l_max 4, 120 projections of 64 x 64 x 16 segments: every weight."""
    st = synth.workload("ell64")
    R0, D0 = oracle.sirt_weights(oracle_geometry(st))
    R, D = tt.Handle(st, "f32").sirt_weights()
    R, D = R.cpu().numpy(), D.cpu().numpy()
    np.testing.assert_array_equal(R > 0, R0 > 0)
    np.testing.assert_array_equal(D > 0, D0 > 0)
    assert rel_l2(inv(R), inv(R0)) <= 1e-5 and rel_l2(inv(D), inv(D0)) <= 1e-5


def test_mitra_descends_on_ell64():
    """Plain SIRT (momentum 0) decreases L_R monotonically on the 64^3 workload;
    Nesterov momentum reaches a lower L_R in the same number of iterations."""
    st = synth.workload("ell64")
    h = tt.Handle(st, "f32")
    ph = synth.phantom("ell64")
    dirs = torch.as_tensor(ph.dirs.reshape(-1, 3), dtype=torch.float32, device="cuda")
    amps = torch.as_tensor(ph.amps.reshape(-1, st.ell_max // 2 + 1), dtype=torch.float32, device="cuda")
    c_true = tt.zonal_to_sh(st.ell_max, dirs, amps).reshape(st.volume_shape).contiguous()
    I = h.project(c_true)
    z = torch.zeros_like(c_true)
    plain = tt.MITRA(h, z, I, eta=1.0, momentum=0.0)
    losses = [plain.step() for _ in range(30)]
    assert all(b <= a * (1 + 1e-6) for a, b in zip(losses, losses[1:]))
    fast = tt.MITRA(h, z, I, eta=1.0, momentum=-1.0)
    for _ in range(30):
        fast.step(want_loss=False)
    R = plain.get()[1]
    Lp = h.gradient_residual(plain.get()[0], I, R, want_grad=False)[0]
    Lf = h.gradient_residual(fast.get()[0], I, R, want_grad=False)[0]
    assert Lp < 0.5 * losses[0]
    assert Lf < Lp
