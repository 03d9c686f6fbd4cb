"""GPU L-BFGS (tt_lbfgs_*) against the oracle's L-BFGS: the same algorithm
step by step.  FP64: iterates agree to 1e-9 relative after 20 steps; FP32:
each step's loss agrees to 1e-4 relative (differences compound from FP32
rounding), and the loss decreases monotonically."""
import numpy as np
import pytest
import torch

import oracle
from oracle.lbfgs import LBFGS as OracleLBFGS
from paper_2504_16446_gb300 import synth
from paper_2504_16446_gb300 import tt
from conftest import oracle_geometry

pytestmark = pytest.mark.gpu


def _problem(seed=0, n=(8, 8, 8), ell_max=2):
    st = synth.small_setup(n=n, nj=10, nk=10, ell_max=ell_max, n_proj=10, n_seg=8, seed=seed)
    g = oracle_geometry(st)
    truth = synth.random_volume(st, seed + 1)
    I = synth.gaussian_noise(oracle.forward(g, truth), 0.01, seed=seed + 2)
    return st, g, I


def test_lbfgs_fp64_matches_oracle_step_by_step():
    st, g, I = _problem(0)
    B = oracle.basis_matrix(g)
    fg = lambda x: oracle.gradient_residual(g, x.reshape(st.volume_shape), I, None, B)
    ref = OracleLBFGS(fg, np.zeros(int(np.prod(st.volume_shape))), m=10)
    h = tt.Handle(st, "f64")
    Id = torch.as_tensor(I, device="cuda")
    opt = tt.LBFGS(h, torch.zeros(st.volume_shape, dtype=torch.float64, device="cuda"), Id, None, m=10)
    assert abs(opt.loss - ref.f) <= 1e-12 * ref.f
    for it in range(20):
        f_ref, ne_ref, st_ref = ref.step()
        f, ne, status = opt.step()
        assert status == st_ref == 0
        assert ne == ne_ref, it
        assert abs(f - f_ref) <= 1e-9 * f_ref, (it, f, f_ref)
    x = opt.get()[0].cpu().numpy().ravel()
    assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)


def test_lbfgs_fp64_rejected_trials_match_the_oracle():
    """A solution of norm ~0.1 against a first step of length 1: the line
    search rejects three trials before accepting one.  The device enqueues
    each trial's pair and dot products before the Armijo test; a rejected
    trial's must leave no trace in the Gram matrix."""
    st = synth.small_setup(n=(7, 8, 6), nj=10, nk=10, ell_max=2, n_proj=10, n_seg=8, seed=5)
    g = oracle_geometry(st)
    I = synth.gaussian_noise(oracle.forward(g, synth.random_volume(st, 6) * 1e-2), 0.01, seed=7)
    W = synth.random_weights(st, seed=8)
    B = oracle.basis_matrix(g)
    fg = lambda x: oracle.gradient_residual(g, x.reshape(st.volume_shape), I, W, B)
    ref = OracleLBFGS(fg, np.zeros(int(np.prod(st.volume_shape))), m=3)
    h = tt.Handle(st, "f64")
    opt = tt.LBFGS(h, torch.zeros(st.volume_shape, dtype=torch.float64, device="cuda"),
                   torch.as_tensor(I, device="cuda"), torch.as_tensor(W, device="cuda"), m=3)
    evals = []
    g0_norm = float(np.linalg.norm(ref.g))
    for it in range(12):
        f_ref, ne_ref, st_ref = ref.step()
        f, ne, status = opt.step()
        evals.append(ne)
        assert status == st_ref == 0 and ne == ne_ref, it
        assert abs(f - f_ref) <= 1e-9 * f_ref, (it, f, f_ref)
        # the accepted step: halvings from 1/|g0| on the first iteration, from 1 after
        a = opt.stats()["last_step"]
        a_ref = (1.0 / g0_norm if it == 0 else 1.0) * 0.5 ** (ne_ref - 1)
        assert abs(a - a_ref) <= 1e-12 * a_ref, (it, a, a_ref)
        h_it = opt.history[-1]
        assert h_it["step"] == a and h_it["evals"] == ne and h_it["loss"] == f
        assert abs(h_it["relative_residual"] - (f / float(np.sum(W * I * I))) ** 0.5) <= 1e-12
    assert evals[0] == 4
    assert opt.stats()["iterations"] == ref.n_iter == 12
    assert opt.stats()["evaluations"] == ref.total_evals
    x = opt.get()[0].cpu().numpy().ravel()
    assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)


@pytest.mark.parametrize("m", [1, 3])
def test_lbfgs_fp64_short_memory_wraps_like_the_oracle(m):
    """With m = 1 or 3 the pair store wraps around within a few iterations:
    the Gram matrix rows of the replaced pair must be rebuilt exactly."""
    st, g, I = _problem(5, n=(7, 8, 6))
    B = oracle.basis_matrix(g)
    fg = lambda x: oracle.gradient_residual(g, x.reshape(st.volume_shape), I, None, B)
    ref = OracleLBFGS(fg, np.zeros(int(np.prod(st.volume_shape))), m=m)
    h = tt.Handle(st, "f64")
    opt = tt.LBFGS(h, torch.zeros(st.volume_shape, dtype=torch.float64, device="cuda"),
                   torch.as_tensor(I, device="cuda"), None, m=m)
    for it in range(12):
        f_ref, ne_ref, st_ref = ref.step()
        f, ne, status = opt.step()
        assert status == st_ref == 0 and ne == ne_ref, it
        assert abs(f - f_ref) <= 1e-9 * f_ref, (it, f, f_ref)


def test_lbfgs_fp32_tracks_oracle_and_decreases():
    st, g, I = _problem(3, n=(10, 9, 8), ell_max=4)
    B = oracle.basis_matrix(g)
    fg = lambda x: oracle.gradient_residual(g, x.reshape(st.volume_shape), I, None, B)
    ref = OracleLBFGS(fg, np.zeros(int(np.prod(st.volume_shape))), m=10)
    h = tt.Handle(st, "f32")
    Id = torch.as_tensor(I, dtype=torch.float32, device="cuda")
    opt = tt.LBFGS(h, torch.zeros(st.volume_shape, dtype=torch.float32, device="cuda"), Id, None, m=10)
    prev = opt.loss
    hist = [(opt.loss, ref.f)]
    for it in range(10):
        f_ref, ne_ref, _ = ref.step()
        f, ne, status = opt.step()
        hist.append((f, f_ref, ne, ne_ref, status))
        assert status == 0, hist
        assert f <= prev
        prev = f
        assert abs(f - f_ref) <= 1e-4 * f_ref, hist


def test_lbfgs_state_buffers_start_from_recycled_nan_memory():
    # Device memory handed back to the driver full of NaN bit patterns is
    # what a new L-BFGS state's cudaMalloc'd vectors may start with; no
    # kernel may read a vector before writing it.
    junk = torch.full((512 << 20,), float("nan"), dtype=torch.float32, device="cuda")
    del junk
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    st, g, I = _problem(3, n=(10, 9, 8), ell_max=4)
    h = tt.Handle(st, "f32")
    Id = torch.as_tensor(I, dtype=torch.float32, device="cuda")
    opt = tt.LBFGS(h, torch.zeros(st.volume_shape, dtype=torch.float32, device="cuda"), Id, None, m=10)
    f0 = opt.loss
    for _ in range(5):
        f, ne, status = opt.step()
        assert status == tt.TT_OK and np.isfinite(f)
    assert f < 0.2 * f0


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_lbfgs_checkpoint_resume_continues_exactly(prec, tmp_path):
    """Save after the pair store has wrapped (m = 4, 6 iterations), continue
    the original for 5 iterations, restore the checkpoint (through a file)
    into a new state and run the same 5: losses, evaluation counts and the
    final iterate are bit-identical.  Checkpoints of another precision or a
    truncated buffer are rejected."""
    st, g, I = _problem(3, n=(9, 8, 7))
    dt = torch.float32 if prec == "f32" else torch.float64
    h = tt.Handle(st, prec)
    Id = torch.as_tensor(I, device="cuda", dtype=dt)
    a = tt.LBFGS(h, torch.zeros(st.volume_shape, dtype=dt, device="cuda"), Id, None, m=4)
    for _ in range(6):
        a.step()
    ck = a.save()
    loss_at_save = a.loss
    path = tmp_path / "lbfgs.npy"
    np.save(path, ck)
    cont = [a.step()[:2] for _ in range(5)]
    xa = a.get()[0]
    b = tt.LBFGS.restore(h, np.load(path), Id)
    assert b.loss == loss_at_save
    assert b.stats()["iterations"] == 6
    assert [b.step()[:2] for _ in range(5)] == cont
    assert torch.equal(b.get()[0], xa)
    other = tt.Handle(st, "f64" if prec == "f32" else "f32")
    with pytest.raises(tt.TTError):
        tt.LBFGS.restore(other, ck, torch.as_tensor(I, device="cuda", dtype=other.dtype))
    with pytest.raises(tt.TTError):
        tt.LBFGS.restore(h, ck[:-8], Id)
    bad = ck.copy()
    bad[0] ^= 1
    with pytest.raises(tt.TTError):
        tt.LBFGS.restore(h, bad, Id)
    a.close()
    b.close()


def _ray_expected(g, st, u, I, W):
    """Oracle (FP64) start on the ray {a u}: a* = <Au, W I> / <Au, W Au>,
    and the loss and gradient evaluated at a* u."""
    B = oracle.basis_matrix(g)
    Au = oracle.forward(g, u, B)
    w = np.ones_like(I) if W is None else W
    alpha = float(np.sum(w * Au * I) / np.sum(w * Au * Au))
    x = alpha * u
    f, grad = oracle.gradient_residual(g, x, I, W, B)
    return alpha, x, f, grad


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_lbfgs_ray_start_matches_the_oracle(prec):
    """tt_lbfgs_create_ray starts at the loss minimiser along u with the loss
    and gradient of a direct evaluation there, from one evaluation at u and
    the gradient at zero."""
    st, g, I = _problem(4, n=(9, 8, 10), ell_max=4)
    W = synth.random_weights(st, 5)
    u = synth.random_volume(st, 6)
    alpha_ref, x_ref, f_ref, g_ref = _ray_expected(g, st, u, I, W)
    h = tt.Handle(st, prec)
    dt = torch.float64 if prec == "f64" else torch.float32
    Id, Wd, ud = (torch.as_tensor(a, dtype=dt, device="cuda").contiguous() for a in (I, W, u))
    z = torch.zeros(st.volume_shape, dtype=dt, device="cuda")
    L0, g0 = h.gradient_residual(z, Id, Wd)
    opt = tt.LBFGS.from_ray(h, ud, g0, L0, Id, Wd, m=10)
    x, gr, f = opt.get()
    tol = 1e-10 if prec == "f64" else 1e-5
    assert abs(opt.alpha - alpha_ref) <= tol * abs(alpha_ref)
    assert abs(f - f_ref) <= tol * f_ref
    rel = lambda a, b: float(np.linalg.norm(a.cpu().numpy().ravel() - b.ravel()) / np.linalg.norm(b.ravel()))
    assert rel(x, x_ref) <= tol
    assert rel(gr, g_ref) <= (1e-9 if prec == "f64" else 1e-4)
    assert opt.stats() == {"iterations": 0, "evaluations": 1, "last_step": 0.0}
    f_prev = f
    for _ in range(5):
        fn, _, status = opt.step()
        assert status == tt.TT_OK and fn < f_prev
        f_prev = fn


def test_lbfgs_ray_start_recovers_the_scale_of_the_truth():
    """Noise-free data of a volume c: along u = c / 2 the minimiser is a = 2
    exactly, with zero loss and zero gradient there."""
    st, g, _ = _problem(7, n=(8, 9, 8), ell_max=2)
    truth = synth.random_volume(st, 8)
    I = oracle.forward(g, truth)
    h = tt.Handle(st, "f64")
    Id = torch.as_tensor(I, device="cuda")
    z = torch.zeros(st.volume_shape, dtype=torch.float64, device="cuda")
    L0, g0 = h.gradient_residual(z, Id, None)
    opt = tt.LBFGS.from_ray(h, torch.as_tensor(0.5 * truth, device="cuda"), g0, L0, Id, None)
    x, gr, f = opt.get()
    assert abs(opt.alpha - 2.0) <= 1e-12
    assert f <= 1e-20 * L0
    assert float(gr.abs().max()) <= 1e-10 * float(g0.abs().max())
    assert float((x - torch.as_tensor(truth, device="cuda")).abs().max()) <= 1e-12 * float(np.abs(truth).max())


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_lbfgs_ray_start_falls_back_to_zero(prec):
    """A ray that cannot lower the loss (u = 0) leaves the state at zero with
    the loss and gradient given for zero, copied unchanged."""
    st, g, I = _problem(9, n=(8, 8, 8), ell_max=2)
    h = tt.Handle(st, prec)
    dt = torch.float64 if prec == "f64" else torch.float32
    Id = torch.as_tensor(I, dtype=dt, device="cuda")
    z = torch.zeros(st.volume_shape, dtype=dt, device="cuda")
    L0, g0 = h.gradient_residual(z, Id, None)
    opt = tt.LBFGS.from_ray(h, z.clone(), g0, L0, Id, None)
    x, gr, f = opt.get()
    assert opt.alpha == 0.0 and f == L0
    assert torch.equal(gr, g0) and float(x.abs().max()) == 0.0
    with pytest.raises(tt.TTError):
        tt.LBFGS.from_ray(h, z, g0, float("nan"), Id, None)


def test_lbfgs_ray_start_on_bfloat16_storage():
    """On a bfloat16-storage handle (the warm-started form's solver) the ray
    start agrees with the oracle's to the storage rounding -- relative to the
    loss and gradient at zero, the scale of the A u terms it rounds -- and
    the solver descends from it."""
    st, g, I = _problem(11, n=(10, 9, 8), ell_max=4)
    u = synth.random_volume(st, 12)
    alpha_ref, x_ref, f_ref, g_ref = _ray_expected(g, st, u, I, None)
    h = tt.Handle(st, "bf16")
    Id, ud = (torch.as_tensor(a, dtype=torch.float32, device="cuda").contiguous() for a in (I, u))
    z = torch.zeros(st.volume_shape, dtype=torch.float32, device="cuda")
    L0, g0 = h.gradient_residual(z, Id, None)
    opt = tt.LBFGS.from_ray(h, ud, g0, L0, Id, None)
    x, gr, f = opt.get()
    assert abs(opt.alpha - alpha_ref) <= 5e-3 * abs(alpha_ref)
    assert abs(f - f_ref) <= 5e-3 * L0
    g0n = float(np.linalg.norm(g0.cpu().numpy().ravel()))
    assert float(np.linalg.norm(gr.cpu().numpy().ravel() - g_ref.ravel())) <= 5e-3 * g0n
    f_prev = f
    for _ in range(3):
        fn, _, status = opt.step()
        assert status == tt.TT_OK and fn < f_prev
        f_prev = fn


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_lbfgs_null_start_is_the_zero_start(prec):
    """c0 = NULL starts at zero with the evaluation that skips the forward
    projection; the iterates are those of an all-zero c0, bit for bit."""
    st, g, I = _problem(13, n=(9, 9, 8), ell_max=4)
    dt = torch.float64 if prec == "f64" else torch.float32
    h = tt.Handle(st, prec)
    Id = torch.as_tensor(I, dtype=dt, device="cuda")
    a = tt.LBFGS(h, torch.zeros(st.volume_shape, dtype=dt, device="cuda"), Id, None, m=5)
    b = tt.LBFGS(h, None, Id, None, m=5)
    assert a.loss == b.loss
    for _ in range(6):
        fa, na, sa = a.step()
        fb, nb, sb = b.step()
        assert (fa, na, sa) == (fb, nb, sb)
    xa, ga, _ = a.get()
    xb, gb, _ = b.get()
    assert torch.equal(xa, xb) and torch.equal(ga, gb)
