"""Pins for the oracle's L-BFGS (two-loop recursion, backtracking Armijo).

A one-dimensional quadratic is solved exactly by the second (secant) step;
on a strictly convex quadratic the loss decreases monotonically and the
iterates approach the closed-form minimiser (numpy solve); on noise-free
tomography data with more measurements than unknowns the relative residual
goes to zero (below 1e-3 within 150 iterations here).
"""
import numpy as np

import oracle
from oracle.lbfgs import LBFGS, OK
from paper_2504_16446_gb300 import synth
from conftest import oracle_geometry


def test_one_dimensional_quadratic_exact_secant_step():
    fg = lambda x: (float((x[0] - 3.0) ** 2), np.array([2.0 * (x[0] - 3.0)]))
    opt = LBFGS(fg, [0.0])
    f1, n1, st1 = opt.step()
    assert st1 == OK and n1 == 1 and abs(opt.x[0] - 1.0) < 1e-15   # unit first step
    f2, n2, st2 = opt.step()
    assert st2 == OK and abs(opt.x[0] - 3.0) < 1e-14 and f2 < 1e-28


def test_convex_quadratic_monotone_and_converges():
    rng = np.random.default_rng(0)
    n = 30
    Q = rng.normal(size=(n, n)); A = Q @ Q.T + 0.5 * np.eye(n)
    bvec = rng.normal(size=n)
    fg = lambda x: (0.5 * x @ A @ x - bvec @ x, A @ x - bvec)
    opt = LBFGS(fg, np.zeros(n), m=10)
    prev = opt.f
    for _ in range(300):
        if np.linalg.norm(opt.g) < 1e-6:   # below this f changes at rounding level
            break
        f, _, status = opt.step()
        assert status == OK
        assert f <= prev
        prev = f
    # |x - x*| <= |g| / lambda_min(A) with lambda_min >= 0.5
    np.testing.assert_allclose(opt.x, np.linalg.solve(A, bvec), atol=3e-6)


def test_noise_free_tomography_residual_goes_to_zero():
    st = synth.small_setup(n=(5, 5, 5), nj=9, nk=9, ell_max=2, n_proj=12, n_seg=8, seed=7, offsets=False)
    g = oracle_geometry(st)
    B = oracle.basis_matrix(g)
    truth = synth.random_volume(st, 1)
    I = oracle.forward(g, truth, B)
    fg = lambda x: oracle.gradient_residual(g, x.reshape(st.volume_shape), I, None, B)
    opt = LBFGS(fg, np.zeros(truth.size))
    f0 = prev = opt.f
    for _ in range(150):
        f, _, status = opt.step()
        assert status == OK and f <= prev
        prev = f
    assert np.sqrt(opt.f / f0) < 1e-3
