"""Pins for the oracle's L-BFGS (two-loop recursion, backtracking Armijo).

A one-dimensional quadratic is solved exactly by the second (secant) step;
on a strictly convex quadratic the loss decreases monotonically and the
iterates approach the closed-form minimiser (numpy solve); on noise-free
tomography data with more measurements than unknowns the relative residual
goes to zero (below 1e-3 within 150 iterations here).  The safeguard
branches (curvature skip and its threshold, the non-descent restart, the
Armijo constant, halving and the 20-evaluation limit) are pinned by scripted
objectives whose accepted iterates follow from the rules by hand.
"""
import numpy as np
import pytest

import oracle
from oracle.lbfgs import LBFGS, LINESEARCH_FAILED, OK
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


# ---------------------------------------------------------------------------
# Safeguard branches.  The objectives below are scripted callables (values and
# gradients chosen by hand, not necessarily those of one smooth function):
# each forces one branch of the iteration and the expected iterate follows
# from the rule by hand.

def test_pair_with_nonpositive_curvature_is_not_stored():
    """s.y <= 0 (here s.y = -1): the pair is dropped, and the next step is
    the restart rule's steepest descent with trial step 1/|g|."""
    g0, g1 = np.array([-1.0, 0.0]), np.array([-2.0, -1.0])
    def fg(x):
        if np.allclose(x, [0.0, 0.0]):
            return 0.0, g0
        if np.allclose(x, [1.0, 0.0]):
            return -10.0, g1          # accepted; y = g1 - g0 = (-1, -1), s = (1, 0): s.y = -1
        return -100.0, np.zeros(2)
    opt = LBFGS(fg, [0.0, 0.0])
    opt.step()
    np.testing.assert_array_equal(opt.x, [1.0, 0.0])
    assert opt.S == [] and opt.Y == [] and opt.rho == []
    opt.step()
    np.testing.assert_allclose(opt.x, np.array([1.0, 0.0]) - g1 / np.linalg.norm(g1), rtol=0, atol=1e-15)


@pytest.mark.parametrize("eps,kept", [(-1.0, False), (0.0, False), (0.5e-10, False), (2e-10, True), (1e-6, True)])
def test_curvature_threshold_is_1e_10_of_s_times_y(eps, kept):
    """The pair is kept exactly when s.y > 1e-10 |s| |y|: s = (1, 0),
    y = (eps, 1), so s.y / (|s| |y|) = eps / sqrt(1 + eps^2)."""
    g0 = np.array([-1.0, 0.0])
    y = np.array([eps, 1.0])
    def fg(x):
        if np.allclose(x, [0.0, 0.0]):
            return 0.0, g0
        return -10.0, g0 + y
    opt = LBFGS(fg, [0.0, 0.0])
    _, n, status = opt.step()
    assert status == OK and n == 1
    np.testing.assert_array_equal(opt.x, [1.0, 0.0])
    assert len(opt.S) == (1 if kept else 0)
    if kept:
        np.testing.assert_array_equal(opt.S[0], [1.0, 0.0])
        # y comes back as (g0 + y) - g0, exact up to the rounding of g0 + y
        np.testing.assert_allclose(opt.Y[0], y, rtol=1e-6, atol=0)
        np.testing.assert_allclose(opt.rho[0], 1.0 / float(opt.S[0] @ opt.Y[0]), rtol=1e-15)


def test_non_descent_direction_clears_memory_and_restarts_along_minus_g():
    """A stored pair with negative rho (set by hand: the update never stores
    one) makes the two-loop direction an ascent direction; the iteration must
    clear the memory and take the first-iteration step -g/|g|."""
    fg = lambda x: (0.5 * float(x @ x), x.copy())
    x0 = np.array([3.0, 4.0])
    opt = LBFGS(fg, x0)
    opt.S, opt.Y, opt.rho = [np.array([1.0, 0.0])], [np.array([-1.0, 0.0])], [-1.0]
    d, alpha = opt.direction()
    assert float(opt.g @ d) > 0            # the stored pair gives an ascent direction
    _, n, status = opt.step()
    assert status == OK and n == 1
    # x0 - x0/|x0| = (3, 4) * (1 - 1/5); the new pair (s, y) = (-x0/5, -x0/5) is the only one stored
    np.testing.assert_allclose(opt.x, x0 * 0.8, rtol=0, atol=1e-15)
    assert len(opt.S) == 1
    np.testing.assert_allclose(opt.S[0], -x0 / 5, rtol=0, atol=1e-15)


def _quadratic_with_secant_scale(kappa):
    """f(x) = x^2/2 in 1-D from x = 1 with one stored pair (s, y) = (kappa, 1):
    the two-loop direction is d = -kappa g and the first trial step is 1."""
    fg = lambda x: (0.5 * float(x @ x), x.copy())
    opt = LBFGS(fg, [1.0])
    opt.S, opt.Y, opt.rho = [np.array([float(kappa)])], [np.array([1.0])], [1.0 / kappa]
    return opt


def test_armijo_backtracking_halves_until_sufficient_decrease():
    """Along d = -kappa g on x^2/2, f(x + alpha d) <= f(x) + c1 alpha g.d holds
    iff alpha kappa <= 2 (1 - c1).  kappa = 1000: the first accepted step is
    2^-9 (alpha kappa = 1.953), the 10th evaluation."""
    opt = _quadratic_with_secant_scale(1000.0)
    _, n, status = opt.step()
    assert status == OK and n == 10
    np.testing.assert_allclose(opt.x, [1.0 - 1000.0 / 512.0], rtol=0, atol=1e-15)


@pytest.mark.parametrize("margin,accepted", [(1.5e-4, False), (2.5e-4, True)])
def test_armijo_constant_is_1e_4(margin, accepted):
    """With alpha kappa = 2 - margin at the first trial (alpha = 1), Armijo
    with c1 = 1e-4 needs margin >= 2e-4: 1.5e-4 is rejected (the step halves),
    2.5e-4 is accepted.  This pins c1 to (0.75e-4, 1.25e-4)."""
    kappa = 2.0 - margin
    opt = _quadratic_with_secant_scale(kappa)
    _, n, status = opt.step()
    assert status == OK
    if accepted:
        assert n == 1
        np.testing.assert_allclose(opt.x, [1.0 - kappa], rtol=0, atol=1e-15)
    else:
        assert n == 2
        np.testing.assert_allclose(opt.x, [1.0 - kappa / 2.0], rtol=0, atol=1e-15)


def test_line_search_gives_up_after_20_evaluations_and_keeps_the_iterate():
    """kappa = 2^20: alpha kappa > 2 for alpha = 1 .. 2^-19 (20 trials), so the
    search fails with status 5 and the iterate, loss, gradient and memory are
    unchanged; kappa = 1.9 * 2^19 is accepted on exactly the 20th trial."""
    opt = _quadratic_with_secant_scale(2.0 ** 20)
    S0 = list(opt.S)
    x0, f0, g0 = opt.x.copy(), opt.f, opt.g.copy()
    evals0 = opt.total_evals
    f, n, status = opt.step()
    assert status == LINESEARCH_FAILED and n == 20
    np.testing.assert_array_equal(opt.x, x0)
    np.testing.assert_array_equal(opt.g, g0)
    assert f == f0 == opt.f and opt.n_iter == 0 and opt.total_evals == evals0 + 20
    assert opt.S == S0
    opt = _quadratic_with_secant_scale(1.9 * 2.0 ** 19)
    _, n, status = opt.step()
    assert status == OK and n == 20
    np.testing.assert_allclose(opt.x, [1.0 - 1.9], rtol=0, atol=1e-15)
