"""Unbounded two-loop L-BFGS with backtracking Armijo line search (FP64, numpy).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper solves the least-squares problem of Eq. (opt_prob_general_form)
with an L-BFGS optimizer (Section "Optimization").  It names no memory size,
line search or bounds; the spherical-harmonic coefficients may take either
sign, so bounds are inactive and the unbounded method is used.  The steps are
those of the published two-loop recursion (Nocedal & Wright, Numerical
Optimization, 2nd ed., Algorithm 7.4 with Eq. 7.20 for H_0):

  direction   q = g; for i newest..oldest: a_i = rho_i s_i.q, q -= a_i y_i
              r = gamma q, gamma = s.y / y.y of the newest pair
              for i oldest..newest: b = rho_i y_i.r, r += (a_i - b) s_i
              d = -r
  first step  with no stored pair, d = -g and the trial step is 1/|g|
  safeguard   if g.d >= 0 the memory is cleared and d = -g
  line search alpha halves until f(x + alpha d) <= f(x) + c1 alpha g.d,
              c1 = 1e-4, at most 20 evaluations
  update      s = x_new - x, y = g_new - g; the pair is kept only when
              s.y > 1e-10 |s| |y|; at most m pairs (oldest dropped)
"""
from __future__ import annotations

import numpy as np

OK = 0
LINESEARCH_FAILED = 5


class LBFGS:
    def __init__(self, fg, x0, m: int = 10, c1: float = 1e-4, max_evals: int = 20):
        self.fg = fg
        self.m, self.c1, self.max_evals = int(m), float(c1), int(max_evals)
        self.x = np.array(x0, dtype=np.float64, copy=True).ravel()
        f, g = fg(self.x)
        self.f = float(f)
        self.g = np.asarray(g, dtype=np.float64).ravel().copy()
        self.S: list[np.ndarray] = []
        self.Y: list[np.ndarray] = []
        self.rho: list[float] = []
        self.n_iter = 0
        self.total_evals = 1

    def direction(self):
        g = self.g
        if not self.S:
            return -g, 1.0 / np.linalg.norm(g)
        q = g.copy()
        alphas = []
        for s, y, rho in zip(reversed(self.S), reversed(self.Y), reversed(self.rho)):
            a = rho * float(s @ q)
            q -= a * y
            alphas.append(a)
        alphas.reverse()
        s_new, y_new = self.S[-1], self.Y[-1]
        gamma = float(s_new @ y_new) / float(y_new @ y_new)
        r = gamma * q
        for s, y, rho, a in zip(self.S, self.Y, self.rho, alphas):
            b = rho * float(y @ r)
            r += (a - b) * s
        return -r, 1.0

    def step(self):
        """One iteration.  Returns (loss, n_evals, status)."""
        d, alpha = self.direction()
        gd = float(self.g @ d)
        if gd >= 0.0:
            self.S.clear(); self.Y.clear(); self.rho.clear()
            d = -self.g
            alpha = 1.0 / np.linalg.norm(self.g)
            gd = float(self.g @ d)
        for n in range(1, self.max_evals + 1):
            x_t = self.x + alpha * d
            f_t, g_t = self.fg(x_t)
            f_t = float(f_t)
            if f_t <= self.f + self.c1 * alpha * gd:
                g_t = np.asarray(g_t, dtype=np.float64).ravel()
                s = x_t - self.x
                y = g_t - self.g
                sy = float(s @ y)
                if sy > 1e-10 * np.linalg.norm(s) * np.linalg.norm(y):
                    self.S.append(s); self.Y.append(y); self.rho.append(1.0 / sy)
                    if len(self.S) > self.m:
                        self.S.pop(0); self.Y.pop(0); self.rho.pop(0)
                self.x, self.f, self.g = x_t, f_t, g_t.copy()
                self.n_iter += 1
                self.total_evals += n
                return self.f, n, OK
            alpha *= 0.5
        self.total_evals += self.max_evals
        return self.f, self.max_evals, LINESEARCH_FAILED
