"""SIRT-style preconditioned gradient descent with Nesterov momentum (MITRA), FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section "Standard reconstruction pipelines": SIRT is a preconditioned
gradient descent on a weighted least-squares loss (Gregor & Fessler, IEEE
Trans. Image Process. 24, 2015); applying the same row/column weighting to
the full model A = (B_s (x) P_s) of Eq. (projection_matrix) and Eq.
(projection_operator) gives the MITRA solver, which adds Nesterov momentum.

Readings (the paper gives no formulas for this solver):

  * A has entries of both signs (spherical harmonics), so the weights are
    built from |A|.  Because every John-transform coefficient P_s is >= 0,
    |A| = |B_s| (x) P_s and
        rho[s,j,k,c] = (sum_i |B_s[c,i]|) (P_s 1)[j,k]          (|A| 1)
        kappa[v,i]   = sum_s (sum_c |B_s[c,i]|) (P_s^T 1)[v]    (|A|^T 1)
  * data weights R = W / rho where the ray's length in the volume
    (P_s 1)[j,k] exceeds 1e-6 a, else 0; preconditioner D = 1 / kappa where
    kappa > 1e-6 a Y00 (Y00 = 1 / (2 sqrt(pi))), else 0 (voxels and channels
    that no ray sees keep their start value).
  * Cauchy-Schwarz (the Schur test) gives ||R^1/2 A D^1/2||_2 <= sqrt(max W),
    so with W <= 1 the step below is stable for 0 < eta < 2.
  * iteration t = 1, 2, ...:
        y_t     = x_t + mu_t (x_t - x_{t-1})            (x_0 = x_1 = c0)
        x_{t+1} = y_t - (eta / 2) D grad L_R(y_t),  L_R(c) = sum R (A c - I)^2
    i.e. x_{t+1} = y_t + eta D A^T R (I - A y_t), which for eta = 1 and
    mu = 0 is the classical SIRT update.  mu_t = (t - 1) / (t + 2)
    (Nesterov 1983; Beck & Teboulle 2009) when momentum < 0, else the
    constant momentum.
"""
from __future__ import annotations

import numpy as np

from . import basis_matrix, gradient_residual, john_adjoint, john_forward

Y00 = 0.5 / np.sqrt(np.pi)


def sirt_weights(g, W=None, B=None):
    """(R, D): SIRT data weights [S,nj,nk,C] and preconditioner [nx,ny,nz,K]."""
    B = basis_matrix(g) if B is None else np.asarray(B, dtype=np.float64)
    absB = np.abs(B)
    row_abs = absB.sum(axis=2)                          # [S, C]
    col_abs = absB.sum(axis=1)                          # [S, K]
    ray_len = john_forward(g, np.ones(g.shape + (1,)))[..., 0]            # P_s 1, [S, nj, nk]
    rho = ray_len[..., None] * row_abs[:, None, None, :]
    R = np.zeros(g.data_shape)
    hit = np.broadcast_to((ray_len > 1e-6 * g.a)[..., None], R.shape)
    Wf = np.ones(g.data_shape) if W is None else np.asarray(W, dtype=np.float64)
    R[hit] = Wf[hit] / rho[hit]
    per_proj = np.broadcast_to(col_abs[:, None, None, :], (g.S, g.nj, g.nk, g.K))
    kappa = john_adjoint(g, per_proj)                   # sum_s col_abs[s] P_s^T 1
    D = np.zeros(g.volume_shape)
    seen = kappa > 1e-6 * g.a * Y00
    D[seen] = 1.0 / kappa[seen]
    return R, D


class MITRA:
    """Preconditioned gradient descent with Nesterov momentum on L_R."""

    def __init__(self, g, c0, I, W=None, eta: float = 1.0, momentum: float = -1.0, B=None):
        self.g = g
        self.B = basis_matrix(g) if B is None else B
        self.R, self.D = sirt_weights(g, W, self.B)
        self.I = np.asarray(I, dtype=np.float64)
        self.eta, self.momentum = float(eta), float(momentum)
        self.x = np.array(c0, dtype=np.float64, copy=True)
        self.x_prev = self.x.copy()
        self.t = 0

    def mu(self, t: int) -> float:
        return (t - 1.0) / (t + 2.0) if self.momentum < 0 else self.momentum

    def step(self) -> float:
        """One iteration; returns L_R at the extrapolated point y_t."""
        self.t += 1
        y = self.x + self.mu(self.t) * (self.x - self.x_prev)
        loss, grad = gradient_residual(self.g, y, self.I, self.R, self.B)
        self.x_prev = self.x
        self.x = y - 0.5 * self.eta * self.D * grad
        return loss
