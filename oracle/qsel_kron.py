"""CPU FP64 reference of the Kronecker preconditioner for grid meshes (test
infrastructure only).

The paper's sampler solves Q x = r by PCG with block-Jacobi or IC(0)
(Section 3.3).  On an m x m grid mesh with unit spacing (the P1 stiffness and
lumped mass of the meshes used here) the prior part of Q factors through
one-dimensional operators:

    G = T (x) D + D (x) T,     C ~= D (x) D,

with T the 1-D Neumann stiffness (1, 2, ..., 2, 1 on the diagonal, -1 off it)
and D = diag(1/2, 1, ..., 1, 1/2), node index i m + j; C equals D (x) D except
at the four corners, whose lumped masses depend on the triangulation.  With
C~ = D (x) D the spatial precision Q~_s = K~ C~^-1 K~, K~ = kappa^2 C~ + G, is

    Q~_s = (D^1/2 (x) D^1/2) S^2 (D^1/2 (x) D^1/2),
    S = kappa^2 I + T^ (x) I + I (x) T^,   T^ = D^-1/2 T D^-1/2 = V diag(lambda) V^T.

The observation term A^T A / sigma^2 (a random subset of nodes) is replaced
by its mean omega C~, omega = (observed fraction) / sigma^2, so that with
Q_t = U diag(mu) U^T the whole preconditioner is diagonal in one basis:

    M = (I (x) D^1/2 (x) D^1/2) [tau Q_t (x) S^2 + omega I] (I (x) D^1/2 (x) D^1/2),
    M^-1 = (I (x) Dh (x) Dh) (U (x) V (x) V) diag(1 / (tau mu_k (kappa^2 +
           lambda_a + lambda_b)^2 + omega)) (U (x) V (x) V)^T (I (x) Dh (x) Dh),

Dh = D^-1/2, index order (t, i, j).  With omega = 0 it is the prior
precision with C~ in place of C.
"""
from __future__ import annotations

import math

import numpy as np

from . import qsel_oracle as o


def neumann_1d(m: int):
    """(T, D) of the 1-D Neumann stiffness and lumped mass, unit spacing."""
    T = 2.0 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)
    T[0, 0] = T[-1, -1] = 1.0
    d = np.ones(m)
    d[0] = d[-1] = 0.5
    return T, np.diag(d)


def grid_factors(m: int):
    """(lambda, V, dh): T^ = V diag(lambda) V^T and dh = diag(D)^-1/2."""
    T, D = neumann_1d(m)
    dh = 1.0 / np.sqrt(np.diag(D))
    lam, V = np.linalg.eigh(dh[:, None] * T * dh[None, :])
    return lam, V, dh


def spatial_inverse(m: int, kappa: float) -> np.ndarray:
    """Dense Q~_s^-1 by the formula above."""
    lam, V, dh = grid_factors(m)
    W = np.kron(V, V)
    s = 1.0 / (kappa ** 2 + lam[:, None] + lam[None, :]) ** 2
    Dh = np.kron(dh, dh)
    return Dh[:, None] * (W @ np.diag(s.ravel()) @ W.T) * Dh[None, :]


def temporal_inverse(rho: float, n_t: int) -> np.ndarray:
    """Q_t^-1 = (1 - rho^2) B^-1 B^-T."""
    Binv = np.linalg.inv(o.ar1_B(rho, n_t))
    return (1.0 - rho ** 2) * Binv @ Binv.T


def omega(model: o.Model) -> float:
    """Mean observation weight: observed fraction / sigma^2."""
    return float(np.count_nonzero(model.obs_mask)) / model.n / model.sigma ** 2


def preconditioner_inverse(model: o.Model, theta, om=None) -> np.ndarray:
    """Dense M^-1 (formula above) for an m x m grid model; om defaults to
    omega(model)."""
    m = int(round(math.sqrt(model.n_s)))
    assert m * m == model.n_s
    kappa, tau, rho = o.theta_to_natural(theta)
    om = omega(model) if om is None else om
    lam, V, dh = grid_factors(m)
    mu, U = np.linalg.eigh(o.temporal_precision(rho, model.n_t))
    S2 = (kappa ** 2 + lam[:, None] + lam[None, :]) ** 2
    diag = 1.0 / (tau * mu[:, None, None] * S2[None, :, :] + om)
    W = np.kron(U, np.kron(V, V))
    Dh = np.kron(np.ones(model.n_t), np.kron(dh, dh))
    return Dh[:, None] * (W @ np.diag(diag.ravel()) @ W.T) * Dh[None, :]
