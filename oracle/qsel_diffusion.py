"""CPU FP64 oracle of the diffusion-based non-separable space-time model and of
overlapping RBMC on an arbitrary block-tridiagonal precision.

TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the CUDA library; plain numpy/scipy in FP64.

The model (Section 2.2, Eqs. spde:5-8) for the "critical diffusion" case
(alpha_t, alpha_s, alpha_e) = (1, 2, 1): the precision is the sum of
Kronecker products

    Q_u = gamma_e^2 sum_{k=0}^{2} gamma_t^k J(1, k/2) (x) K(2 (1 - k/2) + 1)
        = gamma_e^2 [ J0 (x) K3 + gamma_t J1 (x) K2 + gamma_t^2 J2 (x) K1 ],

with the spatial precisions of Eq. spde:4 (tau = 1) for the lumped mass C and
stiffness G, K(a) = C^1/2 (gamma_s^2 I + C^-1/2 G C^-1/2)^a C^1/2, i.e.

    K1 = gamma_s^2 C + G,  K2 = K1 C^-1 K1,  K3 = K2 C^-1 K1,

and the posterior precision Q = Q_u + A^T A / sigma^2 (Section 2.3).

Readings where the paper is silent (listed in the design notes): the J
matrices come from the temporal finite-element discretisation with unit
spacing and lumped mass -- J0 = M0 = diag(1/2, 1, ..., 1, 1/2) (mass),
J1 = 2 M1 with M1 = diag(1/2, 0, ..., 0, 1/2) (boundary term), J2 = M2 the
Neumann stiffness (diagonal 1, 2, ..., 2, 1, off-diagonals -1); the
hyperparameters are theta = (log gamma_s, log gamma_t, log gamma_e).  Every
term is positive semi-definite and J0 (x) K3 is positive definite, so Q is
positive definite; Q is block tridiagonal in time because every J is.

Derivatives: d/dlog gamma_e doubles Q_u; d/dlog gamma_t multiplies the k-th
term by k; d/dlog gamma_s uses dK(a)/dlog gamma_s = 2 gamma_s^2 a K(a - 1)
with K(0) = C.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from oracle import qsel_oracle as o


def theta_to_natural(theta):
    """theta = (log gamma_s, log gamma_t, log gamma_e) -> (gamma_s, gamma_t, gamma_e)."""
    return math.exp(theta[0]), math.exp(theta[1]), math.exp(theta[2])


def temporal_matrices(n_t: int):
    """(M0, M1, M2): lumped temporal mass, boundary term and Neumann stiffness
    of piecewise-linear elements of unit length."""
    M0 = np.eye(n_t)
    M0[0, 0] = M0[-1, -1] = 0.5
    M1 = np.zeros((n_t, n_t))
    M1[0, 0] = M1[-1, -1] = 0.5
    M2 = np.zeros((n_t, n_t))
    for t in range(n_t - 1):
        M2[t, t] += 1.0
        M2[t + 1, t + 1] += 1.0
        M2[t, t + 1] = M2[t + 1, t] = -1.0
    if n_t == 1:
        M0[0, 0] = 1.0
        M1[0, 0] = 1.0
    return M0, M1, M2


def spatial_powers(model: o.Model, gamma_s: float):
    """[K(0), K(1), K(2), K(3)] = [C, K1, K1 C^-1 K1, K1 C^-1 K1 C^-1 K1]."""
    C = sp.diags(model.c_diag).tocsr()
    Ci = sp.diags(1.0 / model.c_diag)
    K1 = (gamma_s ** 2 * C + model.G).tocsr()
    K2 = (K1 @ Ci @ K1).tocsr()
    K3 = (K2 @ Ci @ K1).tocsr()
    return [C, K1, K2, K3]


def _terms(model: o.Model, theta):
    """The three Kronecker terms (J, K-index, power of gamma_t) of Eq. spde:8."""
    M0, M1, M2 = temporal_matrices(model.n_t)
    return [(M0, 3, 0), (2.0 * M1, 2, 1), (M2, 1, 2)]


def prior_precision(model: o.Model, theta) -> sp.csr_matrix:
    """Q_u of Eq. spde:8 for (alpha_t, alpha_s, alpha_e) = (1, 2, 1)."""
    gs, gt, ge = theta_to_natural(theta)
    K = spatial_powers(model, gs)
    Q = None
    for J, a, p in _terms(model, theta):
        term = (ge ** 2 * gt ** p) * sp.kron(sp.csr_matrix(J), K[a])
        Q = term if Q is None else Q + term
    return Q.tocsr()


def precision(model: o.Model, theta) -> sp.csr_matrix:
    """Posterior precision Q = Q_u + A^T A / sigma^2 (Section 2.3)."""
    return (prior_precision(model, theta) + o.obs_precision(model)).tocsr()


def precision_derivatives(model: o.Model, theta) -> list:
    """[dQ/dlog gamma_s, dQ/dlog gamma_t, dQ/dlog gamma_e]."""
    gs, gt, ge = theta_to_natural(theta)
    K = spatial_powers(model, gs)
    d_s = d_t = None
    for J, a, p in _terms(model, theta):
        Jc = sp.csr_matrix(J)
        # dK(a)/dlog gamma_s = 2 gamma_s^2 a K(a - 1)
        ts = (ge ** 2 * gt ** p * 2.0 * gs ** 2 * a) * sp.kron(Jc, K[a - 1])
        tt = (ge ** 2 * p * gt ** p) * sp.kron(Jc, K[a])
        d_s = ts if d_s is None else d_s + ts
        d_t = tt if d_t is None else d_t + tt
    d_e = 2.0 * prior_precision(model, theta)
    return [d_s.tocsr(), d_t.tocsr(), d_e.tocsr()]


# ----------------------------------------------------------------------------
# Overlapping RBMC (Algorithm 4) and the trace estimator (Eq. hyperpar:4) on a
# given block-tridiagonal precision with n_s x n_s blocks
# ----------------------------------------------------------------------------


def rbmc_precision(Q, dQs, n_s: int, n_t: int, slab_start, n_l, X: np.ndarray):
    """Algorithm 4 on the precision Q (sparse, block tridiagonal in time) with
    the derivatives dQs, given global samples X (n x k): the same subdomain
    steps as the separable model's oracle.  Returns (v_hat, t_hat, results)."""
    k = X.shape[1]
    parts = o.partition(n_t, slab_start, n_l)
    v = np.zeros(n_s * n_t)
    t_hat = np.zeros(len(dQs))
    results = []
    for part in parts:
        X_sep = {s: X[s * n_s:(s + 1) * n_s, :] for s in part.sep}
        res = o.subdomain_estimate(Q, dQs, n_s, part, X_sep, k)
        s0, s1 = part.own
        v[s0 * n_s:s1 * n_s] = res.sigma_star_diag + res.corr_diag
        t_hat += res.traces
        results.append(res)
    return v, t_hat, results


def blocks(Q, n_s: int, n_t: int):
    """(diagonal blocks [n_t], coupling blocks Q[t+1, t] [n_t - 1]) as dense arrays."""
    return ([o.block(Q, n_s, t, t) for t in range(n_t)], [o.block(Q, n_s, t + 1, t) for t in range(n_t - 1)])
