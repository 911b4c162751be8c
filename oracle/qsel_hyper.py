"""CPU FP64 reference of the posterior mean and of the gradient of the
hyperparameter marginal (test infrastructure only: imported by tests/ and by
nothing in the product path).

Model without fixed effects (the workloads have none): x | theta ~
N(0, Q_x^-1) with Q_x = tau Q_t (x) Q_s, y | x ~ N(A x, sigma^2 I) on the
observed nodes, Q = Q_x + A^T A / sigma^2.

* Posterior mean (Section 2.3, Eq. mean:5 with n_beta = 0):
      mu = Q^-1 b,   b = A^T Q_y y = A^T y / sigma^2.
* Hyperparameter marginal (Section 3.4, Eq. hyperpar:1, the ratio evaluated
  at x = mu), without the hyperprior pi(theta):
      log p(y | theta) = log N(y; A mu, sigma^2 I) + log N(mu; 0, Q_x^-1)
                         - log N(mu; mu, Q^-1)
                       = 1/2 log|Q_x| - 1/2 log|Q| - |y - A mu|^2 / (2 sigma^2)
                         - 1/2 mu^T Q_x mu - n_obs / 2 log(2 pi sigma^2).
* Its gradient (Section 3.4.2: the log-determinant derivatives through
  traces, Eq. hyperpar:3-4, and the quadratic forms at x = mu, where the
  derivative through mu vanishes because mu maximises the x-dependent part):
      d/dtheta_j = 1/2 tr(Q_x^-1 dQ_x_j) - 1/2 tr(Q^-1 dQ_j) - 1/2 mu^T dQ_x_j mu,
  with dQ_j = dQ_x_j (the likelihood does not depend on theta).
* The prior log-determinant, log|Q_x| = n log tau + n_s log|Q_t| + n_t log|Q_s|
  with log|Q_t| = -(n_t - 1) log(1 - rho^2) (unit-variance AR(1): |B|^2 =
  1 - rho^2) and log|Q_s| = 2 log|K| - log|C|, has the derivatives
      d/dlog kappa = 4 n_t kappa^2 tr(K^-1 C),   d/dlog tau = n,
      d/dlogit rho = n_s 2 rho^2 (n_t - 1) / (1 + rho).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import qsel_oracle as o


def prior_precision(model: o.Model, theta) -> sp.csr_matrix:
    """Q_x = tau Q_t (x) Q_s (Section 2.2)."""
    kappa, tau, rho = o.theta_to_natural(theta)
    Qs = o.spatial_precision(model, kappa)
    Qt = sp.csr_matrix(o.temporal_precision(rho, model.n_t))
    return (tau * sp.kron(Qt, Qs)).tocsr()


def data_rhs(model: o.Model, y_obs: np.ndarray) -> np.ndarray:
    """b = A^T y / sigma^2 (y_obs: the observed nodes in increasing index order)."""
    b = np.zeros(model.n)
    b[np.flatnonzero(model.obs_mask)] = np.asarray(y_obs, dtype=float) / model.sigma ** 2
    return b


def posterior_mean(model: o.Model, theta, y_obs: np.ndarray) -> np.ndarray:
    """mu = Q^-1 A^T y / sigma^2 by a sparse direct solve (Eq. mean:5, n_beta = 0)."""
    Q = o.precision(model, theta).tocsc()
    return spla.spsolve(Q, data_rhs(model, y_obs))


def log_marginal(model: o.Model, theta, y_obs: np.ndarray) -> float:
    """log p(y | theta) by the ratio of Eq. hyperpar:1 at x = mu (formula above);
    log-determinants from the block Cholesky factors."""
    y = np.asarray(y_obs, dtype=float)
    obs = np.flatnonzero(model.obs_mask)
    mu = posterior_mean(model, theta, y)
    Qx = prior_precision(model, theta)
    Q = o.precision(model, theta)
    r = y - mu[obs]
    s2 = model.sigma ** 2
    return float(0.5 * o.logdet(Qx, model.n_s, model.n_t) - 0.5 * o.logdet(Q, model.n_s, model.n_t)
                 - 0.5 * (r @ r) / s2 - 0.5 * mu @ (Qx @ mu) - 0.5 * len(obs) * math.log(2.0 * math.pi * s2))


def prior_logdet_grad(model: o.Model, theta) -> np.ndarray:
    """d log|Q_x| / d theta by the closed forms above (tr(K^-1 C) by a dense solve)."""
    kappa, tau, rho = o.theta_to_natural(theta)
    K = o.spatial_K(model, kappa).toarray()
    tr_KinvC = float(np.trace(np.linalg.solve(K, np.diag(model.c_diag))))
    n_s, n_t = model.n_s, model.n_t
    return np.array([4.0 * n_t * kappa ** 2 * tr_KinvC,
                     float(model.n),
                     n_s * 2.0 * rho ** 2 * (n_t - 1) / (1.0 + rho)])


def quadratic_terms(model: o.Model, theta, mu: np.ndarray) -> np.ndarray:
    """mu^T dQ_x_j mu for j = log kappa, log tau, logit rho."""
    return np.array([float(mu @ (d @ mu)) for d in o.precision_derivatives(model, theta)])


def loglik_grad(model: o.Model, theta, y_obs: np.ndarray, traces=None) -> np.ndarray:
    """Gradient of log p(y | theta) (formula above).  traces: tr(Q^-1 dQ_j)
    (default: exact, from the dense inverse; small problems only)."""
    mu = posterior_mean(model, theta, y_obs)
    if traces is None:
        _, traces = o.exact_selinv(o.precision(model, theta), o.precision_derivatives(model, theta))
    return 0.5 * prior_logdet_grad(model, theta) - 0.5 * np.asarray(traces) - 0.5 * quadratic_terms(model, theta, mu)


# ----------------------------------------------------------------------------
# Fixed effects (Section 2.3, Eqs. mean:4-5 and var:1; Eq. hyperpar:3)
# ----------------------------------------------------------------------------
# y = A_u u + Z beta + eps with beta ~ N(0, I / beta_prec) (Z: n_obs x n_beta).
# Joint precision over (u, beta):
#   Q_uu = Q,  Q_ub = A_u^T Z / sigma^2,  Q_bb = beta_prec I + Z^T Z / sigma^2;
# with W = Q_uu^-1 Q_ub and the Schur complement S = Q_bb - Q_bu W:
#   mu_beta = S^-1 (Z^T y / sigma^2 - Q_bu Q_uu^-1 A_u^T y / sigma^2),
#   mu_u = Q_uu^-1 (A_u^T y / sigma^2) - W mu_beta,          (Eq. mean:5)
#   Var(beta) = S^-1,  diag Var(u) = diag(Q_uu^-1) + diag(W S^-1 W^T),  (Eq. var:1)
#   d log|Q| / d theta_j = tr(Q_uu^-1 dQ_j) + tr(S^-1 W^T dQ_j W),     (Eq. hyperpar:3)
# (dS_j = -Q_bu d(Q_uu^-1) Q_ub = W^T dQ_j W; Q_ub and Q_bb do not depend on theta),
# and the gradient of log p(y | theta) keeps the form above with these.


def fixed_effects(model: o.Model, theta, y_obs, Z, beta_prec):
    """(mu_u, mu_beta, Var(beta), diag(W S^-1 W^T), W) by the formulas above
    (sparse solves with Q_uu)."""
    Z = np.asarray(Z, dtype=float)
    s2 = model.sigma ** 2
    obs = np.flatnonzero(model.obs_mask)
    Q = o.precision(model, theta).tocsc()
    Qub = np.zeros((model.n, Z.shape[1]))
    Qub[obs, :] = Z / s2
    lu = spla.splu(Q)
    W = lu.solve(Qub)
    w0 = lu.solve(data_rhs(model, y_obs))
    S = beta_prec * np.eye(Z.shape[1]) + Z.T @ Z / s2 - Qub.T @ W
    m = Z.T @ np.asarray(y_obs, dtype=float) / s2 - Qub.T @ w0
    Sinv = np.linalg.inv(S)
    mu_b = Sinv @ m
    mu_u = w0 - W @ mu_b
    return mu_u, mu_b, Sinv, np.einsum("ra,ab,rb->r", W, Sinv, W), W


def log_marginal_fe(model: o.Model, theta, y_obs, Z, beta_prec) -> float:
    """log p(y | theta) with the fixed effects integrated out, by the ratio of
    Eq. hyperpar:1 at the joint mode: 1/2 log|Q_x| + n_beta/2 log beta_prec
    - 1/2 log|Q_uu| - 1/2 log|S| - |y - A mu_u - Z mu_beta|^2 / (2 sigma^2)
    - 1/2 mu_u^T Q_x mu_u - beta_prec/2 |mu_beta|^2 - n_obs/2 log(2 pi sigma^2)."""
    y = np.asarray(y_obs, dtype=float)
    Z = np.asarray(Z, dtype=float)
    obs = np.flatnonzero(model.obs_mask)
    mu_u, mu_b, Sinv, _, _ = fixed_effects(model, theta, y, Z, beta_prec)
    Qx = prior_precision(model, theta)
    Q = o.precision(model, theta)
    s2 = model.sigma ** 2
    r = y - mu_u[obs] - Z @ mu_b
    _, ld_Sinv = np.linalg.slogdet(Sinv)
    return float(0.5 * o.logdet(Qx, model.n_s, model.n_t) + 0.5 * Z.shape[1] * math.log(beta_prec)
                 - 0.5 * o.logdet(Q, model.n_s, model.n_t) + 0.5 * ld_Sinv - 0.5 * (r @ r) / s2
                 - 0.5 * mu_u @ (Qx @ mu_u) - 0.5 * beta_prec * (mu_b @ mu_b)
                 - 0.5 * len(obs) * math.log(2.0 * math.pi * s2))


def schur_traces(model: o.Model, theta, W, Sinv) -> np.ndarray:
    """tr(S^-1 W^T dQ_j W) for j = log kappa, log tau, logit rho."""
    return np.array([float(np.sum(Sinv * (W.T @ (d @ W)))) for d in o.precision_derivatives(model, theta)])


def loglik_grad_fe(model: o.Model, theta, y_obs, Z, beta_prec, traces=None) -> np.ndarray:
    """Gradient of log_marginal_fe: 1/2 d log|Q_x| - 1/2 (tr(Q_uu^-1 dQ_j) +
    tr(S^-1 W^T dQ_j W)) - 1/2 mu_u^T dQ_j mu_u (traces: tr(Q_uu^-1 dQ_j),
    default exact)."""
    mu_u, _, Sinv, _, W = fixed_effects(model, theta, y_obs, Z, beta_prec)
    if traces is None:
        _, traces = o.exact_selinv(o.precision(model, theta), o.precision_derivatives(model, theta))
    return (0.5 * prior_logdet_grad(model, theta) - 0.5 * (np.asarray(traces) + schur_traces(model, theta, W, Sinv))
            - 0.5 * quadratic_terms(model, theta, mu_u))
