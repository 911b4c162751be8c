"""Hyperparameter estimation (Section 3.4.1, Algorithm hyperpar:1 with the
update of Eq. hyperpar:2) on top of the library's gradient of the marginal
log p(y | theta) (qsel_loglik_grad: the RBMC traces, the posterior mean's
quadratic forms and the prior's log-determinant derivatives, all on the GPU).

The update theta <- theta - H^-1 grad (ascent, H negative definite) is a
quasi-Newton one, the family Eq. hyperpar:2 names: H starts as the diagonal
of second derivatives, each from two first derivatives (at theta and at
theta + delta e_j, with the context's fixed seed, so that the Monte Carlo
part of both gradients is common and cancels in the difference: the
paper's "stochastic components removed"), and is refined by BFGS updates
from successive gradients (again at common random numbers).  Each step is
scaled down to at most max_step per component; a curvature pair that is not
consistent with a concave marginal is skipped.  A hyperprior enters through
prior_grad(theta).
"""
from __future__ import annotations

import numpy as np

from . import qsel


def optimize_theta(ctx, y_obs, theta0, iters: int = 40, delta: float = 1e-2, max_step: float = 0.5,
                   tol: float = 1e-6, prior_grad=None):
    """Ascend log p(y | theta) (+ log pi(theta)) from theta0.  ctx: a context
    of the model (qsel.qsel_create); y_obs: the data on the observed nodes.
    Returns (theta, history), one dict per iteration (theta, grad, step)."""
    qsel.qsel_set_data(ctx, y_obs)

    def neg_grad(th):
        qsel.qsel_set_theta(ctx, th)
        g = qsel.qsel_loglik_grad(ctx)
        if prior_grad is not None:
            g = g + np.asarray(prior_grad(th), dtype=float)
        return -g

    theta = np.asarray(theta0, dtype=float).copy()
    G = neg_grad(theta)
    # initial inverse Hessian of -log p: the finite-difference diagonal
    d = np.zeros(3)
    for j in range(3):
        tj = theta.copy()
        tj[j] += delta
        d[j] = (neg_grad(tj)[j] - G[j]) / delta
    Hinv = np.diag([1.0 / d[j] if d[j] > 0.0 else max_step / max(abs(G[j]), 1e-300) for j in range(3)])
    history = []
    for _ in range(iters):
        p = -Hinv @ G
        big = np.max(np.abs(p))
        if big > max_step:
            p *= max_step / big
        theta_new = theta + p
        G_new = neg_grad(theta_new)
        yv = G_new - G
        sy = float(p @ yv)
        if sy > 1e-12 * np.linalg.norm(p) * np.linalg.norm(yv):
            r = 1.0 / sy
            eye = np.eye(3)
            Hinv = (eye - r * np.outer(p, yv)) @ Hinv @ (eye - r * np.outer(yv, p)) + r * np.outer(p, p)
        theta, G = theta_new, G_new
        history.append({"theta": theta.copy(), "grad": -G, "step": p})
        if np.max(np.abs(p)) < tol:
            break
    qsel.qsel_set_theta(ctx, theta)
    return theta, history
