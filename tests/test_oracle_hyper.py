"""Pins of the posterior-mean and hyperparameter-gradient reference
(oracle/qsel_hyper.py) against forms that do not share its route: the
Kalman (data-space) form of the posterior mean, the Gaussian density of the
data under its marginal covariance, finite differences of that density and
of the numerical log-determinant of the prior."""
import math

import numpy as np

import qsel_inputs as qi
from oracle import qsel_hyper as h
from oracle import qsel_oracle as o
from tests.models import grid_model, theta


def _setup(m=4, n_t=3, obs_frac=0.4):
    mdl = grid_model(m, n_t, obs_frac=obs_frac)
    th = theta(0.7, 1.3, 0.6)
    y = qi.seeded_normal((int(np.count_nonzero(mdl.obs_mask)), 1), 5)[:, 0]
    return mdl, th, y


def _data_covariance(mdl, th):
    """sigma^2 I + A Q_x^-1 A^T (dense)."""
    obs = np.flatnonzero(mdl.obs_mask)
    Sx = np.linalg.inv(h.prior_precision(mdl, th).toarray())
    return mdl.sigma ** 2 * np.eye(len(obs)) + Sx[np.ix_(obs, obs)], Sx, obs


def test_posterior_mean_matches_the_kalman_form():
    mdl, th, y = _setup()
    Syy, Sx, obs = _data_covariance(mdl, th)
    mu_kalman = Sx[:, obs] @ np.linalg.solve(Syy, y)
    np.testing.assert_allclose(h.posterior_mean(mdl, th, y), mu_kalman, rtol=1e-9, atol=1e-12)


def test_log_marginal_is_the_gaussian_density_of_the_data():
    mdl, th, y = _setup()
    Syy, _, _ = _data_covariance(mdl, th)
    sign, ld = np.linalg.slogdet(Syy)
    direct = -0.5 * (ld + y @ np.linalg.solve(Syy, y) + len(y) * math.log(2.0 * math.pi))
    assert sign > 0
    assert abs(h.log_marginal(mdl, th, y) - direct) < 1e-9 * max(1.0, abs(direct))


def test_gradient_matches_finite_differences():
    mdl, th, y = _setup(5, 4)
    g = h.loglik_grad(mdl, th, y)
    step = 1e-5
    for j in range(3):
        tp = list(th)
        tm = list(th)
        tp[j] += step
        tm[j] -= step
        fd = (h.log_marginal(mdl, tp, y) - h.log_marginal(mdl, tm, y)) / (2 * step)
        assert abs(g[j] - fd) < 1e-5 * max(1.0, abs(fd)), (j, g[j], fd)


def test_prior_logdet_gradient_closed_forms():
    """d log|Q_x| / d theta against finite differences of the numerical
    log-determinant; with one slab the temporal term vanishes."""
    for n_t in (1, 4):
        mdl, th, _ = _setup(4, n_t)
        g = h.prior_logdet_grad(mdl, th)
        step = 1e-5
        for j in range(3):
            tp = list(th)
            tm = list(th)
            tp[j] += step
            tm[j] -= step
            fd = (o.logdet(h.prior_precision(mdl, tp), mdl.n_s, n_t)
                  - o.logdet(h.prior_precision(mdl, tm), mdl.n_s, n_t)) / (2 * step)
            assert abs(g[j] - fd) < 1e-6 * max(1.0, abs(fd)), (n_t, j, g[j], fd)
        if n_t == 1:
            assert g[2] == 0.0
        assert g[1] == mdl.n


# ---------------------------------------------------------------- fixed effects
def _setup_fe(m=4, n_t=3, n_beta=3):
    mdl, th, y = _setup(m, n_t)
    Z = qi.seeded_normal((len(y), n_beta), 8)
    return mdl, th, y, Z, 0.5


def _joint_covariance(mdl, th, Z, beta_prec):
    """Data covariance with beta integrated out: sigma^2 I + A Q_x^-1 A^T + Z Z^T / beta_prec."""
    Syy, Sx, obs = _data_covariance(mdl, th)
    return Syy + Z @ Z.T / beta_prec, Sx, obs


def test_fixed_effects_mean_and_variances_match_the_joint_gaussian():
    """mu_u, mu_beta by the Kalman form of the joint prior (u, beta); Var(beta)
    and diag Var(u) (Eq. var:1) from the dense joint posterior covariance."""
    mdl, th, y, Z, bp = _setup_fe()
    C, Sx, obs = _joint_covariance(mdl, th, Z, bp)
    a = np.linalg.solve(C, y)
    mu_u_k = Sx[:, obs] @ a
    mu_b_k = Z.T @ a / bp
    mu_u, mu_b, Sinv, corr, _ = h.fixed_effects(mdl, th, y, Z, bp)
    np.testing.assert_allclose(mu_u, mu_u_k, rtol=1e-8, atol=1e-11)
    np.testing.assert_allclose(mu_b, mu_b_k, rtol=1e-8, atol=1e-11)
    # joint posterior precision, dense
    n, nb = mdl.n, Z.shape[1]
    J = np.zeros((n + nb, n + nb))
    J[:n, :n] = o.precision(mdl, th).toarray()
    J[obs, n:] = Z / mdl.sigma ** 2
    J[n:, obs] = Z.T / mdl.sigma ** 2
    J[n:, n:] = bp * np.eye(nb) + Z.T @ Z / mdl.sigma ** 2
    Jinv = np.linalg.inv(J)
    np.testing.assert_allclose(Sinv, Jinv[n:, n:], rtol=1e-8, atol=1e-12)
    Quu_inv = np.linalg.inv(J[:n, :n])
    np.testing.assert_allclose(np.diag(Quu_inv) + corr, np.diag(Jinv)[:n], rtol=1e-8, atol=1e-12)


def test_fixed_effects_log_marginal_and_gradient():
    mdl, th, y, Z, bp = _setup_fe(5, 4)
    C, _, _ = _joint_covariance(mdl, th, Z, bp)
    sign, ld = np.linalg.slogdet(C)
    direct = -0.5 * (ld + y @ np.linalg.solve(C, y) + len(y) * math.log(2.0 * math.pi))
    assert sign > 0
    assert abs(h.log_marginal_fe(mdl, th, y, Z, bp) - direct) < 1e-9 * max(1.0, abs(direct))
    g = h.loglik_grad_fe(mdl, th, y, Z, bp)
    step = 1e-5
    for j in range(3):
        tp, tm = list(th), list(th)
        tp[j] += step
        tm[j] -= step
        fd = (h.log_marginal_fe(mdl, tp, y, Z, bp) - h.log_marginal_fe(mdl, tm, y, Z, bp)) / (2 * step)
        assert abs(g[j] - fd) < 1e-5 * max(1.0, abs(fd)), (j, g[j], fd)
