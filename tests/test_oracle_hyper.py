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
