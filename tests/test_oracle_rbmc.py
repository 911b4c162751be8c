"""Pins of the oracle's overlapping RBMC estimator (Algorithm 4) and trace
estimator (Eq. hyperpar:4) against exact dense results, closed forms, the
AR(1) error law of Section 3.2.3 and finite differences of log|Q| (no GPU)."""
import math

import numpy as np
import pytest

from oracle import qsel_oracle as o
from tests.models import ar1_model, grid_model, theta


def test_partition_balanced_clipped_separators():
    ss = o.balanced_slab_start(10, 3)
    assert list(ss) == [0, 4, 7, 10]
    parts = o.partition(10, ss, 2)
    assert [p.own for p in parts] == [(0, 4), (4, 7), (7, 10)]
    assert [p.ext for p in parts] == [(0, 6), (2, 9), (5, 10)]
    assert [p.sep for p in parts] == [[6], [1, 9], [4]]
    one = o.partition(5, o.balanced_slab_start(5, 1), 1)
    assert one[0].ext == (0, 5) and one[0].sep == []
    p0 = o.partition(8, o.balanced_slab_start(8, 2), 0)
    assert [p.sep for p in p0] == [[4], [3]]


@pytest.mark.parametrize("n_l", [0, 1, 3])
def test_single_subdomain_is_exact(n_l):
    """With one subdomain there is no separator: w = 0 and the estimator is the
    exact selected inverse for any samples."""
    model = grid_model(4, 5)
    th = theta(0.5, 1.0, 0.9)
    X = np.random.default_rng(0).standard_normal((model.n, 3))
    v, t, _ = o.rbmc(model, th, o.balanced_slab_start(5, 1), n_l, X)
    Q = o.precision(model, th)
    v_ex, t_ex = o.exact_selinv(Q, o.precision_derivatives(model, th))
    np.testing.assert_allclose(v, v_ex, rtol=1e-12)
    np.testing.assert_allclose(t, t_ex, rtol=1e-11)


@pytest.mark.parametrize("m,n_t,n_p,n_l", [(4, 6, 2, 1), (3, 9, 3, 1), (4, 7, 3, 2), (3, 8, 4, 0)])
def test_square_root_samples_reproduce_exact_result(m, n_t, n_p, n_l):
    """Law of total variance (Eq. var:2): E[w w^T] = Sigma* Q_{*S} Sigma_SS Q_{S*} Sigma*,
    so Sigma* + E[w w^T] is the exact covariance on Omega*.  Samples
    X = sqrt(n) chol(Q^-1) have (1/n) X_S X_S^T = Sigma_SS exactly for every S,
    so with them the RBMC diagonal equals diag(Q^-1) and, when n_l >= 1, the
    trace estimator equals tr(Q^-1 dQ_j) up to rounding."""
    model = grid_model(m, n_t)
    th = theta(0.6, 1.2, 0.85)
    Q = o.precision(model, th)
    dQs = o.precision_derivatives(model, th)
    S = np.linalg.inv(Q.toarray())
    X = math.sqrt(model.n) * np.linalg.cholesky(0.5 * (S + S.T))
    v, t, res = o.rbmc(model, th, o.balanced_slab_start(n_t, n_p), n_l, X)
    v_ex, t_ex = o.exact_selinv(Q, dQs)
    np.testing.assert_allclose(v, v_ex, rtol=1e-10)
    if n_l >= 1:
        np.testing.assert_allclose(t, t_ex, rtol=1e-9)
    # the correction is genuinely non-zero next to the separators
    assert max(r.corr_diag.max() for r in res) > 1e-3 * v_ex.max()


def test_closed_forms_without_observations():
    """No observations: Q = tau Q_t (x) Q_s, so diag(Q^-1) = diag(Q_s^-1)/tau in
    every slab, tr(Q^-1 dQ/dlog tau) = n, tr(Q^-1 dQ/dlogit rho) =
    n_s 2 rho^2 (n_t - 1)/(1 + rho) and tr(Q^-1 dQ/dlog kappa) =
    n_t 4 kappa^2 tr(K^-1 C) with K = kappa^2 C + G."""
    model = grid_model(4, 6, obs_frac=0.0)
    kappa, tau, rho = 0.7, 1.9, 0.8
    th = theta(kappa, tau, rho)
    Q = o.precision(model, th)
    v, t = o.exact_selinv(Q, o.precision_derivatives(model, th))
    Qs = o.spatial_precision(model, kappa).toarray()
    np.testing.assert_allclose(v, np.tile(np.diag(np.linalg.inv(Qs)) / tau, 6), rtol=1e-11)
    K = o.spatial_K(model, kappa).toarray()
    assert abs(t[0] - 6 * 4 * kappa ** 2 * np.trace(np.linalg.solve(K, np.diag(model.c_diag)))) < 1e-9 * abs(t[0])
    assert abs(t[1] - model.n) < 1e-9 * model.n
    assert abs(t[2] - 16 * 2 * rho ** 2 * 5 / (1 + rho)) < 1e-9 * abs(t[2])


def test_log_tau_trace_closed_form_with_observations():
    """dQ/dlog tau = Q - A^T A/sigma^2, so its trace is n - sigma^-2 sum_obs v_i."""
    model = grid_model(4, 5, obs_frac=0.3, sigma=0.5)
    th = theta(0.5, 1.0, 0.9)
    v, t = o.exact_selinv(o.precision(model, th), o.precision_derivatives(model, th))
    assert abs(t[1] - (model.n - np.sum(v[model.obs_mask == 1]) / 0.25)) < 1e-10 * model.n


@pytest.mark.parametrize("th", [theta(0.5, 1.0, 0.9), theta(0.25, 0.6, 0.95)])
def test_traces_match_logdet_finite_differences(th):
    """d log|Q| / d theta_j = tr(Q^-1 dQ/dtheta_j) (Section 1): central
    differences of the block-Cholesky log-determinant with h = 1e-4."""
    model = grid_model(4, 5)
    _, t = o.exact_selinv(o.precision(model, th), o.precision_derivatives(model, th))
    h = 1e-4
    for j in range(3):
        tp = list(th); tp[j] += h
        tm = list(th); tm[j] -= h
        fd = (o.logdet(o.precision(model, tp), 16, 5) - o.logdet(o.precision(model, tm), 16, 5)) / (2 * h)
        assert abs(fd - t[j]) <= 1e-6 * max(1.0, abs(t[j])), (j, fd, t[j])


def test_ar1_error_law_profile():
    """AR(1) example of Section 3.2.3 (phi = 0.95, 99 nodes, split at node 50):
    conditioning on the separator x_50, w_i = phi^d x_50 at distance d, so
    v_hat_i - 1 = phi^(2d) ((1/k) sum x_50^2 - 1) exactly: the error divided by
    phi^(2d) is the same for every node of the subdomain, and its RMS over seeds
    is the MC error sqrt(2/k).  Relative RMSE at distance d: phi^(2d) sqrt(2/k)."""
    phi, k = 0.95, 8
    model, th = ar1_model(99, phi)
    slab_start = np.array([0, 50, 99])
    ratios = []
    for seed in range(300):
        X = o.samples(model, th, seed, k)
        v, _, _ = o.rbmc(model, th, slab_start, 0, X)
        d = 50 - np.arange(50)
        r = (v[:50] - 1.0) / phi ** (2 * d)
        np.testing.assert_allclose(r, r[0], rtol=1e-8, atol=1e-9)
        ratios.append(r[0])
    rmse = math.sqrt(np.mean(np.square(ratios)))
    # sampling spread of the RMS of a scaled chi^2_k over 300 seeds: ~ 6 %
    assert abs(rmse / math.sqrt(2 / k) - 1) < 0.2, rmse


def test_error_estimate_ar1_closed_form():
    """AR(1) example of Section 3.2.3: w_i = phi^d x_s (separator x_s, distance
    d), so m2_i = phi^(2d) mean(x_s^2) and m4_i = phi^(4d) mean(x_s^4); the
    estimated variance of the correction is phi^(4d) (mean x^4 - mean(x^2)^2)
    / (k - 1), written here from the raw separator samples."""
    phi, k = 0.95, 64
    model, th = ar1_model(99, phi)
    X = o.samples(model, th, 7, k)
    v, _, res = o.rbmc(model, th, np.array([0, 50, 99]), 0, X)
    part_err, glob = o.error_estimate(v, res, k)
    q = []
    for rows, sep in ((np.arange(50), 50), (np.arange(50, 99), 49)):
        x = X[sep]
        d = np.abs(rows - sep)
        var = phi ** (4 * d) * (np.mean(x ** 4) - np.mean(x ** 2) ** 2) / (k - 1)
        q.append(var / v[rows] ** 2)
    np.testing.assert_allclose(part_err, [math.sqrt(a.mean()) for a in q], rtol=1e-12)
    assert abs(glob - math.sqrt(np.concatenate(q).mean())) <= 1e-12 * glob
    # a single part has no separator and zero error
    v1, _, r1 = o.rbmc(model, th, np.array([0, 99]), 0, X)
    assert o.error_estimate(v1, r1, k)[1] == 0.0


@pytest.mark.slow
def test_rbmc_unbiased_over_seeds():
    """E[v_hat] = diag(Q^-1) and E[t_hat] = t (Eq. var:2): per-node z-scores
    with the Gaussian variance Var(w_i^2) = 2 c_i^2 / k where c_i = E[w_i^2],
    and traces with their empirical variance."""
    model = grid_model(5, 6, obs_frac=0.3)
    th = theta(0.5, 1.0, 0.9)
    slab_start = o.balanced_slab_start(6, 2)
    Q = o.precision(model, th)
    v_ex, t_ex = o.exact_selinv(Q, o.precision_derivatives(model, th))
    R, k = 200, 8
    vs, ts, c = [], [], None
    for seed in range(R):
        X = o.samples(model, th, 1000 + seed, k)
        v, t, res = o.rbmc(model, th, slab_start, 1, X)
        vs.append(v); ts.append(t)
        sig = np.concatenate([r.sigma_star_diag for r in res])
        c = v_ex - sig
    vs, ts = np.array(vs), np.array(ts)
    big = c > 1e-6 * v_ex
    z = (vs.mean(0) - v_ex)[big] / np.sqrt(2 * c[big] ** 2 / k / R)
    # nodes share the same samples, so only the per-node bound is used
    assert np.abs(z).max() < 4.5
    zt = (ts.mean(0) - np.array(t_ex)) / (ts.std(0, ddof=1) / math.sqrt(R))
    assert np.abs(zt).max() < 4.5


def test_per_part_overlap_equals_uniform_runs():
    """With one overlap per part, part p of the estimate equals part p of the
    uniform-overlap estimate with that overlap (parts are independent given
    the samples, Algorithm 4)."""
    model = grid_model(5, 9, obs_frac=0.3)
    th = theta(0.5, 1.0, 0.9)
    ss = o.balanced_slab_start(9, 3)
    X = o.samples(model, th, 3, 6)
    v, t, res = o.rbmc(model, th, ss, [1, 2, 1], X)
    n_s = 25
    for p, nl in enumerate([1, 2, 1]):
        vu, _, ru = o.rbmc(model, th, ss, nl, X)
        rows = slice(ss[p] * n_s, ss[p + 1] * n_s)
        np.testing.assert_array_equal(v[rows], vu[rows])
        np.testing.assert_array_equal(res[p].traces, ru[p].traces)
    assert res[1].part.ext == (1, 8) and res[0].part.ext == (0, 4)
