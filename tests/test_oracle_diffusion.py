"""Pins of the diffusion-model oracle (oracle/qsel_diffusion.py) against facts
that do not come from its own formulas: the spectral closed form of log|Q_u|,
finite differences, the block-tridiagonal structure, and the exact RBMC
identities of Algorithm 4."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import qsel_inputs as qi
from oracle import qsel_diffusion as od
from oracle import qsel_oracle as o
from tests.models import grid_model

THETAS = [(math.log(0.4), math.log(1.5), math.log(0.8)), (math.log(1.2), math.log(0.3), math.log(2.0))]


def _spectral_logdet(model, theta):
    """log|Q_u| from the eigen-decomposition of C^-1/2 G C^-1/2 = U diag(lam) U^T:
    Q_u = (I (x) C^1/2 U) [sum_k gamma_t^k J_k (x) (gamma_s^2 + lam)^a_k] (I (x) U^T C^1/2),
    so log|Q_u| = n_t log|C| + sum over lam of log|T(lam)| with the n_t x n_t
    matrix T(lam) = gamma_e^2 (M0 a^3 + 2 gamma_t M1 a^2 + gamma_t^2 M2 a),
    a = gamma_s^2 + lam."""
    gs, gt, ge = math.exp(theta[0]), math.exp(theta[1]), math.exp(theta[2])
    c = model.c_diag
    S = model.G.toarray() / np.sqrt(np.outer(c, c))
    lam = np.linalg.eigvalsh(0.5 * (S + S.T))
    n_t = model.n_t
    M0 = np.diag([0.5] + [1.0] * (n_t - 2) + [0.5])
    M1 = np.zeros((n_t, n_t))
    M1[0, 0] = M1[-1, -1] = 0.5
    M2 = 2 * np.eye(n_t) - np.eye(n_t, k=1) - np.eye(n_t, k=-1)
    M2[0, 0] = M2[-1, -1] = 1.0
    total = n_t * np.sum(np.log(c))
    for l in lam:
        a = gs ** 2 + l
        T = ge ** 2 * (M0 * a ** 3 + 2 * gt * M1 * a ** 2 + gt ** 2 * M2 * a)
        sign, ld = np.linalg.slogdet(T)
        assert sign > 0
        total += ld
    return total


@pytest.mark.parametrize("theta", THETAS)
def test_prior_logdet_matches_spectral_closed_form(theta):
    model = grid_model(5, 6, obs_frac=0.0)
    Qu = od.prior_precision(model, theta).toarray()
    sign, ld = np.linalg.slogdet(Qu)
    assert sign > 0
    assert abs(ld - _spectral_logdet(model, theta)) <= 1e-9 * abs(ld)


def test_block_tridiagonal_symmetric_positive_definite():
    model = grid_model(4, 5, obs_frac=0.3)
    Q = od.precision(model, THETAS[0]).toarray()
    n_s = model.n_s
    assert np.max(np.abs(Q - Q.T)) <= 1e-12 * np.max(np.abs(Q))
    for t in range(model.n_t):
        for u in range(model.n_t):
            if abs(t - u) > 1:
                assert not np.any(Q[t * n_s:(t + 1) * n_s, u * n_s:(u + 1) * n_s])
    np.linalg.cholesky(Q)
    # the coupling blocks are -gamma_e^2 gamma_t^2 K1 (the stiffness J2 has -1 off the diagonal)
    gs, gt, ge = od.theta_to_natural(THETAS[0])
    K1 = (gs ** 2 * np.diag(model.c_diag) + model.G.toarray())
    np.testing.assert_allclose(Q[n_s:2 * n_s, 0:n_s], -ge ** 2 * gt ** 2 * K1, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("theta", THETAS)
def test_derivatives_match_finite_differences(theta):
    model = grid_model(4, 4, obs_frac=0.3)
    dQs = od.precision_derivatives(model, theta)
    h = 1e-5
    for j in range(3):
        tp, tm = list(theta), list(theta)
        tp[j] += h
        tm[j] -= h
        fd = (od.precision(model, tp) - od.precision(model, tm)).toarray() / (2 * h)
        d = dQs[j].toarray()
        assert np.max(np.abs(fd - d)) <= 1e-6 * np.max(np.abs(d)), j


@pytest.mark.parametrize("theta", THETAS)
def test_traces_match_logdet_finite_differences(theta):
    model = grid_model(4, 5, obs_frac=0.3)
    Q = od.precision(model, theta)
    _, t_ex = o.exact_selinv(Q, od.precision_derivatives(model, theta))
    h = 1e-5
    for j in range(3):
        tp, tm = list(theta), list(theta)
        tp[j] += h
        tm[j] -= h
        fd = (np.linalg.slogdet(od.precision(model, tp).toarray())[1]
              - np.linalg.slogdet(od.precision(model, tm).toarray())[1]) / (2 * h)
        assert abs(fd - t_ex[j]) <= 1e-6 * max(1.0, abs(t_ex[j])), j


def test_single_part_is_exact():
    model = grid_model(4, 6, obs_frac=0.3)
    th = THETAS[1]
    Q = od.precision(model, th)
    dQs = od.precision_derivatives(model, th)
    v, t, _ = od.rbmc_precision(Q, dQs, model.n_s, model.n_t, [0, model.n_t], 0, np.zeros((model.n, 1)))
    v_ex, t_ex = o.exact_selinv(Q, dQs)
    np.testing.assert_allclose(v, v_ex, rtol=1e-11)
    np.testing.assert_allclose(t, t_ex, rtol=1e-11)


@pytest.mark.parametrize("n_p,n_l", [(2, 1), (3, 1), (3, 2)])
def test_square_root_samples_reproduce_exact_result(n_p, n_l):
    """X = sqrt(n) chol(Q^-1): (1/n) X_S X_S^T = Sigma_SS exactly, so the RBMC
    estimate equals the exact diagonal and traces (law of total variance,
    Eq. var:2 and Eq. var:4)."""
    model = grid_model(4, 7, obs_frac=0.3)
    th = THETAS[0]
    Q = od.precision(model, th)
    dQs = od.precision_derivatives(model, th)
    S = np.linalg.inv(Q.toarray())
    X = math.sqrt(model.n) * np.linalg.cholesky(0.5 * (S + S.T))
    v, t, _ = od.rbmc_precision(Q, dQs, model.n_s, model.n_t, qi.balanced_slab_start(model.n_t, n_p), n_l, X)
    v_ex, t_ex = o.exact_selinv(Q, dQs)
    np.testing.assert_allclose(v, v_ex, rtol=1e-9)
    np.testing.assert_allclose(t, t_ex, rtol=1e-9)


def test_separable_model_through_the_generic_rbmc():
    """rbmc_precision on the separable model's Q equals the separable oracle."""
    model = grid_model(4, 6, obs_frac=0.3)
    th = (math.log(0.5), 0.0, math.log(0.9 / 0.1))
    X = qi.seeded_normal((model.n, 8), 4)
    v1, t1, _ = o.rbmc(model, th, [0, 3, 6], 1, X)
    v2, t2, _ = od.rbmc_precision(o.precision(model, th), o.precision_derivatives(model, th), model.n_s,
                                  model.n_t, [0, 3, 6], 1, X)
    np.testing.assert_allclose(v1, v2, rtol=1e-13)
    np.testing.assert_allclose(t1, t2, rtol=1e-13)
