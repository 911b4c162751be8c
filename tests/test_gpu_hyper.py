"""GPU posterior mean and hyperparameter gradient (qsel_set_data,
qsel_posterior_mean, qsel_loglik_grad) against the oracle
(oracle/qsel_hyper.py) on the same seeded model and data, and the
quasi-Newton loop of paper_2309_05435_gb300.hyper against the oracle's own
maximiser of log p(y | theta).

Tolerances: FP64 1e-7 relative (PCG to 1e-10, dense pieces in binary64);
mixed: the stated mixed trace tolerance 1e-4 on the trace term's scale."""
import numpy as np
import pytest
import scipy.linalg as sla

import qsel_inputs as qi
from oracle import qsel_hyper as h
from oracle import qsel_oracle as o
from tests.test_gpu_parity import Case, q  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def _y(c, seed=11):
    return qi.seeded_normal((int(np.count_nonzero(c.mask)), 1), seed)[:, 0]


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["grid16_nt8", "ragged13"])
def test_posterior_mean_matches_oracle(q, name, precision):
    prec = q.QSEL_FP64 if precision == "fp64" else q.QSEL_MIXED
    c = Case(q, name, precision=prec, pcg_tol=1e-10)
    y = _y(c)
    q.qsel_set_data(c.ctx, y)
    mu = q.qsel_posterior_mean(c.ctx)
    mu_or = h.posterior_mean(c.model, c.theta, y)
    print(f"{name} {precision}: posterior mean vs oracle {_rel(mu, mu_or):.2e}")
    assert _rel(mu, mu_or) < 1e-7


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_loglik_grad_single_part_matches_oracle(q, precision):
    """One part: the traces are exact, so the whole gradient is."""
    prec = q.QSEL_FP64 if precision == "fp64" else q.QSEL_MIXED
    c = Case(q, "grid16_nt8", precision=prec, parts=1, overlap=0, pcg_tol=1e-10)
    y = _y(c)
    q.qsel_set_data(c.ctx, y)
    g, (prior, tr, quad) = q.qsel_loglik_grad(c.ctx, with_terms=True)
    mu_or = h.posterior_mean(c.model, c.theta, y)
    g_or = h.loglik_grad(c.model, c.theta, y)
    np.testing.assert_allclose(prior, h.prior_logdet_grad(c.model, c.theta), rtol=1e-10)
    np.testing.assert_allclose(quad, h.quadratic_terms(c.model, c.theta, mu_or), rtol=1e-7)
    scale = 0.5 * (np.abs(prior) + np.abs(tr) + np.abs(quad))
    tol = 1e-7 if precision == "fp64" else 1e-4
    print(f"{precision}: gradient {g} oracle {g_or}")
    assert np.all(np.abs(g - g_or) <= tol * scale)


def test_loglik_grad_rbmc_matches_oracle_with_injected_samples(q):
    """Several parts: the trace term is the RBMC estimate; with the same
    injected samples the oracle's estimator gives the same gradient."""
    c = Case(q, "overlap2", precision=q.QSEL_FP64, pcg_tol=1e-10)
    X = qi.seeded_normal((c.n_s * c.n_t, c.k), 99)
    q.qsel_debug_set_samples(c.ctx, X)
    y = _y(c)
    q.qsel_set_data(c.ctx, y)
    g, (prior, tr, quad) = q.qsel_loglik_grad(c.ctx, with_terms=True)
    _, t_or, _ = o.rbmc(c.model, c.theta, c.slab_start, c.n_l, X)
    g_or = h.loglik_grad(c.model, c.theta, y, traces=t_or)
    scale = 0.5 * (np.abs(prior) + np.abs(tr) + np.abs(quad))
    assert np.all(np.abs(g - g_or) <= 1e-7 * scale)


def test_optimizer_reaches_the_oracle_mode(q):
    """Data drawn from the model at theta_true; from a start 0.4-0.5 away in
    each component the GPU loop ends at the oracle's maximiser of the exact
    log p(y | theta) (BFGS on the oracle's value and gradient)."""
    import scipy.optimize as so

    from paper_2309_05435_gb300 import hyper
    from tests.models import theta as mk_theta
    m, n_t, sigma = 8, 6, 0.3
    mesh = qi.grid_mesh(m)
    n = m * m * n_t
    mask = qi.obs_mask(n, 0.5, 3)
    model = o.model_from_csr(m * m, n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val, mask, sigma)
    th_true = np.array(mk_theta(0.5, 2.0, 0.8))
    L = np.linalg.cholesky(h.prior_precision(model, th_true).toarray())
    x = sla.solve_triangular(L.T, qi.seeded_normal((n, 1), 21)[:, 0], lower=False)
    obs = np.flatnonzero(model.obs_mask)
    y = x[obs] + sigma * qi.seeded_normal((len(obs), 1), 22)[:, 0]
    th0 = th_true + np.array([0.4, -0.4, -0.5])
    res = so.minimize(lambda t: -h.log_marginal(model, t, y), th0, jac=lambda t: -h.loglik_grad(model, t, y),
                      method="BFGS", options={"gtol": 1e-8})
    ctx = q.qsel_create(m * m, n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val, mask, sigma, th0,
                        n_parts=1, overlap=0, n_samples=2, precision=q.QSEL_FP64, pcg_tol=1e-12)
    th, hist = hyper.optimize_theta(ctx, y, th0)
    print(f"GPU mode {th} after {len(hist)} steps; oracle mode {res.x}")
    assert np.max(np.abs(th - res.x)) < 1e-4


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fixed_effects_match_oracle(q, precision):
    """mu_u, mu_beta, Var(beta) and the Eq. var:1 correction against the
    oracle's Schur-complement formulas (verified there against the joint
    Gaussian)."""
    prec = q.QSEL_FP64 if precision == "fp64" else q.QSEL_MIXED
    c = Case(q, "grid16_nt8", precision=prec, pcg_tol=1e-10)
    y = _y(c)
    Z = qi.seeded_normal((len(y), 3), 8)
    q.qsel_set_data(c.ctx, y)
    q.qsel_set_covariates(c.ctx, Z, 0.5)
    mu = q.qsel_posterior_mean(c.ctx)
    mu_b, var_b, corr = q.qsel_fixed_effects(c.ctx, 3)
    mu_or, mu_b_or, Sinv_or, corr_or, _ = h.fixed_effects(c.model, c.theta, y, Z, 0.5)
    print(f"{precision}: mu_u {_rel(mu, mu_or):.2e} mu_beta {_rel(mu_b, mu_b_or):.2e} "
          f"Var(beta) {_rel(var_b, Sinv_or):.2e} corr {_rel(corr, corr_or):.2e}")
    for a, b in ((mu, mu_or), (mu_b, mu_b_or), (var_b, Sinv_or), (corr, corr_or)):
        assert _rel(a, b) < 1e-7


def test_loglik_grad_with_fixed_effects_single_part(q):
    c = Case(q, "grid16_nt8", precision=q.QSEL_FP64, parts=1, overlap=0, pcg_tol=1e-10)
    y = _y(c)
    Z = qi.seeded_normal((len(y), 2), 9)
    q.qsel_set_data(c.ctx, y)
    q.qsel_set_covariates(c.ctx, Z, 2.0)
    g, (prior, tr, quad) = q.qsel_loglik_grad(c.ctx, with_terms=True)
    g_or = h.loglik_grad_fe(c.model, c.theta, y, Z, 2.0)
    scale = 0.5 * (np.abs(prior) + np.abs(tr) + np.abs(quad))
    print(f"fixed effects: gradient {g} oracle {g_or}")
    assert np.all(np.abs(g - g_or) <= 1e-7 * scale)
    # removing the covariates restores the model without fixed effects
    q.qsel_set_covariates(c.ctx, np.zeros((len(y), 0)), 1.0)
    g0 = q.qsel_loglik_grad(c.ctx)
    g0_or = h.loglik_grad(c.model, c.theta, y)
    assert np.all(np.abs(g0 - g0_or) <= 1e-7 * scale)
