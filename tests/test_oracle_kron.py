"""Pins of the Kronecker grid preconditioner reference (oracle/qsel_kron.py):
the 1-D factors reproduce the grid's stiffness exactly, the temporal inverse
is the AR(1) covariance, and with the corner masses set to D (x) D and no
observations the preconditioner inverts the prior precision exactly."""
import math

import numpy as np

import qsel_inputs as qi
from oracle import qsel_kron as kr
from oracle import qsel_oracle as o
from tests.models import theta


def test_grid_stiffness_and_mass_factor():
    for m in (4, 7):
        mesh = qi.grid_mesh(m)
        T, D = kr.neumann_1d(m)
        np.testing.assert_allclose(mesh.g_dense(), np.kron(T, D) + np.kron(D, T), atol=1e-14)
        C = np.kron(np.diag(D), np.diag(D))
        diff = np.flatnonzero(np.abs(mesh.c_diag - C) > 1e-14)
        assert set(diff) <= {0, m - 1, m * (m - 1), m * m - 1}
        lam, V, dh = kr.grid_factors(m)
        np.testing.assert_allclose(V @ np.diag(lam) @ V.T, dh[:, None] * T * dh[None, :], atol=1e-13)


def test_temporal_inverse_is_ar1_covariance():
    rho, n_t = 0.8, 6
    Ct = kr.temporal_inverse(rho, n_t)
    t = np.arange(n_t)
    np.testing.assert_allclose(Ct, rho ** np.abs(t[:, None] - t[None, :]), atol=1e-14)
    np.testing.assert_allclose(Ct @ o.temporal_precision(rho, n_t), np.eye(n_t), atol=1e-13)


def test_exact_inverse_of_the_prior_with_tensor_mass():
    """No observations and C = D (x) D (corners changed): M^-1 Q = I."""
    m, n_t = 5, 4
    mesh = qi.grid_mesh(m)
    _, D = kr.neumann_1d(m)
    c = np.kron(np.diag(D), np.diag(D))
    mdl = o.model_from_csr(m * m, n_t, c, mesh.g_rowptr, mesh.g_col, mesh.g_val,
                           np.zeros(m * m * n_t, np.uint8), 1.0)
    th = theta(0.7, 1.4, 0.85)
    Minv = kr.preconditioner_inverse(mdl, th)
    Q = o.precision(mdl, th).toarray()
    np.testing.assert_allclose(Minv @ Q, np.eye(mdl.n), atol=1e-9)


def test_eigen_form_equals_explicit_operator():
    """The diagonalised M^-1 is the inverse of the operator written out
    densely: (I (x) D^1/2 (x) D^1/2)(tau Q_t (x) S^2 + omega I)(...), S built
    from T^ directly (no eigenvectors)."""
    m, n_t = 4, 3
    mesh = qi.grid_mesh(m)
    mdl = o.model_from_csr(m * m, n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val,
                           qi.obs_mask(m * m * n_t, 0.25, 3), 0.5)
    th = theta(0.6, 1.3, 0.7)
    kappa, tau, rho = o.theta_to_natural(th)
    T, D = kr.neumann_1d(m)
    Th = np.diag(np.diag(D) ** -0.5) @ T @ np.diag(np.diag(D) ** -0.5)
    S = kappa ** 2 * np.eye(m * m) + np.kron(Th, np.eye(m)) + np.kron(np.eye(m), Th)
    Dsq = np.kron(np.eye(n_t), np.kron(np.sqrt(D), np.sqrt(D)))
    om = kr.omega(mdl)
    assert abs(om - 12 / 48 / 0.25) < 1e-15
    M = Dsq @ (tau * np.kron(o.temporal_precision(rho, n_t), S @ S) + om * np.eye(mdl.n)) @ Dsq
    np.testing.assert_allclose(kr.preconditioner_inverse(mdl, th) @ M, np.eye(mdl.n), atol=1e-10)


def test_preconditioned_spectrum_on_observed_grid():
    """With observations and the true corner masses the preconditioned
    operator is well conditioned (about 10 here, against about 200 for
    64-row block Jacobi and 2400 for Q itself)."""
    mesh = qi.grid_mesh(8)
    mdl = o.model_from_csr(64, 6, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val,
                           qi.obs_mask(384, 0.3, 2), 0.5)
    th = theta(0.5, 1.0, 0.9)
    Q = o.precision(mdl, th).toarray()
    Minv = kr.preconditioner_inverse(mdl, th)
    L = np.linalg.cholesky(Minv)
    ev = np.linalg.eigvalsh(L.T @ Q @ L)
    assert ev.min() > 0.1 and ev.max() / ev.min() < 30 and np.linalg.cond(Q) > 300
    assert math.isfinite(ev.max())
