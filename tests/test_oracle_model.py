"""Pins of the input mesh and the oracle's model assembly against closed forms,
textbook identities and finite differences (no GPU)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import qsel_inputs as qi
from oracle import qsel_oracle as o
from tests.models import grid_model, theta


@pytest.mark.parametrize("m", [2, 3, 5, 16])
def test_mesh_closed_form(m):
    """P1 stiffness on the right-triangle grid is the 5-point stencil with
    -1 between interior neighbours and -1/2 along boundary edges; lumped mass
    sums to the domain area (m-1)^2 and is 1/6 at the two corners touched by
    a single triangle, 1/3 at the other two, 1/2 on edges and 1 inside."""
    mesh = qi.grid_mesh(m)
    G = mesh.g_dense()
    n_s = m * m
    expect = np.zeros((n_s, n_s))
    for i in range(m):
        for j in range(m):
            a = i * m + j
            for di, dj in ((1, 0), (0, 1)):
                ii, jj = i + di, j + dj
                if ii >= m or jj >= m:
                    continue
                b = ii * m + jj
                on_boundary = (di == 1 and (j == 0 or j == m - 1)) or (dj == 1 and (i == 0 or i == m - 1))
                wgt = 0.5 if on_boundary else 1.0
                expect[a, b] -= wgt
                expect[b, a] -= wgt
                expect[a, a] += wgt
                expect[b, b] += wgt
    np.testing.assert_allclose(G, expect, atol=1e-14)
    np.testing.assert_allclose(G.sum(axis=1), 0.0, atol=1e-13)
    assert abs(mesh.c_diag.sum() - (m - 1) ** 2) < 1e-12
    c = mesh.c_diag.reshape(m, m)
    assert abs(c[m - 1, 0] - 1 / 6) < 1e-15 and abs(c[0, m - 1] - 1 / 6) < 1e-15
    assert abs(c[0, 0] - 1 / 3) < 1e-15 and abs(c[m - 1, m - 1] - 1 / 3) < 1e-15
    if m > 2:
        assert np.allclose(c[1:-1, 1:-1], 1.0) and np.allclose(c[0, 1:-1], 0.5)


def test_obs_mask_count():
    for n, frac in ((2048, 0.30), (262144, 0.25), (1000, 0.1)):
        mask = qi.obs_mask(n, frac, 1)
        assert mask.sum() == int(round(frac * n))
    assert qi.obs_mask(2048, 0.3, 1).sum() == 614


@pytest.mark.parametrize("rho,n_t", [(0.9, 8), (0.5, 3), (0.98, 17)])
def test_temporal_precision_inverse_is_ar1_correlation(rho, n_t):
    """The unit-variance AR(1) has covariance rho^|i-j|."""
    Qt = o.temporal_precision(rho, n_t)
    idx = np.arange(n_t)
    cov = rho ** np.abs(idx[:, None] - idx[None, :])
    np.testing.assert_allclose(np.linalg.inv(Qt), cov, rtol=1e-11, atol=1e-12)
    B = o.ar1_B(rho, n_t)
    np.testing.assert_allclose(B.T @ B / (1 - rho ** 2), Qt, rtol=1e-13, atol=1e-13)


def test_spatial_precision_expanded_form():
    """(kappa^2 C + G) C^-1 (kappa^2 C + G) = kappa^4 C + 2 kappa^2 G + G C^-1 G."""
    mesh = qi.grid_mesh(6)
    model = o.model_from_csr(36, 2, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val,
                             np.zeros(72, np.uint8), 1.0)
    kappa = 0.37
    Qs = o.spatial_precision(model, kappa).toarray()
    C = np.diag(mesh.c_diag)
    G = mesh.g_dense()
    np.testing.assert_allclose(Qs, kappa ** 4 * C + 2 * kappa ** 2 * G + G @ np.linalg.inv(C) @ G,
                               rtol=1e-12, atol=1e-12)
    # G C^-1 G couples nodes up to graph distance 2 of the 5-point stencil: 13-point pattern
    assert (np.count_nonzero(Qs[3 * 6 + 3]) == 13)


def test_precision_block_structure():
    model = grid_model(5, 4)
    th = theta(0.5, 1.7, 0.9)
    Q = o.precision(model, th)
    kappa, tau, rho = o.theta_to_natural(th)
    Qs = o.spatial_precision(model, kappa).toarray()
    Qt = o.temporal_precision(rho, 4)
    obs = model.obs_mask.reshape(4, 25) / model.sigma ** 2
    for t in range(4):
        for u in range(4):
            blk = o.block(Q, 25, t, u)
            want = tau * Qt[t, u] * Qs + (np.diag(obs[t]) if t == u else 0)
            np.testing.assert_allclose(blk, want, rtol=1e-13, atol=1e-13)
    ev = np.linalg.eigvalsh(Q.toarray())
    assert ev.min() > 0


@pytest.mark.parametrize("th", [theta(0.5, 1.0, 0.9), theta(0.2, 2.5, 0.5), theta(1.3, 0.4, 0.97)])
def test_precision_derivatives_match_central_differences(th):
    """dQ/dtheta_j against central differences of Q(theta) (h = 1e-5)."""
    model = grid_model(4, 5)
    dQs = o.precision_derivatives(model, th)
    h = 1e-5
    for j in range(3):
        tp = list(th); tp[j] += h
        tm = list(th); tm[j] -= h
        fd = ((o.precision(model, tp) - o.precision(model, tm)) / (2 * h)).toarray()
        an = dQs[j].toarray()
        scale = np.abs(an).max()
        assert np.abs(fd - an).max() <= 1e-7 * scale, j


def test_theta_convention():
    kappa, tau, rho = o.theta_to_natural((math.log(0.2), math.log(3.0), math.log(0.95 / 0.05)))
    assert abs(kappa - 0.2) < 1e-15 and abs(tau - 3.0) < 1e-14 and abs(rho - 0.95) < 1e-14


@pytest.mark.parametrize("m,n_t,kappa,rho", [(5, 4, 0.7, 0.9), (6, 7, 0.3, 0.98)])
def test_unobserved_closed_form_matches_exact_selinv(m, n_t, kappa, rho):
    """The Kronecker closed form used by the full-size GPU tests equals the
    oracle's dense selected inverse of the unobserved prior, diagonal and all
    three traces (each term of the closed form is checked by one of them)."""
    from tests.models import unobserved_closed_form
    tau = 1.7
    mesh = qi.grid_mesh(m)
    model = o.model_from_csr(mesh.n_s, n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val,
                             np.zeros(mesh.n_s * n_t, np.uint8), 0.5)
    th = (np.log(kappa), np.log(tau), np.log(rho / (1 - rho)))
    v_ex, t_ex = o.exact_selinv(o.precision(model, th), o.precision_derivatives(model, th))
    v_cf, t_cf = unobserved_closed_form(mesh, n_t, kappa, tau, rho)
    # both sides round at about cond(Q) x 1e-16 (cond ~ 1e6 at rho = 0.98,
    # kappa = 0.3); a wrong term of the closed form is an O(1) error
    assert np.max(np.abs(v_cf - v_ex) / np.abs(v_ex)) < 1e-8
    assert np.max(np.abs(t_cf - np.asarray(t_ex)) / np.abs(np.asarray(t_ex))) < 1e-8
