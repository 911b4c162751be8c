"""Small seeded models for tests (built from the shared input generator)."""
import numpy as np

import qsel_inputs as qi
from oracle import qsel_oracle as o


def grid_model(m, n_t, obs_frac=0.3, sigma=0.5, seed=1):
    mesh = qi.grid_mesh(m)
    mask = qi.obs_mask(mesh.n_s * n_t, obs_frac, seed)
    return o.model_from_csr(mesh.n_s, n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val,
                            mask, sigma)


def theta(kappa, tau, rho):
    return (float(np.log(kappa)), float(np.log(tau)), float(np.log(rho / (1 - rho))))


def ar1_model(n_t, rho):
    """n_s = 1, C = 1, G = 0, kappa = 1 => Q_s = 1 and Q = Q_t, a unit-variance AR(1)."""
    return o.model_from_csr(1, n_t, np.ones(1), np.array([0, 1], np.int32), np.array([0], np.int32),
                            np.zeros(1), np.zeros(n_t, np.uint8), 1.0), theta(1.0, 1.0, rho)


def unobserved_closed_form(mesh, n_t, kappa, tau, rho):
    """Selected inverse of the separable prior with no observations,
    Q = tau Q_t (x) Q_s with Q_s = K C^-1 K and K = kappa^2 C + G, from its
    Kronecker factors: Q^-1 = tau^-1 Q_t^-1 (x) K^-1 C K^-1, and Q_t^-1 has unit
    diagonal (the AR(1) correlation), so diag(Q^-1) = tau^-1 diag(K^-1 C K^-1)
    on every slab; tr(Q^-1 dQ/dlog kappa) = n_t tr(K^-1 C K^-1 4 kappa^2 K) =
    4 kappa^2 n_t sum_i c_i (K^-1)_ii, tr(Q^-1 dQ/dlog tau) = n, and
    tr(Q^-1 dQ/dlogit rho) = n_s tr(Q_t^-1 dQ_t/dlogit rho).  Dense K^-1: n_s up to
    about 10^4."""
    n_s = mesh.n_s
    m1 = o.model_from_csr(n_s, 1, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val, np.zeros(n_s, np.uint8), 1.0)
    Kinv = np.linalg.inv(o.spatial_K(m1, kappa).toarray())
    c = np.asarray(mesh.c_diag, dtype=np.float64)
    diag_s = (Kinv * Kinv) @ c
    Qt = o.temporal_precision(rho, n_t)
    dQt = o.temporal_precision_drho(rho, n_t) * rho * (1.0 - rho)
    traces = np.array([4.0 * kappa ** 2 * n_t * float(np.sum(c * np.diag(Kinv))), float(n_s * n_t),
                       n_s * float(np.trace(np.linalg.solve(Qt, dQt)))])
    return np.tile(diag_s / tau, n_t), traces
