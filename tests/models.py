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
