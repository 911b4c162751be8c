"""Pins of the oracle's noise generator and perturbation sampler (no GPU)."""
import os

import numpy as np
import scipy.sparse.linalg as spla

from oracle import qsel_oracle as o
from tests.models import grid_model, theta

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    """Published Philox4x32-10 known-answer vectors (Salmon et al., SC'11)."""
    n = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            ctr = np.array(w[0:4], dtype=np.uint32).reshape(4, 1)
            key = np.array(w[4:6], dtype=np.uint32)
            out = o.philox4x32_10(ctr, key)[:, 0]
            assert [int(x) for x in out] == w[6:10]
            n += 1
    assert n == 3


def test_normals_moments_and_streams():
    z = o.philox_normals(7, 0, 2000, 64)
    assert z.shape == (2000, 64) and np.all(np.isfinite(z))
    assert abs(z.mean()) < 4.5 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 4.5 * np.sqrt(2 / z.size)
    # odd k truncates the last pair; streams and seeds decorrelate
    np.testing.assert_array_equal(o.philox_normals(7, 0, 10, 5), z[:10, :5])
    z1 = o.philox_normals(7, 1, 2000, 64)
    z8 = o.philox_normals(8, 0, 2000, 64)
    assert abs(np.mean(z * z1)) < 4.5 / np.sqrt(z.size)
    assert abs(np.mean(z * z8)) < 4.5 / np.sqrt(z.size)


def test_perturbation_rhs_covariance_is_Q():
    """Applying the RHS map to unit noise vectors gives M = [F^T, A^T/sigma];
    the perturbation construction is exact iff M M^T = Q."""
    model = grid_model(4, 5, obs_frac=0.3)
    th = theta(0.6, 1.4, 0.85)
    n = model.n
    n_obs = int(model.obs_mask.sum())
    M1 = o.perturbation_rhs(model, th, np.eye(n), np.zeros((n_obs, n)))
    M2 = o.perturbation_rhs(model, th, np.zeros((n, n_obs)), np.eye(n_obs))
    Q = o.precision(model, th).toarray()
    np.testing.assert_allclose(M1 @ M1.T + M2 @ M2.T, Q, rtol=1e-12, atol=1e-12 * np.abs(Q).max())


def test_direct_samples_solve_the_system():
    model = grid_model(5, 4)
    th = theta(0.5, 1.0, 0.9)
    R = o.rhs(model, th, 11, 6)
    X = o.solve_direct(model, th, R)
    Q = o.precision(model, th).tocsc()
    np.testing.assert_allclose(X, spla.spsolve(Q, R), rtol=1e-10, atol=1e-12)
