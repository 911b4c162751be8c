"""Pins of the preconditioned Krylov sampler reference (oracle/qsel_lanczos.py)
against closed forms: the block factors, the rewind identity of
Eqs. sampling:7-8, the exactness of the Krylov approximation when the
subspace is the whole space, the Lanczos relation, and convergence in m."""
import numpy as np
import scipy.linalg as sla

from oracle import qsel_lanczos as lz
from oracle import qsel_oracle as o
from tests.models import grid_model, theta


def _setup(m=4, n_t=3):
    mdl = grid_model(m, n_t, obs_frac=0.3)
    th = theta(0.6, 1.2, 0.8)
    Q = o.precision(mdl, th).tocsr()
    return mdl, th, Q


def _dense_factor(fac, n):
    Linv = np.zeros((n, n))
    for r0, _, Li in fac:
        Linv[r0:r0 + Li.shape[0], r0:r0 + Li.shape[0]] = Li
    return Linv


def test_block_factors_and_rewind_identity():
    """L_b L_b^T = Q_bb (ragged last block), and with M = L^-T Q~^-1/2 the
    sampler's covariance M M^T equals Q^-1 (Eq. sampling:7)."""
    mdl, th, Q = _setup()
    n = mdl.n
    fac = lz.block_factors(Q, 20)              # 48 rows: blocks 20, 20, 8
    assert [f[1].shape[0] for f in fac] == [20, 20, 8]
    for r0, L, _ in fac:
        r1 = r0 + L.shape[0]
        np.testing.assert_allclose(L @ L.T, Q[r0:r1, r0:r1].toarray(), rtol=1e-13, atol=1e-13)
    Linv = _dense_factor(fac, n)
    Qt = Linv @ Q.toarray() @ Linv.T
    lam, U = np.linalg.eigh(Qt)
    M = Linv.T @ (U * lam ** -0.5) @ U.T
    np.testing.assert_allclose(M @ M.T, np.linalg.inv(Q.toarray()), rtol=1e-9, atol=1e-12)


def test_full_krylov_space_is_exact():
    """m = n: V f(T) eta e1 = Q~^-1/2 z, so the sample is L^-T Q~^-1/2 z."""
    mdl, th, Q = _setup()
    n = mdl.n
    X, alphas, _ = lz.sample(mdl, th, seed=3, k=2, m=n, b=16)
    fac = lz.block_factors(Q, 16)
    Linv = _dense_factor(fac, n)
    Qt = Linv @ Q.toarray() @ Linv.T
    lam, U = np.linalg.eigh(Qt)
    Z = o.philox_normals(3, 0, n, 2)
    X_ex = Linv.T @ (U * lam ** -0.5) @ U.T @ Z
    np.testing.assert_allclose(X, X_ex, rtol=1e-6, atol=1e-8)
    assert len(alphas[0]) <= n


def test_lanczos_relation_and_orthonormal_basis():
    mdl, th, Q = _setup(6, 4)
    fac = lz.block_factors(Q, 32)

    def op(v):
        return lz.apply_Linv(fac, Q @ lz.apply_LinvT(fac, v))

    z = o.philox_normals(5, 0, mdl.n, 1)[:, 0]
    m = 12
    a, b, V = lz.lanczos(op, z, m)
    T = np.diag(a) + np.diag(b[:-1], 1) + np.diag(b[:-1], -1)
    np.testing.assert_allclose(V.T @ V, np.eye(m), atol=1e-10)
    # op V = V T + beta_m v_{m+1} e_m^T: the residual lies in the last column only
    R = np.column_stack([op(V[:, j]) for j in range(m)]) - V @ T
    np.testing.assert_allclose(R[:, :-1], 0.0, atol=1e-10)
    assert abs(np.linalg.norm(R[:, -1]) - b[-1]) <= 1e-10 * max(1.0, b[-1])
    np.testing.assert_allclose(V[:, 0], z / np.linalg.norm(z), rtol=1e-14)


def test_f_T_e1_against_dense_matrix_function():
    rng = np.random.default_rng(1)
    a = rng.uniform(2.0, 4.0, 7)
    b = rng.uniform(0.1, 0.9, 7)
    T = np.diag(a) + np.diag(b[:-1], 1) + np.diag(b[:-1], -1)
    ref = sla.fractional_matrix_power(T, -0.5)[:, 0] * 2.5
    np.testing.assert_allclose(lz.f_T_e1(a, b, 2.5), ref, rtol=1e-9, atol=1e-13)


def test_error_decreases_with_subspace_size():
    """Against the dense L^-T Q~^-1/2 z: the Krylov error falls geometrically
    with m (about 2e-1, 6e-2, 1.5e-3, 6e-6 at m = 3, 8, 20, 40 here)."""
    mdl, th, Q = _setup(6, 5)
    n = mdl.n
    fac = lz.block_factors(Q, 32)
    Linv = _dense_factor(fac, n)
    lam, U = np.linalg.eigh(Linv @ Q.toarray() @ Linv.T)
    X_ex = Linv.T @ (U * lam ** -0.5) @ U.T @ o.philox_normals(9, 0, n, 1)
    errs = []
    for m in (3, 8, 20, 40):
        X, _, _ = lz.sample(mdl, th, seed=9, k=1, m=m, b=32)
        errs.append(np.linalg.norm(X - X_ex) / np.linalg.norm(X_ex))
    assert errs[0] > errs[1] > errs[2] > errs[3] and errs[3] < 1e-4, errs
