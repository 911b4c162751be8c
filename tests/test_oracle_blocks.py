"""Pins of the oracle's block Cholesky, Takahashi recursion, block solve and
log-determinant against dense library routines (no GPU)."""
import numpy as np
import pytest

from oracle import qsel_oracle as o
from tests.models import grid_model, theta


def _blocks(Q, n_s, e0, e1):
    diag_b = [o.block(Q, n_s, t, t) for t in range(e0, e1)]
    sub_b = [o.block(Q, n_s, t + 1, t) for t in range(e0, e1 - 1)]
    return diag_b, sub_b


@pytest.mark.parametrize("m,n_t,e0,e1", [(4, 5, 0, 5), (5, 6, 1, 5), (3, 2, 0, 2), (4, 3, 1, 2)])
def test_block_cholesky_matches_dense(m, n_t, e0, e1):
    model = grid_model(m, n_t)
    Q = o.precision(model, theta(0.5, 1.0, 0.9))
    n_s = m * m
    diag_b, sub_b = _blocks(Q, n_s, e0, e1)
    L_diag, L_sub = o.block_cholesky(diag_b, sub_b)
    sl = slice(e0 * n_s, e1 * n_s)
    Ld = np.linalg.cholesky(Q[sl, sl].toarray())
    T = e1 - e0
    for t in range(T):
        np.testing.assert_allclose(L_diag[t], Ld[t * n_s:(t + 1) * n_s, t * n_s:(t + 1) * n_s],
                                   rtol=1e-11, atol=1e-12)
        if t + 1 < T:
            np.testing.assert_allclose(L_sub[t], Ld[(t + 1) * n_s:(t + 2) * n_s, t * n_s:(t + 1) * n_s],
                                       rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("m,n_t,t_stop", [(4, 5, 0), (5, 6, 2), (3, 1, 0)])
def test_block_takahashi_matches_dense_inverse(m, n_t, t_stop):
    model = grid_model(m, n_t)
    Q = o.precision(model, theta(0.7, 1.3, 0.8))
    n_s = m * m
    diag_b, sub_b = _blocks(Q, n_s, 0, n_t)
    L_diag, L_sub = o.block_cholesky(diag_b, sub_b)
    Sd, Ss = o.block_takahashi(L_diag, L_sub, t_stop)
    S = np.linalg.inv(Q.toarray())
    for t in range(t_stop, n_t):
        np.testing.assert_allclose(Sd[t], S[t * n_s:(t + 1) * n_s, t * n_s:(t + 1) * n_s], rtol=1e-10,
                                   atol=1e-12 * np.abs(S).max())
    for t in range(t_stop, n_t - 1):
        np.testing.assert_allclose(Ss[t], S[(t + 1) * n_s:(t + 2) * n_s, t * n_s:(t + 1) * n_s], rtol=1e-9,
                                   atol=1e-12 * np.abs(S).max())
    for t in range(0, t_stop):
        assert Sd[t] is None


def test_block_solve_and_logdet_match_dense():
    model = grid_model(5, 6)
    Q = o.precision(model, theta(0.4, 0.8, 0.95))
    n_s, n_t = 25, 6
    diag_b, sub_b = _blocks(Q, n_s, 0, n_t)
    L_diag, L_sub = o.block_cholesky(diag_b, sub_b)
    rng = np.random.default_rng(3)
    b = rng.standard_normal((Q.shape[0], 4))
    w = np.concatenate(o.block_solve(L_diag, L_sub, [b[t * n_s:(t + 1) * n_s] for t in range(n_t)]))
    np.testing.assert_allclose(w, np.linalg.solve(Q.toarray(), b), rtol=1e-10, atol=1e-12)
    sign, ld = np.linalg.slogdet(Q.toarray())
    assert sign > 0 and abs(o.logdet(Q, n_s, n_t) - ld) < 1e-9 * abs(ld)
