"""Preconditioned Krylov (Lanczos) sampler on the GPU against the oracle
(oracle/qsel_lanczos.py): the Lanczos coefficients of every column, the
samples after the quadrature and the preconditioner rewind, the RBMC
estimate built on them, and convergence to exact samples as m grows.

Tolerances (FP64): the coefficients and samples follow the same recurrences
with other summation orders, so they agree to about 1e-12 after a dozen
steps; 1e-10 relative is stated (the FP64 tolerance of every other
parity test)."""
import numpy as np
import pytest

import qsel_inputs as qi
from oracle import qsel_lanczos as lz
from oracle import qsel_oracle as o
from tests.test_gpu_parity import Case, q  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def _run(q, name, m, b=64, precision=None, seed=7):
    kw = dict(sampler=q.QSEL_SAMPLER_LANCZOS, lanczos_steps=m, precond_block=b, seed=seed)
    if precision is not None:
        kw["precision"] = precision
    c = Case(q, name, **kw)
    v = c.ctx.diag_inv()
    return c, v


@pytest.mark.parametrize("name,m,b", [("grid16_nt8", 12, 64), ("ragged13", 10, 32), ("overlap2", 15, 16)])
def test_coefficients_and_samples_match_oracle(q, name, m, b):
    c, _ = _run(q, name, m, b)
    alpha, beta = q.qsel_debug_get_lanczos(c.ctx, m)
    X = q.qsel_debug_get_samples(c.ctx)
    X_or, a_or, b_or = lz.sample(c.model, c.theta, c.seed, c.k, m, b)
    for s in range(c.k):
        np.testing.assert_allclose(alpha[:, s], a_or[s], rtol=1e-10)
        np.testing.assert_allclose(beta[:, s], b_or[s], rtol=1e-10)
    assert np.max(np.abs(X - X_or)) <= 1e-10 * np.max(np.abs(X_or))


def test_rbmc_on_lanczos_samples_matches_oracle(q):
    m = 14
    c, v = _run(q, "grid16_nt8", m)
    t = c.ctx.trace_grads()
    X_or, _, _ = lz.sample(c.model, c.theta, c.seed, c.k, m, 64)
    v_or, t_or, _ = o.rbmc(c.model, c.theta, c.slab_start, c.n_l, X_or)
    assert np.max(np.abs(v - v_or) / v_or) <= 1e-10
    assert np.max(np.abs(t - t_or) / np.abs(t_or)) <= 1e-10


def test_mixed_dense_path_with_lanczos_samples(q):
    """The sampler is FP64 in either form; the mixed form's dense part stays
    within its stated tolerance of the FP64 run on the same samples."""
    c64, v64 = _run(q, "ragged13", 10, 32)
    cm, vm = _run(q, "ragged13", 10, 32, precision=q.QSEL_MIXED)
    np.testing.assert_array_equal(q.qsel_debug_get_samples(cm.ctx), q.qsel_debug_get_samples(c64.ctx))
    assert np.max(np.abs(vm - v64) / v64) <= 1e-4


def test_samples_converge_to_exact_with_m(q):
    """Against the dense L^-T Q~^-1/2 z of the same noise: the error of the
    GPU samples falls geometrically with the Krylov dimension (cond(Q~) is
    about 790 here with 16-row blocks: 0.52, 0.020, 1e-6 at m = 4, 40, 160)."""
    name = "overlap2"
    errs = []
    for m in (4, 40, 160):
        c, _ = _run(q, name, m, 16)
        X = q.qsel_debug_get_samples(c.ctx)
        if m == 4:
            Q = o.precision(c.model, c.theta).tocsr()
            fac = lz.block_factors(Q, 16)
            Linv = np.zeros((c.model.n, c.model.n))
            for r0, _, Li in fac:
                Linv[r0:r0 + Li.shape[0], r0:r0 + Li.shape[0]] = Li
            lam, U = np.linalg.eigh(Linv @ Q.toarray() @ Linv.T)
            X_ex = Linv.T @ (U * lam ** -0.5) @ U.T @ o.philox_normals(c.seed, 0, c.model.n, c.k)
        errs.append(np.linalg.norm(X - X_ex) / np.linalg.norm(X_ex))
    print("Lanczos sample error by m:", errs)
    assert errs[0] > errs[1] > errs[2] and errs[1] < 0.05 and errs[2] < 1e-5


def test_lanczos_state_errors(q):
    c = Case(q, "grid16_nt8")
    c.ctx.diag_inv()
    with pytest.raises(q.QselError) as e:
        q.qsel_debug_get_lanczos(c.ctx, 4)
    assert e.value.status == 7
