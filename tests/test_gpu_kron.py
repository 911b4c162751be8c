"""Kronecker grid preconditioner of the sampler's PCG on the GPU against the
oracle (oracle/qsel_kron.py): the applied M^-1 (FP64, 1e-10 relative), then
the sampler with it: same samples within the PCG tolerance, far fewer
iterations than 64-row block Jacobi."""
import numpy as np
import pytest

import qsel_inputs as qi
from oracle import qsel_kron as kr
from oracle import qsel_oracle as o
from tests.models import theta as mk_theta
from tests.test_gpu_parity import Case, q  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def _grid_ctx(q, m, n_t, k, **kw):
    mesh = qi.grid_mesh(m)
    mask = qi.obs_mask(m * m * n_t, 0.25, 4)
    th = mk_theta(0.3, 1.2, 0.9)
    model = o.model_from_csr(m * m, n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val, mask, 0.5)
    ctx = q.qsel_create(m * m, n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val, mask, 0.5, th,
                        n_parts=2, overlap=1, n_samples=k, seed=3, **kw)
    return ctx, model, th


@pytest.mark.parametrize("m,n_t,k", [(16, 8, 64), (13, 7, 10), (6, 70, 33), (9, 130, 64), (12, 10, 128)])
def test_applied_preconditioner_matches_oracle(q, m, n_t, k):
    """n_t = 70 and 130 take two and three 64-wide K slices in the temporal
    passes; m = 13 and 6 take partial tiles; 128 samples take the 128-column
    tiles."""
    ctx, model, th = _grid_ctx(q, m, n_t, k, preconditioner=q.QSEL_PRECOND_KRON)
    R = qi.seeded_normal((model.n, k), 17)
    Z = q.qsel_debug_apply_precond(ctx, R)
    Z_or = kr.preconditioner_inverse(model, th) @ R
    assert np.max(np.abs(Z - Z_or)) <= 1e-10 * np.max(np.abs(Z_or))


@pytest.mark.parametrize("m,n_t,k", [(16, 8, 128), (12, 20, 128), (8, 68, 256), (16, 8, 64)])
def test_mixed_preconditioner_matches_oracle(q, m, n_t, k):
    """The mixed form's binary32 apply (n_t = 68 and m = 12 take partial
    tiles; 64 and 128 samples), within binary32 accuracy (2e-5 of the
    largest entry) of the oracle's FP64 operator applied to the same
    (rounded) input."""
    ctx, model, th = _grid_ctx(q, m, n_t, k, preconditioner=q.QSEL_PRECOND_KRON, precision=q.QSEL_MIXED)
    R = qi.seeded_normal((model.n, k), 19).astype(np.float32).astype(np.float64)
    Z = q.qsel_debug_apply_precond(ctx, R)
    Z_or = kr.preconditioner_inverse(model, th) @ R
    err = np.max(np.abs(Z - Z_or)) / np.max(np.abs(Z_or))
    print(f"m={m} n_t={n_t} k={k}: mixed apply error {err:.2e}")
    assert err <= 2e-5


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sampler_with_kron_preconditioner(q, precision):
    prec = q.QSEL_FP64 if precision == "fp64" else q.QSEL_MIXED
    name = "grid16_nt8"
    tol = 1e-10
    cb = Case(q, name, precision=prec, pcg_tol=tol)
    ck = Case(q, name, precision=prec, pcg_tol=tol, preconditioner=q.QSEL_PRECOND_KRON)
    vb = cb.ctx.diag_inv()
    vk = ck.ctx.diag_inv()
    itb, itk = cb.ctx.stats()["pcg_iterations"], ck.ctx.stats()["pcg_iterations"]
    print(f"{precision}: PCG iterations block Jacobi {itb}, Kronecker {itk}")
    assert itk < 0.5 * itb
    assert ck.ctx.stats()["pcg_max_rel_residual"] <= tol
    X = q.qsel_debug_get_samples(ck.ctx)
    Q = o.precision(ck.model, ck.theta)
    R = o.rhs(ck.model, ck.theta, ck.seed, ck.k)
    res = np.linalg.norm(R - Q @ X, axis=0) / np.linalg.norm(R, axis=0)
    assert res.max() <= 10 * tol
    # same estimate as with block Jacobi up to the sampler tolerance
    ev = np.linalg.eigvalsh(Q.toarray())
    assert np.max(np.abs(vk - vb) / vb) <= 80 * (ev[-1] / ev[0]) * tol + (1e-4 if precision == "mixed" else 0)
