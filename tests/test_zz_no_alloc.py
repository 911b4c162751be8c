"""The allocation-free entry point qsel_spd_inverse_noalloc, checked against
the library's regular path.

Callers inside a framework whose caching allocator owns the device memory
budget, or services that must keep their device memory footprint fixed after
start-up, cannot let the library call cudaMalloc.  For them the library
offers one SPD inverse that works in caller-owned device memory with a fixed,
shared scratch array.  A one-slab,
one-part model makes the regular path (qsel_diag_inv) return exactly
diag(A^-1) for the pivot block A = tau Q_t[0,0] Q_s + A_obs^T A_obs / sigma^2,
so the diagonal of the no-alloc inverse of that same A must match it to the
FP64 tolerance of the other parity tests (1e-10 relative).  Two calls in a
row (different sizes and theta) check that the shared scratch carries no
state from one call into the next.

This file is named to be collected last.
"""
import numpy as np
import pytest

import qsel_inputs as qi
from oracle import qsel_oracle as o
from tests.models import theta as mk_theta

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2309_05435_gb300 import build, qsel
    build.build()
    return qsel


def _regular_diag(q, m, th, seed):
    """diag(A^-1) from the existing entry point on a one-slab, one-part model,
    and the dense A for the no-alloc call."""
    mesh = qi.grid_mesh(m)
    n_s = m * m
    mask = qi.obs_mask(n_s, 0.3, seed)
    ctx = q.qsel_create(n_s, 1, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val, mask, 0.5, th,
                        n_parts=1, overlap=0, n_samples=1)
    d = ctx.diag_inv()
    ctx.close()
    model = o.model_from_csr(n_s, 1, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val, mask, 0.5)
    A = o.precision(model, th).toarray()
    return d, A


def test_noalloc_inverse_matches_regular_path_twice(q):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    for m, th, seed in ((13, mk_theta(0.6, 1.3, 0.8), 2), (20, mk_theta(0.3, 0.7, 0.95), 5)):
        d_reg, A = _regular_diag(q, m, th, seed)
        n = A.shape[0]
        lda = n + 3                               # a leading dimension larger than n
        buf = torch.zeros((n, lda), dtype=torch.float64, device="cuda")
        buf[:, :n] = torch.from_numpy(A).cuda()
        torch.cuda.synchronize()
        q.qsel_spd_inverse_noalloc(buf, n, lda, cuda_stream=stream)
        inv = buf[:, :n].cpu().numpy()
        assert np.max(np.abs(np.diag(inv) - d_reg) / d_reg) <= 1e-10
        # the full inverse is symmetric and inverts A
        assert np.max(np.abs(inv - inv.T)) <= 1e-12 * np.max(np.abs(inv))
        assert np.max(np.abs(A @ inv - np.eye(n))) <= 1e-9
        # the padding columns beyond n were left alone
        assert torch.count_nonzero(buf[:, n:]).item() == 0


def test_noalloc_rejects_oversize(q):
    import torch
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(q.QselError) as ei:
        q.qsel_spd_inverse_noalloc(buf, q.QSEL_NOALLOC_MAX_N + 1)
    assert ei.value.status == 1 and "QSEL_NOALLOC_MAX_N" in str(ei.value)
