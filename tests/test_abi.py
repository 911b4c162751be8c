"""The C-ABI library builds, loads, exports every symbol include/qsel.h declares,
and rejects invalid arguments before touching the GPU (no compute calls)."""
import os
import re

import numpy as np
import pytest

import qsel_inputs as qi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2309_05435_gb300 import build, qsel
    build.build()
    return qsel.load_library()


def header_functions():
    text = open(os.path.join(ROOT, "include", "qsel.h")).read()
    decl = r"^(?:qsel_status|void|const char \*)\s*\**(qsel_[a-z_]+)\s*\("
    return sorted(set(re.findall(decl, text, flags=re.M)))


def test_exports_every_declared_symbol(lib):
    from paper_2309_05435_gb300 import qsel
    declared = header_functions()
    assert len(declared) >= 11
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(qsel.EXPORTED) == declared


def _args(**over):
    w = qi.workload("grid16_nt8")
    m = w.mesh()
    a = dict(n_s=w.n_s, n_t=w.n_t, c_diag=m.c_diag, g_rowptr=m.g_rowptr, g_col=m.g_col, g_val=m.g_val,
             obs_mask=w.mask(), sigma=w.sigma, theta=w.theta, n_parts=2, overlap=1, n_samples=8)
    a.update(over)
    return a


@pytest.mark.parametrize("bad,msg", [
    (dict(sigma=0.0), "sigma"),
    (dict(n_parts=9), "n_parts"),
    (dict(overlap=-1), "overlap"),
    (dict(n_samples=0), "n_samples"),
    (dict(n_samples=513), "n_samples"),
    (dict(precond_block=8), "precond_block"),
    (dict(slab_start=[0, 3, 3, 8], n_parts=3), "increasing"),
    (dict(slab_start=[0, 5, 7], n_parts=2), "0 to n_t"),
    (dict(theta=(0.0, 0.0, 40.0)), "rho"),
    (dict(pcg_tol=0.0), "pcg_tol"),
    (dict(sampler=2), "sampler"),
    (dict(sampler=1, lanczos_steps=0), "lanczos_steps"),
    (dict(sampler=1, lanczos_steps=8, precond_block=1), "blocks of 16, 32 or 64"),
    (dict(part_overlap=[1, -1]), "part_overlap"),
    (dict(pivot_precision=2), "pivot_precision"),
])
def test_invalid_arguments_rejected(lib, bad, msg):
    from paper_2309_05435_gb300 import qsel
    with pytest.raises(qsel.QselError) as ei:
        qsel.qsel_create(**_args(**bad))
    assert ei.value.status == 1 and msg in str(ei.value)


def test_invalid_mesh_rejected(lib):
    from paper_2309_05435_gb300 import qsel
    a = _args()
    c = a["c_diag"].copy()
    c[3] = 0.0
    with pytest.raises(qsel.QselError, match="c_diag"):
        qsel.qsel_create(**dict(a, c_diag=c))
    col = a["g_col"].copy()
    col[5] = 10 ** 6
    with pytest.raises(qsel.QselError, match="g_col"):
        qsel.qsel_create(**dict(a, g_col=col))


def test_kron_preconditioner_needs_a_grid(lib):
    """QSEL_PRECOND_KRON is refused (before any GPU work) for a mesh that is
    not the m x m grid: here the grid with its nodes renumbered."""
    from paper_2309_05435_gb300 import qsel
    w = qi.workload("grid16_nt8")
    m = w.mesh()
    perm = np.random.default_rng(0).permutation(w.n_s)
    inv = np.argsort(perm)
    G = np.zeros((w.n_s, w.n_s))
    for r in range(w.n_s):
        for p in range(m.g_rowptr[r], m.g_rowptr[r + 1]):
            G[inv[r], inv[m.g_col[p]]] = m.g_val[p]
    rp = np.zeros(w.n_s + 1, np.int32)
    cols, vals = [], []
    for r in range(w.n_s):
        nz = np.flatnonzero(G[r])
        cols += list(nz)
        vals += list(G[r, nz])
        rp[r + 1] = len(cols)
    a = _args(c_diag=m.c_diag[perm], g_rowptr=rp, g_col=np.array(cols, np.int32), g_val=np.array(vals),
              preconditioner=1)
    with pytest.raises(qsel.QselError) as ei:
        qsel.qsel_create(**a)
    assert ei.value.status == 1 and "grid" in str(ei.value)
