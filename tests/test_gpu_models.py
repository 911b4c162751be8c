"""The diffusion-based space-time model (QSEL_MODEL_DIFFUSION) and user-given
block-tridiagonal precisions (qsel_create_bt) on the GPU against the oracle
(oracle/qsel_diffusion.py: the model, and Algorithm 4 on any
block-tridiagonal precision; oracle/qsel_lanczos.py: the Krylov sampler).

Tolerances as for the separable model: 1e-10 relative in FP64 for the exact
one-part result and for RBMC with injected samples, 1e-10 for the Lanczos
samples (same recurrences, other summation orders), and the stated mixed
tolerance for the mixed dense path."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import qsel_inputs as qi
from oracle import qsel_diffusion as od
from oracle import qsel_lanczos as lz
from oracle import qsel_oracle as o
from tests.test_gpu_mixed import MIXED_DIAG_TOL, MIXED_TRACE_TOL

pytestmark = pytest.mark.gpu

# name: (m, n_t, gamma_s, gamma_t, gamma_e, obs_frac, sigma, slab_start or n_parts, overlap, k)
DIFF = {
    "diff8": (8, 6, 0.5, 1.5, 0.8, 0.3, 0.5, 2, 1, 24),
    "diff9_ragged": (9, 7, 0.9, 2.0, 1.3, 0.25, 0.7, [0, 3, 7], 2, 33),
    "diff24_panels": (24, 5, 0.3, 2.0, 1.0, 0.2, 0.5, 2, 1, 40),
}


@pytest.fixture(scope="module")
def q():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2309_05435_gb300 import build, qsel
    build.build()
    return qsel


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.abs(np.asarray(b))))


class Diff:
    def __init__(self, q, name, seed=5, **over):
        m, n_t, gs, gt, ge, frac, sigma, parts, n_l, k = DIFF[name]
        n_l = over.pop("overlap", n_l)
        parts = over.pop("parts", parts)
        self.k = over.pop("k", k)
        self.mesh = qi.grid_mesh(m)
        self.n_s, self.n_t, self.n_l = m * m, n_t, n_l
        self.mask = qi.obs_mask(self.n_s * n_t, frac, 2)
        self.theta = (math.log(gs), math.log(gt), math.log(ge))
        self.slab_start = np.array(parts) if isinstance(parts, list) else qi.balanced_slab_start(n_t, parts)
        self.model = o.model_from_csr(self.n_s, n_t, self.mesh.c_diag, self.mesh.g_rowptr, self.mesh.g_col,
                                      self.mesh.g_val, self.mask, sigma)
        self.seed = seed
        kw = dict(sampler=q.QSEL_SAMPLER_LANCZOS, lanczos_steps=12)
        kw.update(over)
        self.ctx = q.qsel_create(self.n_s, n_t, self.mesh.c_diag, self.mesh.g_rowptr, self.mesh.g_col,
                                 self.mesh.g_val, self.mask, sigma, self.theta,
                                 n_parts=len(self.slab_start) - 1, slab_start=self.slab_start, overlap=n_l,
                                 n_samples=self.k, seed=seed, model=q.QSEL_MODEL_DIFFUSION, **kw)
        self.Q = od.precision(self.model, self.theta)
        self.dQs = od.precision_derivatives(self.model, self.theta)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(DIFF))
def test_diffusion_single_part_exact(q, name, precision):
    prec = q.QSEL_FP64 if precision == "fp64" else q.QSEL_MIXED
    c = Diff(q, name, parts=1, overlap=0, precision=prec)
    v, t = c.ctx.diag_inv(), c.ctx.trace_grads()
    v_ex, t_ex = o.exact_selinv(c.Q, c.dQs)
    tv, tt = (1e-10, 1e-10) if precision == "fp64" else (MIXED_DIAG_TOL, MIXED_TRACE_TOL)
    print(f"{name} {precision}: diag {rel(v, v_ex):.2e} traces {rel(t, t_ex):.2e}")
    assert rel(v, v_ex) <= tv
    assert rel(t, t_ex) <= tt


@pytest.mark.parametrize("name", list(DIFF))
def test_diffusion_injected_samples_match_oracle(q, name):
    c = Diff(q, name, precision=q.QSEL_FP64)
    X = qi.seeded_normal((c.n_s * c.n_t, c.k), 17)
    q.qsel_debug_set_samples(c.ctx, X)
    v, t = c.ctx.diag_inv(), c.ctx.trace_grads()
    sel = q.qsel_debug_get_selinv_diag(c.ctx)
    v_or, t_or, res = od.rbmc_precision(c.Q, c.dQs, c.n_s, c.n_t, c.slab_start, c.n_l, X)
    sel_or = np.concatenate([r.sigma_star_diag for r in res])
    assert rel(sel, sel_or) <= 1e-10
    assert rel(v, v_or) <= 1e-10
    assert rel(t, t_or) <= 1e-10
    assert np.max(v_or - sel_or) > 1e-3 * np.max(v_or)   # the correction is a real part of the result


@pytest.mark.parametrize("name", ["diff8", "diff9_ragged"])
def test_diffusion_lanczos_samples_and_rbmc(q, name):
    """Algorithm 5.1 on the diffusion precision: samples and the RBMC estimate
    on them against the oracle's sampler and Algorithm 4."""
    m = 12
    c = Diff(q, name, precision=q.QSEL_FP64, lanczos_steps=m, precond_block=16)
    v, t = c.ctx.diag_inv(), c.ctx.trace_grads()
    X = q.qsel_debug_get_samples(c.ctx)
    X_or, _, _ = lz.sample_q(c.Q, c.seed, c.k, m, 16)
    assert np.max(np.abs(X - X_or)) <= 1e-10 * np.max(np.abs(X_or))
    v_or, t_or, _ = od.rbmc_precision(c.Q, c.dQs, c.n_s, c.n_t, c.slab_start, c.n_l, X_or)
    assert rel(v, v_or) <= 1e-10
    assert rel(t, t_or) <= 1e-10


def test_diffusion_needs_the_krylov_sampler(q):
    with pytest.raises(q.QselError) as ei:
        Diff(q, "diff8", sampler=q.QSEL_SAMPLER_PCG)
    assert ei.value.status == 1


def test_diffusion_set_theta(q):
    c = Diff(q, "diff8", precision=q.QSEL_FP64, parts=1, overlap=0)
    th2 = (math.log(0.7), math.log(0.9), math.log(1.6))
    q.qsel_set_theta(c.ctx, th2)
    v = c.ctx.diag_inv()
    v_ex, _ = o.exact_selinv(od.precision(c.model, th2), [])
    assert rel(v, v_ex) <= 1e-10


# ----------------------------------------------------------------------------
# user-given block-tridiagonal matrices
# ----------------------------------------------------------------------------
def bt_inputs(Q, dQs, n_s, n_t):
    """CSR pattern (union over all blocks, with the diagonal) and the block
    values of Q and the derivatives in the layout of qsel_create_bt."""
    blocks = [sp.csr_matrix(o.block(Q, n_s, t, t)) for t in range(n_t)]
    blocks += [sp.csr_matrix(o.block(Q, n_s, t + 1, t)) for t in range(n_t - 1)]
    pat = sp.identity(n_s, format="csr")
    for b in blocks:
        pat = pat + abs(b)
    pat = pat.tocsr()
    pat.sort_indices()
    rowptr, col = pat.indptr.astype(np.int32), pat.indices.astype(np.int32)
    rows = np.repeat(np.arange(n_s), np.diff(rowptr))

    def vals(M, t, u):
        B = o.block(M, n_s, t, u)
        return np.asarray(B[rows, col]).ravel()

    diag = np.stack([vals(Q, t, t) for t in range(n_t)])
    off = np.stack([vals(Q, t + 1, t) for t in range(n_t - 1)])
    dd = np.stack([np.stack([vals(d, t, t) for t in range(n_t)]) for d in dQs]) if dQs else None
    do = np.stack([np.stack([vals(d, t + 1, t) for t in range(n_t - 1)]) for d in dQs]) if dQs else None
    return rowptr, col, diag, off, dd, do


def random_bt(n_s_side=7, n_t=6, seed=3):
    """A block-tridiagonal SPD matrix whose blocks differ from slab to slab:
    the diffusion model's blocks with a seeded per-slab scaling of the
    couplings and a seeded per-slab diagonal shift, and two derivative
    matrices (dQ/da = the shifts' pattern, dQ/db = the coupling scales')."""
    rng = np.random.default_rng(seed)
    mesh = qi.grid_mesh(n_s_side)
    n_s = mesh.n_s
    model = o.model_from_csr(n_s, n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val,
                             qi.obs_mask(n_s * n_t, 0.3, 4), 0.6)
    Q0 = od.precision(model, (math.log(0.6), math.log(1.1), 0.0)).tolil()
    scale = rng.uniform(0.5, 1.2, n_t - 1)
    shift = rng.uniform(0.2, 1.0, n_t)
    Q = Q0.copy()
    dQa = sp.lil_matrix(Q0.shape)
    dQb = sp.lil_matrix(Q0.shape)
    for t in range(n_t):
        sl = slice(t * n_s, (t + 1) * n_s)
        Q[sl, sl] = Q0[sl, sl] + shift[t] * sp.identity(n_s)
        dQa[sl, sl] = (t + 1) * sp.identity(n_s)
    for t in range(n_t - 1):
        a, b = slice((t + 1) * n_s, (t + 2) * n_s), slice(t * n_s, (t + 1) * n_s)
        Q[a, b] = scale[t] * Q0[a, b]
        Q[b, a] = scale[t] * Q0[b, a]
        dQb[a, b] = Q0[a, b]
        dQb[b, a] = Q0[b, a]
    return n_s, n_t, Q.tocsr(), [dQa.tocsr(), dQb.tocsr()]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bt_single_part_exact(q, precision):
    n_s, n_t, Q, dQs = random_bt()
    rowptr, col, diag, off, dd, do = bt_inputs(Q, dQs, n_s, n_t)
    prec = q.QSEL_FP64 if precision == "fp64" else q.QSEL_MIXED
    ctx = q.qsel_create_bt(n_s, n_t, rowptr, col, diag, off, dd, do, n_parts=1, n_samples=4, precision=prec)
    v = ctx.diag_inv()
    t = q.qsel_trace_grads_n(ctx, 2)
    v_ex, t_ex = o.exact_selinv(Q, dQs)
    tv, tt = (1e-10, 1e-10) if precision == "fp64" else (MIXED_DIAG_TOL, MIXED_TRACE_TOL)
    assert rel(v, v_ex) <= tv
    assert rel(t, t_ex) <= tt


@pytest.mark.parametrize("chain", ["two_ended", "forward"])
@pytest.mark.parametrize("n_t", [2, 3, 4, 5, 9])
def test_bt_single_part_both_chains(q, n_t, chain):
    """One part, factored from both ends toward the middle slab n_t // 2 (or,
    for n_t = 2 and with QSEL_CHAIN_FORWARD, in one chain from slab 0): the
    exact selected inverse and traces of the oracle.  The blocks and the
    derivatives differ from slab to slab, so a wrong slab or coupling index in
    either half, or a missing neighbour term of the middle slab, shows."""
    n_s, n_t, Q, dQs = random_bt(n_t=n_t, seed=5)
    rowptr, col, diag, off, dd, do = bt_inputs(Q, dQs, n_s, n_t)
    v_ex, t_ex = o.exact_selinv(Q, dQs)
    ch = q.QSEL_CHAIN_TWO_ENDED if chain == "two_ended" else q.QSEL_CHAIN_FORWARD
    for prec, tv, tt in ((q.QSEL_FP64, 1e-10, 1e-10), (q.QSEL_MIXED, MIXED_DIAG_TOL, MIXED_TRACE_TOL)):
        ctx = q.qsel_create_bt(n_s, n_t, rowptr, col, diag, off, dd, do, n_parts=1, n_samples=4,
                               precision=prec, chain=ch)
        v = ctx.diag_inv()
        t = q.qsel_trace_grads_n(ctx, 2)
        ctx.close()
        assert rel(v, v_ex) <= tv
        assert rel(t, t_ex) <= tt


@pytest.mark.parametrize("parts,n_l", [(2, 1), ([0, 1, 4, 6], 2)])
def test_bt_injected_samples_match_oracle(q, parts, n_l):
    n_s, n_t, Q, dQs = random_bt()
    rowptr, col, diag, off, dd, do = bt_inputs(Q, dQs, n_s, n_t)
    ss = np.array(parts) if isinstance(parts, list) else qi.balanced_slab_start(n_t, parts)
    k = 21
    ctx = q.qsel_create_bt(n_s, n_t, rowptr, col, diag, off, dd, do, n_parts=len(ss) - 1, slab_start=ss,
                           overlap=n_l, n_samples=k, precision=q.QSEL_FP64)
    X = qi.seeded_normal((n_s * n_t, k), 8)
    q.qsel_debug_set_samples(ctx, X)
    v = ctx.diag_inv()
    t = q.qsel_trace_grads_n(ctx, 2)
    v_or, t_or, _ = od.rbmc_precision(Q, dQs, n_s, n_t, ss, n_l, X)
    assert rel(v, v_or) <= 1e-10
    assert rel(t, t_or) <= 1e-10


def test_bt_lanczos_end_to_end_and_new_values(q):
    n_s, n_t, Q, dQs = random_bt(seed=9)
    rowptr, col, diag, off, dd, do = bt_inputs(Q, dQs, n_s, n_t)
    m, k = 10, 16
    ctx = q.qsel_create_bt(n_s, n_t, rowptr, col, diag, off, dd, do, n_parts=2, overlap=1, n_samples=k,
                           precision=q.QSEL_FP64, seed=3, lanczos_steps=m, precond_block=16)
    v = ctx.diag_inv()
    X_or, _, _ = lz.sample_q(Q, 3, k, m, 16)
    v_or, _, _ = od.rbmc_precision(Q, dQs, n_s, n_t, qi.balanced_slab_start(n_t, 2), 1, X_or)
    assert rel(v, v_or) <= 1e-10
    # new values on the same pattern
    n_s2, n_t2, Q2, dQs2 = random_bt(seed=10)
    _, _, diag2, off2, dd2, do2 = bt_inputs(Q2, dQs2, n_s2, n_t2)
    q.qsel_set_bt_values(ctx, diag2, off2, dd2, do2)
    v2 = ctx.diag_inv()
    X2, _, _ = lz.sample_q(Q2, 3, k, m, 16)
    v2_or, _, _ = od.rbmc_precision(Q2, dQs2, n_s, n_t, qi.balanced_slab_start(n_t, 2), 1, X2)
    assert rel(v2, v2_or) <= 1e-10


def test_bt_rejects_invalid_input(q):
    n_s, n_t, Q, dQs = random_bt()
    rowptr, col, diag, off, dd, do = bt_inputs(Q, dQs, n_s, n_t)
    bad = diag.copy()
    bad[0, 1] += 1.0                       # one entry of A_0 without its mirror
    with pytest.raises(q.QselError) as ei:
        q.qsel_create_bt(n_s, n_t, rowptr, col, bad, off, dd, do)
    assert ei.value.status == 1 and "symmetric" in str(ei.value)
    with pytest.raises(q.QselError) as ei:
        q.qsel_create_bt(n_s, n_t, rowptr, col, diag, off, dd, do, sampler=q.QSEL_SAMPLER_PCG)
    assert ei.value.status == 1
    ctx = q.qsel_create_bt(n_s, n_t, rowptr, col, diag, off, dd, do, n_samples=4)
    with pytest.raises(q.QselError) as ei:
        q.qsel_set_theta(ctx, (0.0, 0.0, 0.0))
    assert ei.value.status == 1
    with pytest.raises(q.QselError) as ei:
        ctx.trace_grads()                  # two derivatives, not three
    assert ei.value.status == 1
