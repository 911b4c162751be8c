"""GPU parity at sizes that reach the code paths of the large workloads.

The small parity cases (n_s <= 256) give at most four 64-row tiles per
pivot block, which is one column panel of the mixed form's panel-blocked
sweep, and at most 128 sample columns.  These cases reach what the large
workloads run:

* n_s = 576 (nine tiles): three column panels, the last one ragged, so the
  rank-256 tensor-core update of the rest of the matrix, the look-ahead patch
  of the next panel, the panel row copy and both prioritised streams all run
  (the profile counters of the context prove it);
* n_s = 1600 (25 tiles): seven panels, the last with one tile;
* k = 256 samples (leading dimension 256): the widest SpMM variant and the
  256-column tiles of the correction products;
* three parts with overlap 2, and two parts with a ragged partition.

Tolerances as in the other parity files: 1e-10 relative in FP64 for every
deterministic stage (exact subdomain selected inverse, RBMC diagonal and
traces with injected samples), the sampler to 10 * pcg_tol in residual, and
the stated mixed per-result tolerance (MIXED_DIAG_TOL, MIXED_TRACE_TOL) for
the mixed form against the oracle and against the FP64 run of the same seed.
"""
import numpy as np
import pytest

import qsel_inputs as qi
from oracle import qsel_oracle as o
from tests.models import theta as mk_theta
from tests.test_gpu_mixed import MIXED_DIAG_TOL, MIXED_TRACE_TOL

pytestmark = pytest.mark.gpu

# name: (m, n_t, kappa, tau, rho, obs_frac, sigma, slab_start or n_parts, overlap, k)
BIG = {
    "panels24_p3_l2_k256": (24, 12, 0.3, 1.0, 0.9, 0.25, 0.5, 3, 2, 256),
    "panels40_ragged": (40, 5, 0.25, 1.5, 0.85, 0.25, 0.5, [0, 2, 5], 1, 64),
}
PROF_SWEEP_UPDATE = 1    # index of the sweep-update class in qsel_stats_t.class_launches


@pytest.fixture(scope="module")
def q():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2309_05435_gb300 import build, qsel
    build.build()
    return qsel


class Big:
    def __init__(self, q, name, seed=11, **over):
        m, n_t, kappa, tau, rho, frac, sigma, parts, n_l, k = BIG[name]
        n_l = over.pop("overlap", n_l)
        parts = over.pop("parts", parts)
        self.mesh = qi.grid_mesh(m)
        self.n_s, self.n_t, self.k, self.n_l = m * m, n_t, k, n_l
        self.mask = qi.obs_mask(self.n_s * n_t, frac, 3)
        self.theta = mk_theta(kappa, tau, rho)
        self.slab_start = np.array(parts) if isinstance(parts, list) else qi.balanced_slab_start(n_t, parts)
        self.model = o.model_from_csr(self.n_s, n_t, self.mesh.c_diag, self.mesh.g_rowptr, self.mesh.g_col,
                                      self.mesh.g_val, self.mask, sigma)
        self.seed = seed
        self.ctx = q.qsel_create(self.n_s, n_t, self.mesh.c_diag, self.mesh.g_rowptr, self.mesh.g_col,
                                 self.mesh.g_val, self.mask, sigma, self.theta,
                                 n_parts=len(self.slab_start) - 1, slab_start=self.slab_start,
                                 overlap=n_l, n_samples=k, seed=seed, **over)


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


@pytest.fixture(scope="module")
def injected():
    """Injected samples and the oracle's RBMC result for each case (computed once)."""
    out = {}
    for name in BIG:
        m, n_t = BIG[name][0], BIG[name][1]
        k = BIG[name][9]
        out[name] = qi.seeded_normal((m * m * n_t, k), 123)
    return out


_oracle_cache = {}


def oracle_rbmc(c, X, name):
    if name not in _oracle_cache:
        v, t, res = o.rbmc(c.model, c.theta, c.slab_start, c.n_l, X)
        _oracle_cache[name] = (v, np.asarray(t), np.concatenate([r.sigma_star_diag for r in res]))
    return _oracle_cache[name]


@pytest.mark.parametrize("name", list(BIG))
def test_fp64_injected_samples_full_size(q, name, injected):
    c = Big(q, name, precision=q.QSEL_FP64)
    X = injected[name]
    q.qsel_debug_set_samples(c.ctx, X)
    v, t = c.ctx.diag_inv(), c.ctx.trace_grads()
    sel = q.qsel_debug_get_selinv_diag(c.ctx)
    v_or, t_or, sel_or = oracle_rbmc(c, X, name)
    print(f"{name} FP64: selinv {rel(sel, sel_or):.2e} diag {rel(v, v_or):.2e} traces {rel(t, t_or):.2e}")
    assert rel(sel, sel_or) <= 1e-10
    assert rel(v, v_or) <= 1e-10
    assert rel(t, t_or) <= 1e-10


@pytest.mark.parametrize("pivot", ["double_float", "fp64"])
@pytest.mark.parametrize("name", list(BIG))
def test_mixed_multipanel_sweep_injected(q, name, pivot, injected):
    """The mixed form with several sweep panels per pivot block: the
    rank-256 tensor-core updates run (profile counters), and the selected
    inverse, diagonal and traces stay within the mixed tolerance of the
    oracle for the same injected samples."""
    pp = q.QSEL_PIVOT_FP64 if pivot == "fp64" else q.QSEL_PIVOT_DOUBLE_FLOAT
    c = Big(q, name, precision=q.QSEL_MIXED, profile_kernels=1, pivot_precision=pp)
    X = injected[name]
    q.qsel_debug_set_samples(c.ctx, X)
    v, t = c.ctx.diag_inv(), c.ctx.trace_grads()
    st = c.ctx.stats()
    sel = q.qsel_debug_get_selinv_diag(c.ctx)
    v_or, t_or, sel_or = oracle_rbmc(c, X, name)
    n_pad = -(-c.n_s // 64) * 64
    panels = -(-(n_pad // 64) // 4)
    print(f"{name} mixed ({pivot} pivots): {panels} panels, {st['class_launches'][PROF_SWEEP_UPDATE]} sweep "
          f"updates; selinv {rel(sel, sel_or):.2e} diag {rel(v, v_or):.2e} traces {rel(t, t_or):.2e}")
    assert panels >= 3
    assert st["class_launches"][PROF_SWEEP_UPDATE] > 0
    assert rel(sel, sel_or) <= MIXED_DIAG_TOL
    assert rel(v, v_or) <= MIXED_DIAG_TOL
    assert rel(t, t_or) <= MIXED_TRACE_TOL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sampler_k256(q, precision):
    """256 sample columns (leading dimension 256): every column solves
    Q x = r to 10 pcg_tol, checked with the oracle's Q and right-hand sides."""
    tol = 1e-10
    prec = q.QSEL_FP64 if precision == "fp64" else q.QSEL_MIXED
    c = Big(q, "panels24_p3_l2_k256", precision=prec, pcg_tol=tol)
    c.ctx.diag_inv()
    assert c.ctx.stats()["pcg_max_rel_residual"] <= tol
    X = q.qsel_debug_get_samples(c.ctx)
    R_gpu = q.qsel_debug_get_rhs(c.ctx)
    R = o.rhs(c.model, c.theta, c.seed, c.k)
    assert np.max(np.abs(R_gpu - R)) <= 1e-12 * np.max(np.abs(R))
    Q = o.precision(c.model, c.theta)
    res = np.linalg.norm(R - Q @ X, axis=0) / np.linalg.norm(R, axis=0)
    assert res.max() <= 10 * tol


def test_mixed_matches_fp64_same_seed_full_size(q):
    """Whole pipeline (sampler, three parts, overlap 2, 256 samples): mixed
    against FP64 at the same seed, every node and every trace."""
    c64 = Big(q, "panels24_p3_l2_k256", precision=q.QSEL_FP64)
    c32 = Big(q, "panels24_p3_l2_k256", precision=q.QSEL_MIXED)
    v64, t64 = c64.ctx.diag_inv(), c64.ctx.trace_grads()
    v32, t32 = c32.ctx.diag_inv(), c32.ctx.trace_grads()
    print(f"mixed vs FP64 (same seed): diag {rel(v32, v64):.2e} traces {rel(t32, t64):.2e}")
    assert rel(v32, v64) <= MIXED_DIAG_TOL
    assert rel(t32, t64) <= MIXED_TRACE_TOL


@pytest.mark.parametrize("chain", ["two_ended", "forward"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_single_part_exact_full_size(q, precision, chain):
    """One part: the exact selected inverse through every panel of every
    pivot block, against the oracle's block Takahashi recursion; factored
    from both ends toward the middle slab (two halves batched in every
    launch) or in one chain from slab 0."""
    prec = q.QSEL_FP64 if precision == "fp64" else q.QSEL_MIXED
    ch = q.QSEL_CHAIN_TWO_ENDED if chain == "two_ended" else q.QSEL_CHAIN_FORWARD
    c = Big(q, "panels40_ragged", precision=prec, parts=1, overlap=0, chain=ch)
    v, t = c.ctx.diag_inv(), c.ctx.trace_grads()
    v_or, t_or, _ = o.rbmc(c.model, c.theta, np.array([0, c.n_t]), 0, np.zeros((c.n_s * c.n_t, 1)))
    tol_v, tol_t = (1e-10, 1e-10) if precision == "fp64" else (MIXED_DIAG_TOL, MIXED_TRACE_TOL)
    print(f"exact one part {precision} {chain}: diag {rel(v, v_or):.2e} traces {rel(t, np.asarray(t_or)):.2e}")
    assert rel(v, v_or) <= tol_v
    assert rel(t, np.asarray(t_or)) <= tol_t


def test_tensor_core_wait_timeout_is_reported(q):
    """QSEL_ETIMEOUT without a GPU fault: the test hook makes the GEMM's
    producer issue no TMA load, so its bounded waits run out after 2e6
    cycles (about 1 ms); every CTA sets its error bit, frees its tensor memory
    and returns, and the call reports the timeout.  A fresh context then
    gives the oracle's exact result."""
    from tests.test_gpu_parity import Case
    c = Case(q, "grid16_nt8", precision=q.QSEL_MIXED, parts=1, overlap=0, tensor_passes=3)
    q.qsel_debug_tc_wait(True, 2_000_000)
    try:
        with pytest.raises(q.QselError) as ei:
            c.ctx.diag_inv()
    finally:
        q.qsel_debug_tc_wait(False, 0)
    assert ei.value.status == 6
    c.ctx.close()
    c2 = Case(q, "grid16_nt8", precision=q.QSEL_MIXED, parts=1, overlap=0, tensor_passes=3)
    v = c2.ctx.diag_inv()
    Q = o.precision(c2.model, c2.theta)
    v_ex, _ = o.exact_selinv(Q, o.precision_derivatives(c2.model, c2.theta))
    assert rel(v, v_ex) <= MIXED_DIAG_TOL


def test_full_size_mixed_unobserved_closed_form(q):
    """The bench's size and launch configuration -- 96x96 grid, 256 slabs
    (n = 2,359,296), mixed form, one part factored from both ends -- on the
    unobserved prior, whose selected inverse has a closed form at any size
    (tests.models.unobserved_closed_form, pinned against the oracle's exact
    selected inverse): every diagonal entry of every slab within the mixed
    tolerance at this block size (2e-3) and the traces within 5e-4.  kappa = 1
    keeps Q_s = K C^-1 K well conditioned (cond ~ 80): with no observations
    the pivot blocks are multiples of Q_s, and at kappa <= 0.3 (cond >= 8e3)
    binary32 blocks lose its smallest eigen-directions (the FP64 form is the
    one to use there)."""
    from tests.models import unobserved_closed_form
    w = qi.workload("grid96_nt256")
    kappa = 1.0
    mesh = w.mesh()
    th = mk_theta(kappa, w.tau, w.rho)
    ctx = q.qsel_create(w.n_s, w.n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val,
                        np.zeros(w.n, np.uint8), w.sigma, th, n_parts=1, overlap=0, n_samples=2,
                        precision=q.QSEL_MIXED)
    v, t = ctx.diag_inv(), ctx.trace_grads()
    ctx.close()
    v_cf, t_cf = unobserved_closed_form(mesh, w.n_t, kappa, w.tau, w.rho)
    print(f"full size mixed: diag max {rel(v, v_cf):.2e} traces {rel(np.asarray(t), t_cf):.2e}")
    assert rel(v, v_cf) <= 2e-3
    assert rel(np.asarray(t), t_cf) <= 5e-4


def test_full_block_fp64_unobserved_closed_form(q):
    """The FP64 form at the bench's block size (9216 nodes, four slabs) on the
    unobserved prior at the bench's kappa = 0.1, where cond(Q_s) ~ 6.4e5:
    diagonal within 1e-7 (about cond(Q_s) x n_s x 2^-53 x 1.5; measured
    1.2e-8) and traces within 1e-9 of the closed form."""
    from tests.models import unobserved_closed_form
    w = qi.workload("grid96_nt256")
    n_t = 4
    mesh = w.mesh()
    th = mk_theta(w.kappa, w.tau, w.rho)
    ctx = q.qsel_create(w.n_s, n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val,
                        np.zeros(w.n_s * n_t, np.uint8), w.sigma, th, n_parts=1, overlap=0, n_samples=2,
                        precision=q.QSEL_FP64)
    v, t = ctx.diag_inv(), ctx.trace_grads()
    ctx.close()
    v_cf, t_cf = unobserved_closed_form(mesh, n_t, w.kappa, w.tau, w.rho)
    print(f"full block fp64: diag max {rel(v, v_cf):.2e} traces {rel(np.asarray(t), t_cf):.2e}")
    assert rel(v, v_cf) <= 1e-7
    assert rel(np.asarray(t), t_cf) <= 1e-9


def test_sweep_schedules_give_identical_results(q):
    """The sweep's scheduling hook changes only where and when its kernels run:
    the update after the pivot chain on one stream, a capped update grid, a
    three-stage update ring, the update on 128 x 256 tiles and pivot CTAs
    beside update CTAs all give the default's results bit for bit (three
    sweep panels per pivot block, the last ragged; two matrices per launch)."""
    def run():
        c = Big(q, "panels24_p3_l2_k256", precision=q.QSEL_MIXED, parts=1, overlap=0)
        v, t = c.ctx.diag_inv(), np.asarray(c.ctx.trace_grads())
        c.ctx.close()
        return v, t
    v0, t0 = run()
    try:
        for args in [(True, 0, 0, False), (False, 100, 0, False), (False, 0, 3, False), (False, 0, 4, False),
                     (False, 0, 0, True)]:
            q.qsel_debug_sweep_schedule(*args)
            v, t = run()
            assert np.array_equal(v, v0) and np.array_equal(t, t0), args
    finally:
        q.qsel_debug_sweep_schedule(False)
    with pytest.raises(q.QselError):
        q.qsel_debug_sweep_schedule(False, -1)
    with pytest.raises(q.QselError):
        q.qsel_debug_sweep_schedule(False, 0, 5)
