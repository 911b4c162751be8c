"""GPU parity: the CUDA path through the C ABI against the CPU oracle, stage by
stage, on the same seeded inputs.

FP64 tolerances: 1e-10 relative for everything that is a deterministic
function of the inputs (perturbation RHS, exact subdomain selected inverse,
RBMC diagonal and traces given injected samples).  The GPU sampler is
iterative (PCG to relative residual pcg_tol) while the oracle solves
directly, so samples agree to cond(Q) * pcg_tol and the end-to-end results to
the tolerance that this implies (derived in test_end_to_end_matches_oracle).
"""
import numpy as np
import pytest

import qsel_inputs as qi
from oracle import qsel_oracle as o
from tests.models import theta as mk_theta

pytestmark = pytest.mark.gpu

# name: (m, n_t, kappa, tau, rho, obs_frac, sigma, slab_start or n_parts, overlap, k)
CASES = {
    "grid16_nt8": (16, 8, 0.5, 1.0, 0.9, 0.30, 0.5, 2, 1, 64),
    "ragged13": (13, 7, 0.6, 1.3, 0.8, 0.30, 0.5, [0, 2, 5, 7], 1, 10),
    "overlap2": (9, 9, 0.4, 0.7, 0.95, 0.25, 0.5, 3, 2, 33),
    "uneven4": (8, 10, 0.8, 2.0, 0.7, 0.20, 0.8, 4, 1, 70),
}


@pytest.fixture(scope="module")
def q():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2309_05435_gb300 import build, qsel
    build.build()
    return qsel


class Case:
    def __init__(self, q, name, seed=7, **over):
        m, n_t, kappa, tau, rho, frac, sigma, parts, n_l, k = CASES[name]
        over_k = over.pop("k", k)
        n_l = over.pop("overlap", n_l)
        parts = over.pop("parts", parts)
        self.mesh = qi.grid_mesh(m)
        self.n_s, self.n_t, self.k, self.n_l = m * m, n_t, over_k, n_l
        self.mask = qi.obs_mask(self.n_s * n_t, frac, 1)
        self.theta = mk_theta(kappa, tau, rho)
        self.sigma = sigma
        if isinstance(parts, list):
            self.slab_start = np.array(parts)
        else:
            self.slab_start = qi.balanced_slab_start(n_t, parts)
        self.model = o.model_from_csr(self.n_s, n_t, self.mesh.c_diag, self.mesh.g_rowptr, self.mesh.g_col,
                                      self.mesh.g_val, self.mask, sigma)
        self.seed = seed
        self.ctx = q.qsel_create(self.n_s, n_t, self.mesh.c_diag, self.mesh.g_rowptr, self.mesh.g_col,
                                 self.mesh.g_val, self.mask, sigma, self.theta,
                                 n_parts=len(self.slab_start) - 1, slab_start=self.slab_start,
                                 overlap=n_l, n_samples=self.k, seed=seed, **over)


def rel_err(a, b):
    return np.max(np.abs(a - b) / np.abs(b))


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_matches_oracle(q, name):
    c = Case(q, name)
    c.ctx.diag_inv()
    R_gpu = q.qsel_debug_get_rhs(c.ctx)
    R_or = o.rhs(c.model, c.theta, c.seed, c.k)
    # same Philox words; Box-Muller log/cos evaluated by CUDA vs libm (~1 ulp)
    assert np.max(np.abs(R_gpu - R_or)) <= 1e-12 * np.max(np.abs(R_or))


@pytest.mark.parametrize("name", list(CASES))
def test_single_subdomain_exact(q, name):
    """One part: no separator, exact selected inverse (Section 3.2.2)."""
    c = Case(q, name, parts=1, overlap=0)
    v = c.ctx.diag_inv()
    t = c.ctx.trace_grads()
    Q = o.precision(c.model, c.theta)
    v_ex, t_ex = o.exact_selinv(Q, o.precision_derivatives(c.model, c.theta))
    assert rel_err(v, v_ex) <= 1e-10
    assert rel_err(t, np.array(t_ex)) <= 1e-10


@pytest.mark.parametrize("name", list(CASES))
def test_injected_samples_match_oracle(q, name):
    """Stages (i) and (ii): exact subdomain selected inverse, then the RBMC
    diagonal and traces for the same injected samples X."""
    c = Case(q, name)
    X = qi.seeded_normal((c.n_s * c.n_t, c.k), 99)
    q.qsel_debug_set_samples(c.ctx, X)
    v = c.ctx.diag_inv()
    t = c.ctx.trace_grads()
    sel = q.qsel_debug_get_selinv_diag(c.ctx)
    v_or, t_or, res = o.rbmc(c.model, c.theta, c.slab_start, c.n_l, X)
    sel_or = np.concatenate([r.sigma_star_diag for r in res])
    assert rel_err(sel, sel_or) <= 1e-10
    assert rel_err(v, v_or) <= 1e-10
    assert rel_err(t, t_or) <= 1e-10
    # the correction is a real part of the result
    assert np.max(v_or - sel_or) > 1e-3 * np.max(v_or)


def test_diag_only_without_overlap(q):
    c = Case(q, "grid16_nt8", overlap=0)
    X = qi.seeded_normal((c.n_s * c.n_t, c.k), 5)
    q.qsel_debug_set_samples(c.ctx, X)
    v = c.ctx.diag_inv()
    v_or, _, _ = o.rbmc(c.model, c.theta, c.slab_start, 0, X)
    assert rel_err(v, v_or) <= 1e-10
    with pytest.raises(q.QselError) as ei:
        c.ctx.trace_grads()
    assert ei.value.status == 1


@pytest.mark.parametrize("name", ["grid16_nt8", "ragged13"])
def test_sampler_matches_oracle(q, name):
    """Stage (iii): every GPU sample column solves Q x = r to pcg_tol, checked
    with the oracle's Q and r; samples agree with the oracle's direct solve to
    within 10 cond(Q) pcg_tol."""
    tol = 1e-10
    c = Case(q, name, pcg_tol=tol)
    c.ctx.diag_inv()
    st = c.ctx.stats()
    assert st["pcg_max_rel_residual"] <= tol
    X = q.qsel_debug_get_samples(c.ctx)
    Q = o.precision(c.model, c.theta)
    R = o.rhs(c.model, c.theta, c.seed, c.k)
    res = np.linalg.norm(R - Q @ X, axis=0) / np.linalg.norm(R, axis=0)
    assert res.max() <= 10 * tol
    ev = np.linalg.eigvalsh(Q.toarray())
    cond = ev[-1] / ev[0]
    X_or = o.solve_direct(c.model, c.theta, R)
    assert np.linalg.norm(X - X_or) / np.linalg.norm(X_or) <= 10 * cond * tol


@pytest.mark.parametrize("name", ["grid16_nt8", "overlap2"])
def test_end_to_end_matches_oracle(q, name):
    """Stage (iv): full GPU pipeline against the oracle with its own exact
    samples.  v_hat depends on the samples through (1/k) sum w^2, so a relative
    sample difference eps moves the correction by about 2 eps; with
    eps <= 10 cond(Q) tol (stage iii) the diagonal and traces agree to
    4 * 10 * cond(Q) * tol relative."""
    tol = 1e-10
    c = Case(q, name, pcg_tol=tol)
    v = c.ctx.diag_inv()
    t = c.ctx.trace_grads()
    Q = o.precision(c.model, c.theta)
    ev = np.linalg.eigvalsh(Q.toarray())
    bound = 4 * 10 * (ev[-1] / ev[0]) * tol
    X_or = o.samples(c.model, c.theta, c.seed, c.k)
    v_or, t_or, _ = o.rbmc(c.model, c.theta, c.slab_start, c.n_l, X_or)
    assert rel_err(v, v_or) <= bound
    assert rel_err(t, t_or) <= bound


@pytest.mark.parametrize("block", [1, 16, 32, 64])
def test_preconditioner_blocks_converge(q, block):
    tol = 1e-10
    c = Case(q, "ragged13", pcg_tol=tol, precond_block=block)
    c.ctx.diag_inv()
    X = q.qsel_debug_get_samples(c.ctx)
    Q = o.precision(c.model, c.theta)
    R = o.rhs(c.model, c.theta, c.seed, c.k)
    res = np.linalg.norm(R - Q @ X, axis=0) / np.linalg.norm(R, axis=0)
    assert res.max() <= 10 * tol


def test_device_output_and_set_theta(q):
    import torch
    c = Case(q, "grid16_nt8")
    v_host = c.ctx.diag_inv()
    out = torch.empty(c.n_s * c.n_t, dtype=torch.float64, device="cuda")
    c.ctx.diag_inv(out)
    assert np.array_equal(out.cpu().numpy(), v_host)
    th2 = mk_theta(0.3, 1.5, 0.6)
    q.qsel_set_theta(c.ctx, th2)
    X = qi.seeded_normal((c.n_s * c.n_t, c.k), 3)
    q.qsel_debug_set_samples(c.ctx, X)
    v2 = c.ctx.diag_inv()
    v_or, _, _ = o.rbmc(c.model, th2, c.slab_start, c.n_l, X)
    assert rel_err(v2, v_or) <= 1e-10


def test_errors_reported_not_faulted(q):
    """Failures come back as status codes: too few PCG iterations gives
    QSEL_ENOCONV; a singular pivot block (K = 0, no observations) gives
    QSEL_ENOTSPD from the pivot flag; the context stays usable."""
    c = Case(q, "grid16_nt8", pcg_max_iter=2)
    with pytest.raises(q.QselError) as ei:
        c.ctx.diag_inv()
    assert ei.value.status == 5
    m = qi.grid_mesh(4)
    g_zero = np.zeros(16)
    rowptr = np.arange(17, dtype=np.int32)
    col = np.arange(16, dtype=np.int32)
    g_val = -1.0 * m.c_diag          # K = kappa^2 C + G = 0 for kappa = 1
    ctx = q.qsel_create(16, 3, m.c_diag, rowptr, col, g_val, np.zeros(48, np.uint8), 1.0,
                        (0.0, 0.0, 0.0), n_parts=1, overlap=0, n_samples=4)
    with pytest.raises(q.QselError) as ei:
        ctx.diag_inv()
    assert ei.value.status == 4
    del g_zero
