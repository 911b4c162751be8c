"""Batch of independent models under one captured graph.

The graph replays exactly the kernels of the single-context pipeline in the
same order, with the sampler's convergence checks moved to the device
(conditional while nodes, checked every 8 iterations like the host loop), so
its results equal those of separate contexts bit for bit; those are checked
against the oracle in test_gpu_parity.py / test_gpu_mixed.py, and one batch
model is also checked end to end against the oracle here."""
import numpy as np
import pytest

import qsel_inputs as qi
from oracle import qsel_oracle as o
from tests.models import theta as mk_theta
from tests.test_gpu_parity import q  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

# (m, n_t, n_parts, kappa, tau, rho)
SPECS = [(12, 9, 2, 0.6, 1.0, 0.9), (8, 14, 3, 0.9, 0.7, 0.8), (16, 6, 2, 0.5, 1.5, 0.7),
         (10, 11, 4, 0.4, 1.2, 0.95), (9, 7, 2, 1.2, 0.8, 0.6)]


def _models(specs=SPECS):
    out = []
    for i, (m, n_t, n_p, kappa, tau, rho) in enumerate(specs):
        mesh = qi.grid_mesh(m)
        out.append({"n_s": m * m, "n_t": n_t, "c_diag": mesh.c_diag, "g_rowptr": mesh.g_rowptr,
                    "g_col": mesh.g_col, "g_val": mesh.g_val, "obs_mask": qi.obs_mask(m * m * n_t, 0.25, 10 + i),
                    "sigma": 0.5, "theta": mk_theta(kappa, tau, rho), "n_parts": n_p})
    return out


def _single(q, mdl, i, **kw):
    c = q.qsel_create(mdl["n_s"], mdl["n_t"], mdl["c_diag"], mdl["g_rowptr"], mdl["g_col"], mdl["g_val"],
                      mdl["obs_mask"], mdl["sigma"], kw.pop("theta", mdl["theta"]), n_parts=mdl["n_parts"],
                      overlap=1, seed=kw.pop("seed") + i, **kw)
    return c.diag_inv(), c.trace_grads(), c.stats()["pcg_iterations"]


def _batch(q, models, **kw):
    return q.qsel_create_batch(models, [m["theta"] for m in models], [(m["n_parts"], None) for m in models],
                               [1] * len(models), **kw)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_separate_contexts(q, precision):
    prec = q.QSEL_FP64 if precision == "fp64" else q.QSEL_MIXED
    models = _models()
    opts = dict(n_samples=40, seed=3, precision=prec, pcg_tol=1e-9, pcg_max_iter=4000)
    b = _batch(q, models, n_streams=3, **opts)
    q.qsel_batch_run(b)
    info = q.qsel_batch_info(b)
    print(f"{precision}: replay {info['ms_replay']:.2f} ms, capture {info['ms_capture']:.1f} ms, "
          f"{info['launches_per_replay']} launches captured")
    for i, mdl in enumerate(models):
        v, t, it = _single(q, mdl, i, **opts)
        vb = q.qsel_batch_diag_inv(b, i)
        tb = q.qsel_batch_trace_grads(b, i)
        assert q.qsel_batch_stats(b, i)["pcg_iterations"] == it
        np.testing.assert_array_equal(vb, v)
        np.testing.assert_array_equal(tb, t)


def test_replay_with_new_theta(q):
    models = _models()
    opts = dict(n_samples=32, seed=5, precision=q.QSEL_MIXED, pcg_tol=1e-9, pcg_max_iter=4000)
    b = _batch(q, models, n_streams=2, **opts)
    q.qsel_batch_run(b)
    th = mk_theta(0.7, 0.9, 0.85)
    q.qsel_batch_set_theta(b, 1, th)
    q.qsel_batch_run(b)
    v, t, _ = _single(q, models[1], 1, theta=th, **opts)
    np.testing.assert_array_equal(q.qsel_batch_diag_inv(b, 1), v)
    np.testing.assert_array_equal(q.qsel_batch_trace_grads(b, 1), t)
    # the other models are unchanged by the replay
    v0, _, _ = _single(q, models[0], 0, **opts)
    np.testing.assert_array_equal(q.qsel_batch_diag_inv(b, 0), v0)


def test_batch_model_against_oracle(q):
    """End to end against the oracle's direct solve (FP64), at the bound
    implied by the PCG tolerance (as in test_gpu_parity.py)."""
    models = _models(SPECS[:2])
    tol = 1e-10
    b = _batch(q, models, n_samples=24, seed=7, precision=q.QSEL_FP64, pcg_tol=tol, n_streams=2)
    for i, mdl in enumerate(models):
        model = o.model_from_csr(mdl["n_s"], mdl["n_t"], mdl["c_diag"], mdl["g_rowptr"], mdl["g_col"],
                                 mdl["g_val"], mdl["obs_mask"], mdl["sigma"])
        ss = qi.balanced_slab_start(mdl["n_t"], mdl["n_parts"])
        X = o.samples(model, mdl["theta"], 7 + i, 24)
        v_or, t_or, _ = o.rbmc(model, mdl["theta"], ss, 1, X)
        ev = np.linalg.eigvalsh(o.precision(model, mdl["theta"]).toarray())
        bound = 40 * (ev[-1] / ev[0]) * tol
        v = q.qsel_batch_diag_inv(b, i)
        t = q.qsel_batch_trace_grads(b, i)
        assert np.max(np.abs(v - v_or) / v_or) <= bound
        assert np.max(np.abs(t - t_or) / np.abs(t_or)) <= bound


def test_batch_reports_nonconvergence(q):
    models = _models(SPECS[:3])
    b = _batch(q, models, n_samples=32, seed=1, precision=q.QSEL_FP64, pcg_tol=1e-12, pcg_max_iter=8,
               n_streams=2)
    with pytest.raises(q.QselError) as e:
        q.qsel_batch_run(b)
    assert e.value.status == 5 and "model" in str(e.value)


def test_autotune_choices(q):
    models = _models()
    opts = dict(n_samples=32, seed=2, precision=q.QSEL_MIXED, pcg_tol=1e-9, pcg_max_iter=4000)
    b = _batch(q, models, n_streams=4, autotune=True, **opts)
    q.qsel_batch_run(b)
    info = q.qsel_batch_info(b)
    print(f"autotune {info['ms_autotune']:.0f} ms")
    assert info["ms_autotune"] > 0
    for i, mdl in enumerate(models):
        tu = q.qsel_batch_tuning(b, i)
        assert tu["precond_block"] in (16, 32, 64) and tu["tensor_passes"] in (0, 1, 3)
        assert 0 <= tu["stream"] < 4
        pb = tu["precond_block"]
        tp = tu["tensor_passes"] if tu["tensor_passes"] > 0 else -1
        v, t, _ = _single(q, mdl, i, precond_block=pb, tensor_passes=tp, **opts)
        np.testing.assert_array_equal(q.qsel_batch_diag_inv(b, i), v)
