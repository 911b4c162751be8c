"""Learned control variate on the GPU against the oracle (oracle/qsel_mlp.py,
oracle/qsel_oracle.py): features, the BF16-weight network's forward pass and
gradients, Adam, targets, the planner, the sample-based error estimate and
per-part overlaps; then what the trained network gains over plain RBMC.

Tolerances: features are FP64 values rounded to float (1e-6 relative); the
network accumulates in FP32 over at most 64 terms per dot product with
erff-based GELU (1e-4 of the largest value per result); the error estimate
and the per-part-overlap pipeline are FP64 (1e-10)."""
import math

import numpy as np
import pytest

import qsel_inputs as qi
from oracle import qsel_mlp as om
from oracle import qsel_oracle as o
from tests.test_gpu_parity import Case, q  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _params(seed=0):
    rng = np.random.default_rng(seed)
    return {"W1": rng.normal(0, 0.4, (64, 14)), "b1": rng.normal(0, 0.1, 64),
            "W2": rng.normal(0, 0.2, (64, 64)), "b2": rng.normal(0, 0.1, 64),
            "W3": rng.normal(0, 0.2, (1, 64)), "b3": rng.normal(0, 0.1, 1),
            "mu": rng.normal(0, 1, 14), "scale": rng.uniform(0.5, 2.0, 14)}


ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def _flat(P):
    return np.concatenate([np.ravel(P[k]) for k in ORDER + ("mu", "scale")]).astype(np.float32)


def _as_used(P):
    """The oracle sees exactly the float32 values the device holds."""
    return {k: np.asarray(v, dtype=np.float32).astype(np.float64) for k, v in P.items()}


def _dev(a):
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("name,overlap", [("grid16_nt8", 1), ("grid16_nt8", 2), ("ragged13", 1),
                                          ("uneven4", 3), ("overlap2", 2)])
def test_features_match_oracle(q, name, overlap):
    torch = _torch()
    c = Case(q, name)
    F = torch.empty((c.n_s * c.n_t, 14), dtype=torch.float32, device="cuda")
    q.qsel_cv_features(c.ctx, overlap, F)
    F_or = om.features(c.model, c.theta, c.slab_start, overlap)
    np.testing.assert_allclose(F.cpu().numpy(), F_or, rtol=1e-6, atol=1e-5)


def test_forward_matches_oracle(q):
    P = _as_used(_params(1))
    cv = q.qsel_cv_create(0)
    q.qsel_cv_set_params(cv, _flat(P))
    X = np.random.default_rng(2).normal(0, 1.5, (1000, 14))
    y = _torch().empty(1000, dtype=_torch().float32, device="cuda")
    q.qsel_cv_predict(cv, _dev(X), y, 1000)
    y_or, _ = om.forward(P, X.astype(np.float32).astype(np.float64), bf16=True)
    assert np.max(np.abs(y.cpu().numpy() - y_or)) <= 1e-4 * max(1.0, np.max(np.abs(y_or)))
    # BF16 rounding is visible: the FP64 network without it differs by more
    y_full, _ = om.forward(P, X.astype(np.float32).astype(np.float64), bf16=False)
    assert np.max(np.abs(y_full - y_or)) > 1e-3


@pytest.mark.parametrize("n", [1000, 64, 7])
def test_gradient_matches_oracle(q, n):
    P = _as_used(_params(3))
    cv = q.qsel_cv_create(0)
    q.qsel_cv_set_params(cv, _flat(P))
    rng = np.random.default_rng(4)
    X = rng.normal(0, 1.5, (n, 14)).astype(np.float32).astype(np.float64)
    t = rng.normal(0, 1, n).astype(np.float32).astype(np.float64)
    g, loss = q.qsel_cv_grad(cv, _dev(X), _dev(t), n)
    loss_or, g_or = om.loss_and_grad(P, X, t, bf16=True)
    assert abs(loss - loss_or) <= 1e-5 * loss_or
    off = 0
    for k in ORDER:
        ref = np.ravel(g_or[k])
        got = g[off:off + ref.size]
        off += ref.size
        assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref)), k
    assert off == q.QSEL_CV_PARAMS


def test_adam_first_step_and_training(q):
    """Adam's first step moves every parameter by lr * g / (|g| + eps), i.e.
    lr * sign(g) where |g| >> eps; then training on a teacher network's
    outputs lowers the loss by well over an order of magnitude and sets the
    input standardisation from the data."""
    torch = _torch()
    rng = np.random.default_rng(5)
    n = 4096
    X = rng.normal(0, 1, (n, 14)) * rng.uniform(0.5, 3, 14) + rng.normal(0, 2, 14)
    teacher = _params(6)
    t, _ = om.forward(teacher, X, bf16=False)
    Xd, td = _dev(X), _dev(t)
    cv = q.qsel_cv_create(11)
    p0 = q.qsel_cv_get_params(cv)
    g, _ = q.qsel_cv_grad(cv, Xd, td, n)
    lr = 1e-3
    q.qsel_cv_train(cv, Xd, td, n, 1, lr)
    p1 = q.qsel_cv_get_params(cv)
    big = np.abs(g) > 1e-4
    np.testing.assert_allclose((p1 - p0)[:q.QSEL_CV_PARAMS][big], -lr * np.sign(g[big]), rtol=1e-3, atol=1e-7)

    cv = q.qsel_cv_create(12)
    loss0 = q.qsel_cv_train(cv, Xd, td, n, 0, 1e-3, set_input_stats=True)
    p = q.qsel_cv_get_params(cv)
    Xf = X.astype(np.float32).astype(np.float64)
    np.testing.assert_allclose(p[5185:5199], Xf.mean(0), rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(p[5199:5213], Xf.std(0), rtol=1e-3)
    loss1 = q.qsel_cv_train(cv, Xd, td, n, 600, 3e-3)
    print(f"teacher fit: loss {loss0:.3e} -> {loss1:.3e}")
    assert loss1 < 0.1 * loss0
    torch.cuda.synchronize()


@pytest.mark.parametrize("name", ["grid16_nt8", "overlap2", "uneven4"])
def test_error_estimate_matches_oracle(q, name):
    c = Case(q, name)
    X = qi.seeded_normal((c.n_s * c.n_t, c.k), 21)
    q.qsel_debug_set_samples(c.ctx, X)
    v = c.ctx.diag_inv()
    part, glob = q.qsel_error_estimate(c.ctx)
    v_or, _, res = o.rbmc(c.model, c.theta, c.slab_start, c.n_l, X)
    part_or, glob_or = o.error_estimate(v_or, res, c.k)
    np.testing.assert_allclose(part, part_or, rtol=1e-10)
    assert abs(glob - glob_or) <= 1e-10 * glob_or


def test_error_estimate_needs_a_run(q):
    c = Case(q, "grid16_nt8")
    with pytest.raises(q.QselError) as e:
        q.qsel_error_estimate(c.ctx)
    assert e.value.status == 7


@pytest.mark.parametrize("po", [[1, 2, 1], [0, 3, 2], [2, 2, 2]])
def test_per_part_overlap_matches_oracle(q, po):
    c = Case(q, "overlap2", part_overlap=po, overlap=1)
    X = qi.seeded_normal((c.n_s * c.n_t, c.k), 8)
    q.qsel_debug_set_samples(c.ctx, X)
    v = c.ctx.diag_inv()
    v_or, t_or, _ = o.rbmc(c.model, c.theta, c.slab_start, po, X)
    assert np.max(np.abs(v - v_or) / v_or) <= 1e-10
    if min(po) >= 1:
        t = c.ctx.trace_grads()
        assert np.max(np.abs(t - t_or) / np.abs(t_or)) <= 1e-10
    else:
        with pytest.raises(q.QselError):
            c.ctx.trace_grads()


def test_targets_from_several_runs(q):
    torch = _torch()
    cs = [Case(q, "grid16_nt8", seed=s) for s in (1, 2, 3)]
    vs = [c.ctx.diag_inv() for c in cs]
    sel = q.qsel_debug_get_selinv_diag(cs[0].ctx)
    y = torch.empty(cs[0].n_s * cs[0].n_t, dtype=torch.float32, device="cuda")
    q.qsel_cv_targets([c.ctx for c in cs], y)
    cbar = np.mean([v - sel for v in vs], axis=0)
    ref = np.log(np.maximum(cbar / (sel + cbar), 1e-9))
    np.testing.assert_allclose(y.cpu().numpy(), ref, rtol=1e-6, atol=1e-6)


def _constant_network(q, r0):
    P = _params(0)
    P["W3"][:] = 0.0
    P["b3"][:] = math.log(r0)
    cv = q.qsel_cv_create(0)
    q.qsel_cv_set_params(cv, _flat(P))
    return cv


def test_planner_with_constant_prediction(q):
    """A network that predicts c/v = r0 everywhere: the error at k samples is
    sqrt(2 r0^2 / k) for every part and overlap, so the plan is the smallest
    multiple of 32 with 2 r0^2 / k <= target^2 and the smallest overlap."""
    c = Case(q, "uneven4")
    cv = _constant_network(q, 0.05)
    plan = q.qsel_cv_plan(c.ctx, cv, 0.01, max_overlap=3)
    k_need = 2 * 0.05 ** 2 / 0.01 ** 2                      # 50
    assert plan["feasible"] and plan["n_samples"] == 32 * math.ceil(k_need / 32)
    assert list(plan["part_overlap"]) == [1, 1, 1, 1]
    assert abs(plan["predicted_err"] - math.sqrt(2 * 0.05 ** 2 / plan["n_samples"])) < 1e-6
    # infeasible within 512 samples: best effort at the limits
    plan = q.qsel_cv_plan(c.ctx, _constant_network(q, 0.5), 0.01, max_overlap=3)
    assert not plan["feasible"] and plan["n_samples"] == 512 and list(plan["part_overlap"]) == [3, 3, 3, 3]
    # cost model: cheaper PCG favours fewer dense slabs, and the k grid is a multiple of 32
    plan = q.qsel_cv_plan(c.ctx, cv, 0.01, max_overlap=3, min_samples=100, max_samples=300)
    assert plan["n_samples"] == 128


def test_planner_chooses_part_count(q):
    """With candidate part counts the planner also picks the partition: under
    a constant prediction every partition needs the same k, so the one with
    the fewest factorised slabs wins (two parts of five slabs, overlap 1:
    12 slabs, against 16 for four parts); with 1 among the candidates the
    exact one-part form (n_t slabs, no samples, error 0) is cheaper still."""
    c = Case(q, "uneven4")                                   # n_t = 10, four parts
    cv = _constant_network(q, 0.05)
    plan = q.qsel_cv_plan(c.ctx, cv, 0.01, max_overlap=3, part_counts=[4, 2])
    assert plan["feasible"] and plan["n_parts"] == 2 and list(plan["slab_start"]) == [0, 5, 10]
    assert plan["n_samples"] == 64 and list(plan["part_overlap"]) == [1, 1]
    plan = q.qsel_cv_plan(c.ctx, cv, 0.01, max_overlap=3, part_counts=[4, 2, 1])
    assert plan["n_parts"] == 1 and plan["n_samples"] == 0 and plan["predicted_err"] == 0.0
    assert plan["predicted_cost"] == pytest.approx(plan["single_part_cost"])
    # without candidates: the context's own four parts, as before
    plan = q.qsel_cv_plan(c.ctx, cv, 0.01, max_overlap=3)
    assert plan["n_parts"] == 4 and list(plan["slab_start"]) == [0, 3, 6, 8, 10]


def test_cv_gain_over_plain_rbmc(q):
    """What the trained network gains.  Train on GPU-produced targets of small
    models (16 x 16 grid, 24 slabs, 3 parts, overlaps 1-3, 12 theta), then on
    two held-out theta of a different model (32 slabs, 4 parts): plain RBMC at
    overlap 1 doubles k from 32 until its error estimate meets the target;
    the planned run picks k and per-part overlaps once.  The planned solve
    must reach the target (after at most one corrective run) drawing fewer
    samples in fewer pipeline runs."""
    from paper_2309_05435_gb300 import cv as cvm
    mesh = qi.grid_mesh(16)
    train_spec = cvm.ModelSpec(mesh, 24, qi.obs_mask(256 * 24, 0.25, 3), 0.5, qi.balanced_slab_start(24, 3))
    thetas = cvm.sobol_thetas(16, seed=1)[:12]
    X, y = cvm.training_set(train_spec, thetas, (1, 2, 3), k=256, seeds=(1, 2))
    net = cvm.train(X, y, steps=(800, 400))
    _, loss = q.qsel_cv_grad(net, X, y, X.shape[0])
    print(f"training samples {X.shape[0]}, final loss {loss:.3e}, target variance {float(y.var()):.3e}")
    assert loss < 0.25 * float(y.var())
    eval_spec = cvm.ModelSpec(mesh, 32, qi.obs_mask(256 * 32, 0.25, 4), 0.5, qi.balanced_slab_start(32, 4))
    for th in cvm.sobol_thetas(2, seed=99):
        th = (th[0], th[1], max(th[2], math.log(0.85 / 0.15)))   # strong time correlation: corrections matter
        ref = cvm.solve_plain(eval_spec, th, 1e-9, overlap=1, k0=128, k_max=128, precision=q.QSEL_MIXED,
                              max_batches=1)
        target = 0.5 * ref["err"]          # plain needs about 4x the samples: 32 -> 512 in 5 runs
        plain = cvm.solve_plain(eval_spec, th, target, overlap=1, precision=q.QSEL_MIXED)
        planned = cvm.solve_planned(eval_spec, th, net, target, max_overlap=3)
        print(f"theta {np.round(th, 3)} target {target:.4f}: plain k={plain['k']} runs={len(plain['runs'])} "
              f"samples={plain['samples_drawn']} err={plain['err']:.4f}; planned k={planned['k']} "
              f"overlaps={planned['part_overlap']} runs={len(planned['runs'])} "
              f"samples={planned['samples_drawn']} err={planned['err']:.4f} "
              f"(predicted {planned['plan']['predicted_err']:.4f})")
        assert planned["met"]
        assert planned["samples_drawn"] < plain["samples_drawn"]
        assert len(planned["runs"]) < len(plain["runs"])
