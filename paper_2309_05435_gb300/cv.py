"""Learned control variate: training set, training and planned solves.

Orchestration over the C ABI only: features, targets, the network's forward
and backward passes, Adam, the planner and the RBMC pipeline all run in
libqsel.so.  PyTorch provides the device buffers.

The network predicts each node's share c_i / v_i of the variance that the
Rao-Blackwell correction carries (Algorithm 4); the planner turns the
prediction into one sample count and an overlap per part, and the sample-based
error estimate of the finished run judges the choice (a miss triggers one
more run with the sample count scaled by the squared miss).  The estimate is
always plain RBMC at the chosen settings, so it is unbiased whatever the
network predicts.
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np

from . import qsel as q


@dataclasses.dataclass
class ModelSpec:
    """One space-time model (host arrays, as qsel_create takes them)."""
    mesh: object            # qsel_inputs.GridMesh
    n_t: int
    mask: np.ndarray
    sigma: float
    slab_start: np.ndarray

    @property
    def n_s(self) -> int:
        return self.mesh.n_s

    @property
    def n(self) -> int:
        return self.mesh.n_s * self.n_t

    @property
    def n_parts(self) -> int:
        return len(self.slab_start) - 1

    def context(self, theta, overlap, k, seed, precision=q.QSEL_MIXED, pcg_tol=1e-8, part_overlap=None,
                cuda_stream=None, preconditioner=q.QSEL_PRECOND_BLOCK_JACOBI) -> q.Context:
        return q.qsel_create(self.n_s, self.n_t, self.mesh.c_diag, self.mesh.g_rowptr, self.mesh.g_col,
                             self.mesh.g_val, self.mask, self.sigma, theta, n_parts=self.n_parts,
                             slab_start=self.slab_start, overlap=overlap, n_samples=k, seed=seed,
                             precision=precision, pcg_tol=pcg_tol, pcg_max_iter=50000,
                             part_overlap=part_overlap, cuda_stream=cuda_stream, preconditioner=preconditioner)


def training_set(spec: ModelSpec, thetas, overlaps, k: int = 512, seeds=(1, 2), precision=q.QSEL_MIXED):
    """Features and targets log(c_i / v_i) over a theta grid and overlaps.
    The targets average the corrections of len(seeds) runs of k samples each
    (together an RBMC estimate with len(seeds) * k samples)."""
    import torch
    Xs, ys = [], []
    for th in thetas:
        for nl in overlaps:
            ctxs = [spec.context(th, nl, k, s, precision) for s in seeds]
            for c in ctxs:
                c.diag_inv()
            F = torch.empty((spec.n, q.QSEL_CV_FEATURES), dtype=torch.float32, device="cuda")
            y = torch.empty(spec.n, dtype=torch.float32, device="cuda")
            q.qsel_cv_features(ctxs[0], nl, F)
            q.qsel_cv_targets(ctxs, y)
            Xs.append(F)
            ys.append(y)
            for c in ctxs:
                c.close()
    return torch.cat(Xs), torch.cat(ys)


def train(X, y, steps=(1500, 1000), lrs=(3e-3, 5e-4), seed: int = 0) -> q.ControlVariate:
    """Full-batch Adam on the device: one phase per (steps, lr); the input
    standardisation is taken from X first."""
    cv = q.qsel_cv_create(seed)
    n = X.shape[0]
    q.qsel_cv_train(cv, X, y, n, 0, 1e-3, set_input_stats=True)
    for st, lr in zip(steps, lrs):
        q.qsel_cv_train(cv, X, y, n, st, lr)
    return cv


def _timed_run(spec, theta, overlap, k, seed, precision, part_overlap=None,
               preconditioner=q.QSEL_PRECOND_BLOCK_JACOBI):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = spec.context(theta, overlap, k, seed, precision, part_overlap=part_overlap, preconditioner=preconditioner)
    v = ctx.diag_inv()
    t = ctx.trace_grads()
    _, err = q.qsel_error_estimate(ctx)
    wall = time.perf_counter() - t0
    ms = ctx.stats()["ms_total"]
    ctx.close()
    return v, t, err, wall, ms


def solve_plain(spec: ModelSpec, theta, target: float, overlap: int, k0: int = 32, k_max: int = 512,
                seed: int = 11, precision=q.QSEL_FP64, max_batches: int = 8):
    """Plain RBMC without a predictor: fixed overlap, k doubled from k0 until
    the sample-based error estimate meets the target.  Past k_max, further
    independent k_max-sample batches (new seeds) are averaged with the last
    one: the mean of B estimates is the RBMC estimate with B * k_max samples,
    its error estimate sqrt(sum_b err_b^2) / B (per-batch errors combined as
    independent)."""
    runs, k, wall, ms, samples = [], k0, 0.0, 0.0, 0
    batch = []
    while True:
        v, t, err, w, m = _timed_run(spec, theta, overlap, k, seed + len(runs), precision)
        runs.append({"k": k, "err": err, "wall_s": w})
        wall += w
        ms += m
        samples += k
        if k < k_max:
            if err <= target:
                break
            k = min(2 * k, k_max)
            continue
        batch.append((v, t, err))
        err = math.sqrt(sum(b[2] ** 2 for b in batch)) / len(batch)
        if err <= target or len(batch) >= max_batches:
            v = np.mean([b[0] for b in batch], axis=0)
            t = np.mean([b[1] for b in batch], axis=0)
            break
    return {"v": v, "t": t, "err": err, "k": k * max(1, len(batch)), "overlap": overlap, "runs": runs,
            "wall_s": wall, "device_ms": ms, "samples_drawn": samples, "met": err <= target}


def solve_planned(spec: ModelSpec, theta, cv: q.ControlVariate, target: float, max_overlap: int = 8,
                  k_max: int = 512, seed: int = 11, precision=q.QSEL_MIXED, margin: float = 0.85,
                  preconditioner=q.QSEL_PRECOND_BLOCK_JACOBI, cost_pcg: float = 0.0):
    """Planned RBMC: predict, plan for margin * target (one k, an overlap per
    part), run once, judge by the error estimate; a miss of the target reruns
    once with k scaled by (err / (margin * target))^2 (at most k_max)."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    probe = spec.context(theta, 1, 32, seed, precision)
    plan = q.qsel_cv_plan(probe, cv, margin * target, max_overlap=max_overlap, max_samples=k_max,
                          cost_pcg=cost_pcg)
    probe.close()
    t_plan = time.perf_counter() - t0
    k, po = plan["n_samples"], plan["part_overlap"].copy()
    runs, wall, ms, samples = [], t_plan, 0.0, 0
    while True:
        v, t, err, w, m = _timed_run(spec, theta, 1, k, seed, precision, part_overlap=po,
                                     preconditioner=preconditioner)
        runs.append({"k": k, "part_overlap": po.tolist(), "err": err, "wall_s": w})
        wall += w
        ms += m
        samples += k
        if err <= target or k >= k_max or len(runs) >= 2:
            break
        k = min(k_max, int(math.ceil(k * (err / (margin * target)) ** 2 / 32.0)) * 32)
        seed += 1
    return {"v": v, "t": t, "err": err, "k": k, "part_overlap": po.tolist(), "plan": plan, "runs": runs,
            "plan_s": t_plan, "wall_s": wall, "device_ms": ms, "samples_drawn": samples,
            "met": err <= target}


def sobol_thetas(n: int, seed: int):
    """Scrambled-Sobol points over log kappa in [-3, 0], log tau in [-1, 1],
    rho in [0.5, 0.99] (returned as (log kappa, log tau, logit rho))."""
    from scipy.stats import qmc
    u = qmc.Sobol(d=3, scramble=True, seed=seed).random_base2(max(0, math.ceil(math.log2(n))))[:n]
    lk = -3.0 + 3.0 * u[:, 0]
    lt = -1.0 + 2.0 * u[:, 1]
    rho = 0.5 + 0.49 * u[:, 2]
    return [(float(a), float(b), float(math.log(r / (1 - r)))) for a, b, r in zip(lk, lt, rho)]
