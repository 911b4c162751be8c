#!/usr/bin/env python
"""Benchmark: time to diag(Q^-1) + tr(Q^-1 dQ/dtheta_j) at 1 % relative error
on one GB300.

Workload (default): 96 x 96 grid (n_s = 9216), n_t = 256 (n = 2,359,296),
kappa = 0.1, rho = 0.98, 10 % observed, PCG to 1e-10 -- synthetic, seeded.

The chosen form is mixed precision with the learned control variate: a
network trained first on the GPU (reported separately, not timed) predicts
every node's correction share, the planner picks the part count, one sample
count and an overlap per part for a 1 % RMS relative standard error, and
RBMC runs at those settings.  One step = one pass through the C ABI on a
resident context with a new seed: qsel_cv_plan (features + network + plan),
qsel_set_seed, qsel_set_theta, qsel_diag_inv (perturbation RHS, multi-RHS
PCG, per-subdomain block factorisation + Takahashi, RB correction),
qsel_trace_grads and qsel_error_estimate.  Reported beside it: the accuracy
over the W + K seeds against the exact one-part result, the exact one-part
form itself (timed), plain FP64 RBMC's time to 1 % (errors measured, FP64
time extrapolated per slab), the class breakdown of a profiled pass, the
end-to-end call from host buffers, the CPU oracle on a bounded sample, and
a second workload (64 x 64 grid, n_t = 64).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
  python bench.py --cv-eval      # held-out evaluation of the control variate

N > 1 runs under torch.distributed.run: every rank solves its own independent
replica (weak scaling, no data-path collective); the barrier and the max over
ranks bracket the timed region.  --impl reference times the CPU FP64 oracle
on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import qsel_inputs as qi  # noqa: E402

METRIC = "time to diag(Q^-1)+trace grads at 1% rel err; chosen vs plain FP64, 1 GB300"
FP64_PEAK_TFLOPS = 1.25      # GB300 nominal FP64 (152 SMs x 2.07 GHz x 4 FLOP/clk/SM)
FP32_PEAK_TFLOPS = 80.5      # GB300 FP32 CUDA cores (152 SMs x 128 lanes x 2 FLOP x 2.07 GHz)
# DRAM bytes per FLOP of k_gemm64 from one ncu capture (profiles/k_gemm64_grid64_nt16_fp64.md)
GEMM64_DRAM_BYTES_PER_FLOP = 7.808e9 / 2.749e11
# DRAM bytes of one rank-256 sweep panel update of a 4096^2 FP32 matrix on the
# tensor cores (profiles/k_tc_gemm_grid64_nt16_mixed.md: 104.8 MB for 2 matrices)
TC_UPDATE_DRAM_BYTES_PER_MATRIX = 104.8e6 / 2
# planner's PCG cost per sample and node with the Kronecker preconditioner
# (seconds; the library default describes 64-row block Jacobi)
KRON_PCG_COST = 0.36e-8
L2_BYTES = 126 * 2 ** 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", default="grid96_nt256")
    ap.add_argument("--secondary", default="grid64_nt64",
                    help="second workload timed after the bench line's (chosen and exact forms); '' = none")
    ap.add_argument("--plain-seeds", type=int, default=1,
                    help="seeds per overlap of the plain-FP64 time-to-target procedure (0 = skip it)")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep", default=None,
                    help="time-to-accuracy sweep instead of the bench line: comma list of "
                         "form:n_parts:overlap:n_samples entries, form in {mixed, fp64}")
    ap.add_argument("--seeds", type=int, default=1, help="RBMC seeds per sweep entry")
    ap.add_argument("--target", type=float, default=0.01, help="RMS relative error target of the plan")
    ap.add_argument("--max-overlap", type=int, default=8)
    ap.add_argument("--preconditioner", choices=["kron", "bj"], default="kron",
                    help="PCG preconditioner of the chosen form: Kronecker grid (kron) or 64-row block Jacobi "
                         "(bj); plain FP64 always uses block Jacobi, the paper's choice")
    ap.add_argument("--margin", type=float, default=0.85,
                    help="the planner aims at margin * target (absorbs the prediction error)")
    ap.add_argument("--cv-train-thetas", type=int, default=32)
    ap.add_argument("--cv-train-steps", type=int, default=2000)
    ap.add_argument("--cv-params", default=None,
                    help="load the control-variate network (QSEL_CV_PARAMS_ALL floats, .npy) instead of training")
    ap.add_argument("--save-cv-params", default=None, help="save the trained network (.npy)")
    ap.add_argument("--cv-eval", action="store_true",
                    help="held-out evaluation: 64x64 grid, n_t=128, 8 parts, 8 theta; planned vs plain")
    ap.add_argument("--cv-eval-thetas", type=int, default=8)
    ap.add_argument("--cv-controls", type=int, default=8,
                    help="held-out theta on which plain RBMC also runs at fixed overlaps 1, 2, 4, 8")
    ap.add_argument("--cv-fp64-thetas", type=int, default=2,
                    help="held-out theta on which plain FP64 is also run to the target")
    ap.add_argument("--batch", action="store_true",
                    help="uneven batch: 64 independent models under one captured graph vs one at a time")
    ap.add_argument("--batch-models", type=int, default=64)
    ap.add_argument("--batch-streams", type=int, default=16)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--kron-apply", default=None,
                    help="one mixed Kronecker preconditioner apply (k = 256) on WORKLOAD (profiling captures)")
    ap.add_argument("--exact-pass", default=None,
                    help="one exact one-part mixed pass at this workload (for kernel captures)")
    ap.add_argument("--chain", choices=["two_ended", "forward"], default="two_ended",
                    help="order of the one-part block factorisation (qsel_options.chain)")
    ap.add_argument("--oracle-e2e", default=None,
                    help="comma list of workloads: time the CPU oracle end to end (all host cores)")
    ap.add_argument("--oracle-e2e-single", default="grid16_nt8",
                    help="workloads of --oracle-e2e also timed on one thread")
    ap.add_argument("--hyper-eval", action="store_true",
                    help="time the posterior mean and the hyperparameter gradient (mixed and FP64)")
    ap.add_argument("--lanczos-eval", default=None,
                    help="comma list of Krylov dimensions: the Lanczos sampler against PCG at the workload")
    return ap.parse_args()


CV_TRAIN_OVERLAPS = (1, 2, 3, 4, 5, 6, 7, 8)


def train_control_variate(args):
    """Training set from the method itself on 16 x 16 grid models (n_t = 32,
    4 parts, overlaps 1-8, scrambled-Sobol theta, 2 x 512 samples per target),
    then full-batch Adam -- all on the GPU through the C ABI."""
    import torch
    from paper_2309_05435_gb300 import cv as cvm
    mesh = qi.grid_mesh(16)
    spec = cvm.ModelSpec(mesh, 32, qi.obs_mask(256 * 32, 0.25, 5), 0.5, qi.balanced_slab_start(32, 4))
    thetas = cvm.sobol_thetas(args.cv_train_thetas, seed=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X, y = cvm.training_set(spec, thetas, CV_TRAIN_OVERLAPS, k=512, seeds=(1, 2))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    s1 = args.cv_train_steps * 3 // 5
    net = cvm.train(X, y, steps=(s1, args.cv_train_steps - s1), lrs=(3e-3, 5e-4))
    from paper_2309_05435_gb300 import qsel
    _, loss = qsel.qsel_cv_grad(net, X, y, X.shape[0])
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    info = {"models": "16x16 grid, n_t=32, 4 parts, overlaps 1-8, 25% observed",
            "thetas": len(thetas), "samples_per_target": 1024, "training_rows": int(X.shape[0]),
            "adam_steps": args.cv_train_steps, "final_mse": loss, "target_variance": float(y.var()),
            "data_s": t1 - t0, "train_s": t2 - t1}
    return net, info



def rank_seed(rank: int) -> int:
    """Independent replica per rank: its own noise seed."""
    return 1000 + rank


def job_time_ms(local_ms: float, world: int, dist=None, device="cpu") -> float:
    """Job time of a timed region = max over ranks of the per-rank times
    (every rank brackets the region with a barrier)."""
    if world <= 1 or dist is None:
        return float(local_ms)
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value_s(job_ms: float, steps: int, world: int) -> float:
    """Seconds per solved problem for the whole job: `world` replicas each
    solve `steps` problems within job_ms (weak scaling)."""
    return job_ms / 1e3 / (steps * world)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s (no MEASURED_PEAKS.json)"


def tf32_peak_tflops():
    """Dense TF32 tensor peak for kernels timed inside a seconds-long step: the
    measured sustained bf16 peak times the nominal TF32 / bf16 ratio
    (1.1 / 2.25 PFLOP/s)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        bf16 = float(d["bf16_tflops_sustained"])
        return bf16 * 1.1 / 2.25, (f"measured sustained bf16 {bf16:.0f} TFLOP/s x nominal TF32/bf16 ratio "
                                   "1.1/2.25")
    except (OSError, KeyError, ValueError):
        return 1700.0 * 1.1 / 2.25, "fallback sustained bf16 1.7 PFLOP/s x nominal TF32/bf16 ratio 1.1/2.25"


def workload_inputs(w, rank=0):
    mesh = w.mesh()
    mask = w.mask()
    return mesh, mask


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline and the reference arm)
# ----------------------------------------------------------------------------
def oracle_sample(w, exact=True, frac=1.0):
    """Time the oracle's per-slab dense work at the workload's block size: block
    Cholesky and Takahashi of a 2-slab chain of Q's blocks.  The exact one-part
    form (the form the GPU line times when the planner picks it) needs n_t slab
    units of factor + Takahashi; plain RBMC at the workload's partition needs
    sum_p T_p of them plus n_t units of factor for the oracle's direct sampler.
    With frac < 1 the sample takes the leading frac n_s rows and columns of
    every block (a principal submatrix: SPD and block tridiagonal again) and
    scales its time by frac^-3, the dense blocks' cubic cost.  Returns
    (extrapolated seconds, sample seconds, description)."""
    from oracle import qsel_oracle as o
    mesh, mask = workload_inputs(w)
    model = o.model_from_csr(w.n_s, w.n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val, mask, w.sigma)
    Q = o.precision(model, w.theta)
    m = w.n_s if frac >= 1.0 else max(64, int(round(w.n_s * frac)))
    diag_b = [o.block(Q, w.n_s, t, t)[:m, :m] for t in (0, 1)]
    sub_b = [o.block(Q, w.n_s, 1, 0)[:m, :m]]
    t0 = time.perf_counter()
    L_diag, L_sub = o.block_cholesky(diag_b, sub_b)
    t1 = time.perf_counter()
    o.block_takahashi(L_diag, L_sub)
    t2 = time.perf_counter()
    scale = (w.n_s / m) ** 3
    chol, tak = scale * (t1 - t0) / 2, scale * (t2 - t1) / 2
    part = "" if m == w.n_s else f"leading {m}x{m} of every block, time x {scale:.1f} for the cubic cost; "
    if exact:
        est = w.n_t * (chol + tak)
        desc = (f"oracle block Cholesky + Takahashi of a 2-slab chain of {w.n_s}x{w.n_s} blocks "
                f"({part}{t2 - t0:.1f} s), extrapolated to the {w.n_t} slabs of the exact one-part selected "
                "inversion (the form of the GPU line)")
        return est, t2 - t0, desc
    parts = o.partition(w.n_t, qi.balanced_slab_start(w.n_t, w.n_parts), w.overlap)
    units = sum(p.ext[1] - p.ext[0] for p in parts)
    est = units * (chol + tak) + w.n_t * chol
    desc = (f"oracle block Cholesky + Takahashi of a 2-slab chain of {w.n_s}x{w.n_s} blocks "
            f"({part}{t2 - t0:.1f} s), extrapolated to {units} subdomain slabs + {w.n_t} sampler slabs of plain "
            "RBMC; excludes the correction solves (lower bound)")
    return est, t2 - t0, desc


def cpu_cores():
    return os.cpu_count() or 1


def oracle_sample_single_thread(w):
    """The same oracle sample in a child process whose BLAS / OpenMP pools are
    limited to one thread before numpy loads; (extrapolated seconds, sample
    seconds) or None if the child fails."""
    env = dict(os.environ)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[var] = "1"
    try:
        p = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", "--workload", w.name],
                           env=env, capture_output=True, text=True, timeout=600)
        d = json.loads(p.stdout.strip().splitlines()[-1])
        return d["est"], d["spent"]
    except Exception:   # a missing single-thread figure must not fail the bench line
        return None


# ----------------------------------------------------------------------------
# native arm
# ----------------------------------------------------------------------------
RBMC_PART_COUNTS = (2, 4, 8, 16)
PLAN_MAX_OVERLAP = 16        # the network's time-distance feature is capped at 16 slabs


def _errs(v, g, v_ex, t_ex):
    r = (v - v_ex) / v_ex
    return {"eps_diag_rms": float(np.sqrt(np.mean(r ** 2))), "eps_diag_p99": float(np.quantile(np.abs(r), 0.99)),
            "eps_diag_max": float(np.max(np.abs(r))),
            "eps_traces": [float(abs(a - b) / abs(b)) for a, b in zip(g, t_ex)]}


def _seed_errors(vs, gs, v_ex, t_ex):
    """Error definitions of the metric over R seeds: eps_diag = RMS over seeds
    and nodes of the relative error, eps_j = RMS over seeds per trace, and
    the 99th percentile over nodes of the per-node RMS."""
    rd = np.array([((v - v_ex) / v_ex) ** 2 for v in vs])
    rt = np.array([[((a - b) / b) ** 2 for a, b in zip(g, t_ex)] for g in gs])
    eps_d = float(np.sqrt(rd.mean()))
    eps_t = [float(np.sqrt(rt[:, j].mean())) for j in range(rt.shape[1])]
    return {"eps_diag": eps_d, "eps_diag_p99": float(np.quantile(np.sqrt(rd.mean(axis=0)), 0.99)),
            "eps_traces": eps_t, "seeds": len(vs), "meets_1pct": bool(max(eps_d, *eps_t) <= 0.01)}


def _subdomain_slabs(n_t, slab_start, overlaps):
    """(forward slabs, backward slabs) of the block factorisation and the
    Takahashi recursion over every extended part."""
    fwd = bwd = 0
    for p in range(len(slab_start) - 1):
        e0 = max(0, slab_start[p] - overlaps[p])
        e1 = min(n_t, slab_start[p + 1] + overlaps[p])
        lo = slab_start[p] - e0
        fwd += e1 - e0
        bwd += (e1 - e0) - 1 - max(lo - 1, 0)
    return fwd, bwd


class Native:
    """The library's contexts for one workload (inputs resident in HBM)."""

    def __init__(self, q, w, stream, dev, chain="two_ended"):
        self.q, self.w, self.stream, self.dev = q, w, stream, dev
        self.mesh, self.mask = workload_inputs(w)
        self.chain = q.QSEL_CHAIN_FORWARD if chain == "forward" else q.QSEL_CHAIN_TWO_ENDED

    def ctx(self, precision, n_parts=None, slab_start=None, overlap=None, k=None, part_overlap=None, seed=1000,
            preconditioner=None, profile=0, mesh_mask=None, n_t=None):
        q, w = self.q, self.w
        mesh, mask = (self.mesh, self.mask) if mesh_mask is None else mesh_mask
        pc = preconditioner if preconditioner is not None else (
            q.QSEL_PRECOND_KRON if precision == q.QSEL_MIXED else q.QSEL_PRECOND_BLOCK_JACOBI)
        return q.qsel_create(w.n_s, n_t or w.n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val, mask,
                             w.sigma, w.theta, n_parts=n_parts or w.n_parts, slab_start=slab_start,
                             overlap=w.overlap if overlap is None else overlap,
                             n_samples=k or w.n_samples, seed=seed, precision=precision, pcg_tol=w.pcg_tol,
                             cuda_stream=self.stream.cuda_stream, profile_kernels=profile,
                             part_overlap=part_overlap, preconditioner=pc, chain=self.chain)

    def exact(self, precision):
        """One pass of the exact one-part form: (s, diag, traces, stats)."""
        import torch
        c = self.ctx(precision, n_parts=1, overlap=0, k=2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        v = self.q.qsel_diag_inv(c)
        g = self.q.qsel_trace_grads(c)
        e1.record(self.stream)
        torch.cuda.synchronize()
        st = self.q.qsel_stats(c)
        c.close()
        return e0.elapsed_time(e1) / 1e3, v, np.asarray(g), st


def measure_exact(args, nat, world, dist, clocks=True):
    """The exact one-part form (n_p = 1, the whole chain one subdomain, no
    samples) timed like the RBMC form: W untimed and K timed steps, each one
    full pass (set theta + diag + traces)."""
    import torch
    q, w, stream = nat.q, nat.w, nat.stream
    ctx = nat.ctx(q.QSEL_MIXED, n_parts=1, overlap=0, k=2)
    outs = [torch.empty(w.n, dtype=torch.float64, device=nat.dev) for _ in range(args.warmup + args.steps)]
    grads = []

    def step(i):
        q.qsel_set_theta(ctx, w.theta)
        q.qsel_diag_inv(ctx, outs[i])
        grads.append(np.asarray(q.qsel_trace_grads(ctx)))
        return q.qsel_stats(ctx)

    for i in range(args.warmup):
        step(i)
    sampler = ClockSampler(int(str(nat.dev).split(":")[-1])) if clocks else None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = [step(args.warmup + i) for i in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = sampler.stop() if sampler else None
    ms_total = job_time_ms(e0.elapsed_time(e1), world, dist if world > 1 else None, nat.dev)
    v = outs[-1].cpu().numpy()
    ctx.close()
    return {"ms_total": ms_total, "stats": stats, "clocks": clk, "diag": v, "grads": grads[-1],
            "launches": int(sum(s["kernel_launches"] for s in stats))}


def planner_pick(args, nat, net):
    """The planner's recommendation over part counts including one (the exact
    one-part form), from the same probe context as measure_chosen's plan."""
    q, w = nat.q, nat.w
    counts = [p for p in RBMC_PART_COUNTS if p <= w.n_t]
    probe = nat.ctx(q.QSEL_MIXED, k=32)
    rec = q.qsel_cv_plan(probe, net, args.margin * args.target, max_overlap=PLAN_MAX_OVERLAP,
                         cost_pcg=KRON_PCG_COST, part_counts=[1] + counts)
    probe.close()
    return rec


def measure_chosen(args, nat, net, world, dist, rank, clocks=True):
    """Plan (part count >= 2, per-part overlaps, k) with the network, then time
    the RBMC form: W untimed and K timed steps, each one full pass with a new
    seed (plan + set seed + set theta + diag + traces + error estimate).
    Returns the measurements, the per-step estimates (for the accuracy over
    seeds) and the planner's recommendation over part counts including the
    exact one-part form."""
    import torch
    q, w, stream = nat.q, nat.w, nat.stream
    counts = [p for p in RBMC_PART_COUNTS if p <= w.n_t]

    def plan_on(ctx, with_exact=False):
        return q.qsel_cv_plan(ctx, net, args.margin * args.target, max_overlap=PLAN_MAX_OVERLAP,
                              cost_pcg=KRON_PCG_COST, part_counts=([1] if with_exact else []) + counts)

    probe = nat.ctx(q.QSEL_MIXED, k=32)
    plan = plan_on(probe)
    recommendation = plan_on(probe, with_exact=True)
    probe.close()
    ss = [int(x) for x in plan["slab_start"]]
    po = [int(x) for x in plan["part_overlap"]]
    k_run = int(plan["n_samples"])
    ctx = nat.ctx(q.QSEL_MIXED, n_parts=plan["n_parts"], slab_start=ss, overlap=min(po), k=k_run,
                  part_overlap=po)
    outs = [torch.empty(w.n, dtype=torch.float64, device=nat.dev) for _ in range(args.warmup + args.steps)]
    grads, errs = [], []

    def step(i):
        p = plan_on(ctx)
        if [int(x) for x in p["slab_start"]] != ss or [int(x) for x in p["part_overlap"]] != po \
                or p["n_samples"] != k_run:
            raise RuntimeError("the plan changed between steps at fixed theta")
        q.qsel_set_seed(ctx, 5000 + 97 * rank + i)
        q.qsel_set_theta(ctx, w.theta)
        q.qsel_diag_inv(ctx, outs[i])
        grads.append(np.asarray(q.qsel_trace_grads(ctx)))
        errs.append(q.qsel_error_estimate(ctx)[1])
        return q.qsel_stats(ctx)

    for i in range(args.warmup):
        step(i)
    sampler = ClockSampler(int(str(nat.dev).split(":")[-1])) if clocks else None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = [step(args.warmup + i) for i in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = sampler.stop() if sampler else None
    ms_total = job_time_ms(e0.elapsed_time(e1), world, dist if world > 1 else None, nat.dev)
    vs = [o.cpu().numpy() for o in outs]
    ctx.close()
    # the planner launches 5 kernels per separator distance (time coefficients,
    # Q_s values, features, network, per-slab reduction), 16 distances
    launches = int(sum(s["kernel_launches"] for s in stats)) + 80 * args.steps
    return {"plan": plan, "recommendation": recommendation, "slab_start": ss, "part_overlap": po, "k": k_run,
            "ms_total": ms_total, "stats": stats, "clocks": clk, "diags": vs, "grads": grads,
            "err_estimates": errs, "launches": launches}


def profile_pass(nat, ch, exact=False):
    """One pass of the RBMC plan (or of the exact one-part form) with
    per-launch event timing (class breakdown for the roofline), on a context
    of its own."""
    q = nat.q
    if exact:
        c = nat.ctx(q.QSEL_MIXED, n_parts=1, overlap=0, k=2, profile=1)
    else:
        c = nat.ctx(q.QSEL_MIXED, n_parts=len(ch["slab_start"]) - 1, slab_start=ch["slab_start"],
                    overlap=min(ch["part_overlap"]), k=ch["k"], part_overlap=ch["part_overlap"], profile=1)
    q.qsel_set_seed(c, 4242)
    q.qsel_diag_inv(c)
    q.qsel_trace_grads(c)
    st = q.qsel_stats(c)
    c.close()
    return st


# DRAM traffic of the Takahashi products on 9216-node blocks, two matrices per
# launch (the exact one-part form factored from both ends): dram__bytes_read.sum
# + dram__bytes_write.sum of one ncu capture (`bench.py --exact-pass
# grid96_nt8`, a full-size launch of this kernel), the mean of the Y launch
# (14.03 GB) and the Sigma launch (11.58 GB)
TAKAHASHI_TRAFFIC_9216_X2 = 12.81e9


def roofline_of(st, w, hbm_peak, hbm_src, tf32_peak, tf32_src, exact=False):
    """Dominant kernel class of one profiled pass (event time), with its
    algorithmic work per launch over its average event-timed launch."""
    from paper_2309_05435_gb300 import qsel as q
    classes = q.PROF_CLASSES
    cms, cwork, cl = st["class_ms"], st["class_work"], st["class_launches"]
    desc = {"gemm": "k_tc_gemm256 (Takahashi products: persistent 128x256 tiles, tcgen05 3xTF32 on operands "
                    "split once in HBM, TMA, double-buffered TMEM accumulators)",
            "sweep_update": "k_tc_update (persistent rank-256 sweep panel updates, tcgen05 3xTF32)",
            "spmm": "k_bt_spmm (block-tridiagonal sliced-ELL SpMM, PCG)",
            "pivot": "k_bsweep_pivot (64x64 double-float pivot-tile inverses, 2x2 block sweep)",
            "precond": "k_kron_transpose_in + k_kron_tc x6 (Kronecker preconditioner on tcgen05)"}
    cand = [i for i, nm in enumerate(classes) if nm in desc and cwork[i] > 0 and cms[i] > 0]
    dom = max(cand, key=lambda i: cms[i])
    name = classes[dom]
    if name == "spmm":
        ach = cwork[dom] / (cms[dom] * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "peak_source": hbm_src}
    elif name in ("gemm", "sweep_update"):
        ach = 3.0 * cwork[dom] / (cms[dom] * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": ach, "peak": tf32_peak, "unit": "TFLOP/s",
                "peak_source": tf32_src + "; achieved counts the three TF32 products of each 3xTF32 product"}
    elif name == "pivot":
        ach = cwork[dom] / (cms[dom] * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS / 15.0, "unit": "TFLOP/s",
                "peak_source": "FP32 CUDA-core rate from unit counts / 15 FP32 operations per double-float "
                               "multiply-subtract"}
    else:
        ach = cwork[dom] / (cms[dom] * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "peak_source": "FP32 CUDA-core rate from unit counts (152 x 128 x 2 x 2.07 GHz)"}
    traffic, traffic_src = None, "not captured for this kernel at this size"
    if exact and name == "gemm" and w.n_s == 9216:
        traffic = TAKAHASHI_TRAFFIC_9216_X2
        traffic_src = ("bytes per launch: ncu dram__bytes_read.sum + dram__bytes_write.sum of full-size launches "
                       "(bench.py --exact-pass grid96_nt8, two 9216^2 matrices per launch), mean of a Y and a Sigma "
                       "launch; about 3.8x the operand and output bytes (the right operand re-read once per group "
                       "of 16 tile rows), 1.3-2.1 TB/s at the tensor-bound rate")
    return {"kernel": desc[name], "class": name, **roof, "frac": roof["achieved"] / roof["peak"],
            "traffic": traffic, "traffic_source": traffic_src, "launches": int(cl[dom]),
            "avg_launch_ms": cms[dom] / max(1, cl[dom]),
            "timing": "per-launch CUDA events on the launching streams in a separate profiled pass of the "
                      "chosen form (the timed steps run without per-launch events)",
            "kernel_classes_ms_per_pass": {classes[i]: cms[i] for i in range(len(classes))}}


def slab_sample(nat, n_t_sample=4):
    """Exact one-part passes on the first n_t_sample slabs of the workload (its
    mesh, theta and observation mask) in FP64 and in the mixed form: the
    mixed form's per-result error against FP64 at the workload's block size,
    and the FP64 dense time per slab (factorisation, Takahashi)."""
    q, w = nat.q, nat.w
    mm = (nat.mesh, np.ascontiguousarray(nat.mask[:w.n_s * n_t_sample]))
    out = {}
    for name, prec in (("fp64", q.QSEL_FP64), ("mixed", q.QSEL_MIXED)):
        c = nat.ctx(prec, n_parts=1, overlap=0, k=2, mesh_mask=mm, n_t=n_t_sample)
        v = q.qsel_diag_inv(c)
        g = np.asarray(q.qsel_trace_grads(c))
        st = q.qsel_stats(c)
        c.close()
        out[name] = (v, g, st)
    v64, g64, st64 = out["fp64"]
    vm, gm, _ = out["mixed"]
    return {"slabs": n_t_sample, "mixed_vs_fp64": _errs(vm, gm, v64, g64),
            "fp64_factor_s_per_slab": st64["ms_factor"] / 1e3 / n_t_sample,
            "fp64_takahashi_s_per_slab": st64["ms_takahashi"] / 1e3 / max(1, n_t_sample - 1)}


def plain_fp64_time_to_target(args, nat, v_ex, t_ex, sample):
    """Plain FP64 RBMC (the workload's partition, block-Jacobi PCG) by the
    procedure of the metric: overlap n_l in {given, +1, +2}; for each, the
    error at k = 512 measured over --plain-seeds seeds (run in the mixed form,
    whose results agree with FP64 to the slab sample's error, far below the
    target); the samples needed for 1 % are k = 512 (eps / 0.01)^2, in
    512-sample runs whose averages reduce the error as 1/sqrt(runs); the
    time of each run is extrapolated from the FP64 dense time per slab of
    the slab sample over the run's factorised slabs (a lower bound: the FP64
    sampler and correction solves are not counted).  The cheapest n_l wins."""
    q, w = nat.q, nat.w
    ss = [int(x) for x in qi.balanced_slab_start(w.n_t, w.n_parts)]
    rows = []
    for nl in (w.overlap, w.overlap + 1, w.overlap + 2):
        vs, gs = [], []
        for sd in range(args.plain_seeds):
            c = nat.ctx(q.QSEL_MIXED, overlap=nl, k=512, seed=7000 + sd)
            vs.append(q.qsel_diag_inv(c))
            gs.append(np.asarray(q.qsel_trace_grads(c)))
            c.close()
        e = _seed_errors(vs, gs, v_ex, t_ex)
        eps = max(e["eps_diag"], *e["eps_traces"])
        k_need = 512 * (eps / args.target) ** 2
        runs = max(1, math.ceil(k_need / 512))
        fwd, bwd = _subdomain_slabs(w.n_t, ss, [nl] * w.n_parts)
        t_run = fwd * sample["fp64_factor_s_per_slab"] + bwd * sample["fp64_takahashi_s_per_slab"]
        rows.append({"overlap": nl, "k": 512, **e, "k_needed": k_need, "runs_of_512": runs,
                     "slabs_forward": fwd, "slabs_backward": bwd, "fp64_s_per_run_lower_bound": t_run,
                     "time_to_target_s_lower_bound": runs * t_run})
    best = min(rows, key=lambda r: r["time_to_target_s_lower_bound"])
    return {"procedure": plain_fp64_time_to_target.__doc__.split("\n\n")[0].replace("\n    ", " "),
            "settings": rows, "best": {"overlap": best["overlap"], "time_s": best["time_to_target_s_lower_bound"]},
            "extrapolated": True}


def run_native(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2309_05435_gb300 import build, qsel
    build.build()
    dev = f"cuda:{local}"
    stream = torch.cuda.current_stream()
    w = qi.workload(args.workload)
    nat = Native(qsel, w, stream, dev, chain=args.chain)

    if args.cv_params:
        net = qsel.qsel_cv_create(0)
        qsel.qsel_cv_set_params(net, np.load(args.cv_params))
        cv_info = {"loaded": os.path.basename(args.cv_params)}
    else:
        net, cv_info = train_control_variate(args)
        if args.save_cv_params:
            np.save(args.save_cv_params, qsel.qsel_cv_get_params(net))

    # the planner over part counts {1} + the RBMC counts picks the form; the
    # picked form is timed with W warm-up and K timed steps, the other one
    # (reported beside it) with at most 2 and 3
    chosen_exact = int(planner_pick(args, nat, net)["n_parts"]) == 1
    alt = argparse.Namespace(**{**vars(args), "warmup": min(args.warmup, 2), "steps": min(args.steps, 3)})
    a_ch, a_ex = (alt, args) if chosen_exact else (args, alt)
    ch = measure_chosen(a_ch, nat, net, world, dist, rank)
    ex = measure_exact(a_ex, nat, world, dist)
    ch["warmup"], ch["steps"] = a_ch.warmup, a_ch.steps
    ex["warmup"], ex["steps"] = a_ex.warmup, a_ex.steps
    ms_per_step = (ex if chosen_exact else ch)["ms_total"] / args.steps

    # end to end through the public API with host buffers: create from pinned
    # host arrays, plan, diag to pinned host memory, traces, destroy
    h2d = (nat.mesh.c_diag.nbytes + nat.mesh.g_rowptr.nbytes + nat.mesh.g_col.nbytes + nat.mesh.g_val.nbytes
           + nat.mask.nbytes + 3 * 8 + 8)
    d2h = w.n * 8 + 3 * 8
    e2e_s = None
    if args.e2e_steps > 0:
        pin = lambda a: torch.from_numpy(a).pin_memory().numpy()  # noqa: E731
        c_pin, gv_pin, rp_pin, gc_pin, mk_pin = (pin(nat.mesh.c_diag), pin(nat.mesh.g_val), pin(nat.mesh.g_rowptr),
                                                 pin(nat.mesh.g_col), pin(nat.mask))
        diag_host = torch.empty(w.n, dtype=torch.float64).pin_memory().numpy()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(args.e2e_steps):
            if chosen_exact:
                c2 = qsel.qsel_create(w.n_s, w.n_t, c_pin, rp_pin, gc_pin, gv_pin, mk_pin, w.sigma, w.theta,
                                      n_parts=1, overlap=0, n_samples=2, precision=qsel.QSEL_MIXED,
                                      pcg_tol=w.pcg_tol, cuda_stream=stream.cuda_stream)
            else:
                c2 = qsel.qsel_create(w.n_s, w.n_t, c_pin, rp_pin, gc_pin, gv_pin, mk_pin, w.sigma, w.theta,
                                      n_parts=len(ch["slab_start"]) - 1, slab_start=ch["slab_start"],
                                      overlap=min(ch["part_overlap"]), n_samples=ch["k"], seed=6000 + i,
                                      precision=qsel.QSEL_MIXED, pcg_tol=w.pcg_tol, cuda_stream=stream.cuda_stream,
                                      part_overlap=ch["part_overlap"], preconditioner=qsel.QSEL_PRECOND_KRON)
            # the plan over part counts including the exact form, as in the timed steps
            p = qsel.qsel_cv_plan(c2, net, args.margin * args.target, max_overlap=PLAN_MAX_OVERLAP,
                                  cost_pcg=KRON_PCG_COST,
                                  part_counts=[1] + [c for c in RBMC_PART_COUNTS if c <= w.n_t])
            if (int(p["n_parts"]) == 1) != chosen_exact:
                raise RuntimeError("the plan changed between calls at fixed theta")
            qsel.qsel_diag_inv(c2, diag_host)
            qsel.qsel_trace_grads(c2)
            c2.close()
        torch.cuda.synchronize()
        el = torch.tensor([time.perf_counter() - t0], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(el, op=dist.ReduceOp.MAX)
        e2e_s = float(el.item()) / (args.e2e_steps * world)

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    hbm_peak, hbm_src = measured_peaks()
    tf32_peak, tf32_src = tf32_peak_tflops()
    st_prof = profile_pass(nat, ch, exact=chosen_exact)
    roof = roofline_of(st_prof, w, hbm_peak, hbm_src, tf32_peak, tf32_src, exact=chosen_exact)
    roof_rbmc = None
    if chosen_exact:
        roof_rbmc = roofline_of(profile_pass(nat, ch), w, hbm_peak, hbm_src, tf32_peak, tf32_src)

    # the exact one-part form in the same precision is also the reference of
    # the RBMC form's accuracy (its own error against FP64 from the slab sample)
    v_ex, t_ex, st_ex = ex["diag"], ex["grads"], ex["stats"][-1]
    accuracy = None
    sample = plain = None
    if not args.no_accuracy:
        sample = slab_sample(nat)
        rb = _seed_errors(ch["diags"], ch["grads"], v_ex, t_ex)
        own = sample["mixed_vs_fp64"]
        exact_acc = {"eps_diag": own["eps_diag_rms"], "eps_diag_p99": own["eps_diag_p99"],
                     "eps_traces": own["eps_traces"], "against": "FP64 on the slab sample",
                     "meets_1pct": bool(own["eps_diag_rms"] <= 0.01 and max(own["eps_traces"]) <= 0.01)}
        accuracy = {"reference": "exact one-part selected inversion in the mixed form on the GPU (n_p = 1); its "
                                 "own error against FP64 is `slab_sample.mixed_vs_fp64` at this block size",
                    "chosen": exact_acc if chosen_exact else rb, "rbmc": rb, "exact": exact_acc,
                    "rbmc_error_estimates": ch["err_estimates"], "slab_sample": sample}
        if args.plain_seeds > 0:
            plain = plain_fp64_time_to_target(args, nat, v_ex, t_ex, sample)
    chosen_ok = accuracy["chosen"]["meets_1pct"] if accuracy else None
    forms = {
        "exact": {"form": "exact one-part selected inversion (n_p = 1), mixed precision",
                  "s_per_pass": ex["ms_total"] / ex["steps"] / 1e3, "warmup": ex["warmup"], "steps": ex["steps"],
                  "phases_ms": {"factor": st_ex["ms_factor"], "takahashi": st_ex["ms_takahashi"]},
                  "planner_model_cost_s": ch["plan"]["single_part_cost"], "gpu_launches": ex["launches"],
                  "clocks": ex["clocks"]},
        "rbmc": {"form": "mixed-precision RBMC at the planner's part count >= 2", "s_per_pass":
                 ch["ms_total"] / ch["steps"] / 1e3, "warmup": ch["warmup"], "steps": ch["steps"],
                 "n_parts": len(ch["slab_start"]) - 1,
                 "slab_start": ch["slab_start"], "overlap": ch["part_overlap"], "n_samples": ch["k"],
                 "planner_model_cost_s": ch["plan"]["predicted_cost"], "gpu_launches": ch["launches"],
                 "phases_ms": {k: ch["stats"][-1]["ms_" + k] for k in
                               ("rhs", "pcg", "factor", "takahashi", "correction", "total")},
                 "pcg_iterations": ch["stats"][-1]["pcg_iterations"], "clocks": ch["clocks"],
                 "roofline": roof_rbmc},
    }

    cpu = None
    if not args.no_cpu_baseline and world == 1:   # the CPU baseline is an N = 1 figure
        est, spent, desc = oracle_sample(w, exact=chosen_exact)
        cpu = {"value": est, "unit": "s", "cores": cpu_cores(), "kind": "oracle", "sample": desc,
               "sample_seconds": spent}

    cm = ex if chosen_exact else ch
    st = cm["stats"][-1]
    plan = ch["plan"]
    planner = ("the learned control-variate planner over part counts {1, %s} (per-part overlap and k for %g RMS "
               "relative error; n_p = 1 is the exact one-part form)"
               % (", ".join(str(c) for c in RBMC_PART_COUNTS if c <= w.n_t), args.target))
    form = (("exact one-part selected inversion (mixed precision: FP32 tiles on tcgen05 3xTF32, double-float "
             "pivots), chosen by " if chosen_exact else
             "mixed precision RBMC (FP32 PCG with the Kronecker grid preconditioner on tcgen05 + FP64 refinement; "
             "FP32 tiles on tcgen05 3xTF32 + double-float pivots), chosen by ") + planner)
    result = {
        "metric": METRIC,
        "value": job_value_s(cm["ms_total"], args.steps, world),
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic (seeded grid FEM mesh, Philox noise)",
        "config": {"workload": f"{w.name}: {w.m}x{w.m} grid, n_t={w.n_t}, n={w.n}, kappa={w.kappa}, "
                               f"rho={w.rho}, {int(w.obs_frac * 100)}% observed",
                   "form": form, "n_parts": 1 if chosen_exact else len(ch["slab_start"]) - 1,
                   "slab_start": [0, w.n_t] if chosen_exact else ch["slab_start"],
                   "overlap": [0] if chosen_exact else ch["part_overlap"],
                   "n_samples": 0 if chosen_exact else ch["k"], "pcg_tol": w.pcg_tol,
                   "seeds": "a new Philox seed every step",
                   "l2": ("inputs larger than L2 (each 9216^2 FP32 block 340 MB)" if chosen_exact else
                          "inputs larger than L2 (samples alone %.2f GB)" % (w.n * ch["k"] * 8 / 1e9)),
                   "parallelism": f"replicas x{world}"},
        "roofline": roof,
        "phases_ms": {"rhs": st["ms_rhs"], "pcg": st["ms_pcg"], "factor": st["ms_factor"],
                      "takahashi": st["ms_takahashi"], "correction": st["ms_correction"],
                      "total": st["ms_total"]},
        "pcg_iterations": st["pcg_iterations"],
        "gpu_launches": cm["launches"],
        "chosen_meets_target": chosen_ok,
        "plan": {"chosen_n_parts": int(ch["recommendation"]["n_parts"]),
                 "chosen_predicted_cost_s": ch["recommendation"]["predicted_cost"],
                 "rbmc_n_parts": plan["n_parts"], "rbmc_n_samples": plan["n_samples"],
                 "rbmc_part_overlap": ch["part_overlap"], "rbmc_predicted_err": plan["predicted_err"],
                 "rbmc_predicted_cost_s": plan["predicted_cost"], "feasible": plan["feasible"],
                 "margin": args.margin},
        "cv_training": cv_info,
        "forms": forms,
        "plain_fp64": plain,
        "speedup_chosen_vs_plain_fp64": (plain["best"]["time_s"] / (ms_per_step / 1e3)) if plain else None,
        "clocks": cm["clocks"],
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "cpu_baseline": cpu,
        "accuracy": accuracy,
    }
    if args.secondary and args.secondary != w.name:
        result["secondary"] = secondary_workload(args, qsel, qi.workload(args.secondary), stream, dev, net)
    print(json.dumps(result), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def secondary_workload(args, q, w2, stream, dev, net):
    """The planner's best RBMC plan and the exact one-part form on a second
    workload (one warm-up and two timed steps), with the accuracy over those
    seeds and the form the planner picks over part counts including one."""
    nat = Native(q, w2, stream, dev, chain=args.chain)
    a2 = argparse.Namespace(**{**vars(args), "warmup": 1, "steps": 2})
    ch = measure_chosen(a2, nat, net, 1, None, 0, clocks=False)
    t_exact, v_ex, t_ex, _ = nat.exact(q.QSEL_MIXED)
    t_rbmc = ch["ms_total"] / 2 / 1e3
    picked_exact = int(ch["recommendation"]["n_parts"]) == 1
    return {"workload": w2.name, "picked": "exact one-part" if picked_exact else "rbmc",
            "picked_s_per_pass": t_exact if picked_exact else t_rbmc,
            "rbmc": {"s_per_pass": t_rbmc, "n_parts": len(ch["slab_start"]) - 1, "overlap": ch["part_overlap"],
                     "n_samples": ch["k"], "accuracy": _seed_errors(ch["diags"], ch["grads"], v_ex, t_ex)},
            "exact_one_part_s": t_exact}


# ----------------------------------------------------------------------------
# reference arm: the CPU oracle
# ----------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = qi.workload(args.workload)
    # steps of a few seconds at any block size: above 4096 nodes each step
    # samples the leading half of every block, scaled by the ratio of one
    # full-block sample to one half-block sample taken untimed first, so that
    # the driver's W + K steps stay within minutes
    frac = 0.5 if w.n_s > 4096 else 1.0
    ratio = 1.0
    if frac < 1.0:
        full, _, _ = oracle_sample(w)
        half, _, _ = oracle_sample(w, frac=frac)
        ratio = full / half
    for _ in range(max(0, args.warmup - (2 if frac < 1.0 else 0))):
        oracle_sample(w, frac=frac)
    vals, spent, desc = [], 0.0, ""
    for _ in range(args.steps):
        est, sp, desc = oracle_sample(w, frac=frac)
        vals.append(est * ratio)
        spent += sp
    if frac < 1.0:
        desc += f"; scaled by {ratio:.3f}, the measured ratio of a full-block to a half-block sample"
    v = float(np.mean(vals))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": spent / args.steps * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded grid FEM mesh)",
        "config": {"workload": w.name, "form": "CPU FP64 oracle: exact one-part selected inversion "
                   "(block Cholesky + Takahashi), the form the planner picks on this workload"},
        "cpu_baseline": {"value": v, "unit": "s", "kind": "oracle", "cores": cpu_cores(), "sample": desc},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def oracle_end_to_end(name: str):
    """The CPU oracle end to end at a workload's own settings: exact samples by
    its direct block-tridiagonal solve (the sampler), then Algorithm 4 and the
    trace estimator (factorisation, Takahashi recursion, correction solves) for
    every part.  Returns (seconds, phase seconds)."""
    from oracle import qsel_oracle as o
    w = qi.workload(name)
    mesh, mask = workload_inputs(w)
    model = o.model_from_csr(w.n_s, w.n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val, mask, w.sigma)
    for _ in range(2 if w.n < 100_000 else 1):   # small workloads: the second, warm run
        t0 = time.perf_counter()
        X = o.samples(model, w.theta, 1000, w.n_samples)
        t1 = time.perf_counter()
        o.rbmc(model, w.theta, qi.balanced_slab_start(w.n_t, w.n_parts), w.overlap, X)
        t2 = time.perf_counter()
    return t2 - t0, {"sampler": t1 - t0, "rbmc": t2 - t1}


def run_exact_pass(args):
    """--exact-pass WORKLOAD: one exact one-part pass in the mixed form (the
    command the kernel captures under profiles/ run); prints its time."""
    import torch
    from paper_2309_05435_gb300 import build, qsel
    build.build()
    w = qi.workload(args.exact_pass)
    mesh, mask = workload_inputs(w)
    c = qsel.qsel_create(w.n_s, w.n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val, mask, w.sigma, w.theta,
                         n_parts=1, overlap=0, n_samples=2, precision=qsel.QSEL_MIXED,
                         chain=qsel.QSEL_CHAIN_FORWARD if args.chain == "forward" else qsel.QSEL_CHAIN_TWO_ENDED)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    qsel.qsel_diag_inv(c)
    torch.cuda.synchronize()
    st = qsel.qsel_stats(c)
    c.close()
    print(json.dumps({"mode": "exact_pass", "workload": w.name, "chain": args.chain, "s": time.perf_counter() - t0,
                      "factor_ms": st["ms_factor"], "takahashi_ms": st["ms_takahashi"]}), flush=True)


def run_kron_apply(args):
    """--kron-apply WORKLOAD: one apply of the mixed form's Kronecker
    preconditioner to 256 seeded columns (the command the tensor-core passes
    are captured with under profiles/); prints its host-side time."""
    from paper_2309_05435_gb300 import build, qsel
    build.build()
    w = qi.workload(args.kron_apply)
    mesh, mask = workload_inputs(w)
    c = qsel.qsel_create(w.n_s, w.n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val, mask, w.sigma, w.theta,
                         n_parts=2, overlap=1, n_samples=256, precision=qsel.QSEL_MIXED,
                         preconditioner=qsel.QSEL_PRECOND_KRON)
    R = qi.seeded_normal((w.n, 256), 17)
    t0 = time.perf_counter()
    Z = qsel.qsel_debug_apply_precond(c, R)
    c.close()
    print(json.dumps({"mode": "kron_apply", "workload": w.name, "s_with_host_copies": time.perf_counter() - t0,
                      "max_abs": float(np.max(np.abs(Z)))}), flush=True)


def run_oracle_e2e(args):
    """--oracle-e2e: the oracle end to end on the listed workloads with all host
    cores, and in a child process limited to one BLAS / OpenMP thread on the
    workloads in --oracle-e2e-single; one JSON line per run."""
    for name in [x for x in args.oracle_e2e.split(",") if x]:
        s, ph = oracle_end_to_end(name)
        print(json.dumps({"mode": "oracle_e2e", "workload": name, "threads": "all", "cores": cpu_cores(),
                          "seconds": s, "phases_s": ph}), flush=True)
    env = dict(os.environ)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[var] = "1"
    for name in [x for x in args.oracle_e2e_single.split(",") if x]:
        p = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-e2e", name,
                            "--oracle-e2e-single", ""], env=env, capture_output=True, text=True, timeout=3600)
        for line in p.stdout.strip().splitlines():
            d = json.loads(line)
            d["threads"] = 1
            print(json.dumps(d), flush=True)


def run_sweep(args):
    """Time one pass (after one warm-up) and measure the error against the exact
    single-subdomain FP64 result for each requested (form, n_p, n_l, k), with
    the error definitions of the time-to-1% metric: eps_diag = RMS over nodes
    and seeds of the relative error, eps_j = RMS over seeds per trace."""
    import torch
    from paper_2309_05435_gb300 import build, qsel
    build.build()
    w = qi.workload(args.workload)
    mesh, mask = workload_inputs(w)
    stream = torch.cuda.current_stream()
    ref = qsel.qsel_create(w.n_s, w.n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val, mask, w.sigma,
                           w.theta, n_parts=1, overlap=0, n_samples=1, cuda_stream=stream.cuda_stream)
    v_ex = qsel.qsel_diag_inv(ref)
    t_ex = qsel.qsel_trace_grads(ref)
    ref.close()
    rows = []
    for entry in args.sweep.split(","):
        form, np_, nl, k = entry.split(":")
        prec = qsel.QSEL_MIXED if form == "mixed" else qsel.QSEL_FP64
        errs_d, errs_t, times, iters = [], [], [], []
        for sd in range(args.seeds):
            ctx = qsel.qsel_create(w.n_s, w.n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val, mask,
                                   w.sigma, w.theta, n_parts=int(np_), overlap=int(nl), n_samples=int(k),
                                   seed=2000 + sd, precision=prec, pcg_tol=w.pcg_tol,
                                   cuda_stream=stream.cuda_stream)
            out = torch.empty(w.n, dtype=torch.float64, device="cuda")
            for rep in range(2 if sd == 0 else 1):
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                qsel.qsel_set_theta(ctx, w.theta)
                qsel.qsel_diag_inv(ctx, out)
                g = qsel.qsel_trace_grads(ctx)
                e1.record(stream)
                torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            iters.append(qsel.qsel_stats(ctx)["pcg_iterations"])
            ctx.close()
            v = out.cpu().numpy()
            errs_d.append(((v - v_ex) / v_ex) ** 2)
            errs_t.append([((a - b) / b) ** 2 for a, b in zip(g, t_ex)])
        ed = np.array(errs_d)
        row = {"form": form, "n_parts": int(np_), "overlap": int(nl), "n_samples": int(k),
               "ms": float(np.median(times)), "pcg_iterations": int(np.median(iters)),
               "eps_diag": float(np.sqrt(ed.mean())),
               "eps_diag_p99": float(np.quantile(np.sqrt(ed.mean(axis=0)), 0.99)),
               "eps_traces": [float(np.sqrt(np.mean([e[j] for e in errs_t]))) for j in range(3)],
               "seeds": args.seeds}
        row["meets_1pct"] = bool(max(row["eps_diag"], *row["eps_traces"]) <= 0.01)
        print(json.dumps(row), flush=True)
        rows.append(row)
    return rows


def run_cv_eval(args):
    """Held-out evaluation of the learned control variate: 64 x 64 grid,
    n_t = 128, 8 parts, 25 % observed, scrambled-Sobol theta (seed 2, apart
    from the training grid).  Per theta: planned mixed RBMC (plan, one run, at
    most one corrective run; the chosen --preconditioner) against plain RBMC
    (block-Jacobi PCG) at overlap 2 that doubles k
    from 32 (then averages 512-sample batches) until its error estimate meets
    the target -- in mixed precision on every theta and in FP64 on the first
    --cv-fp64-thetas.  Errors are also measured against the exact
    single-subdomain result.  Wall-clock seconds include context creation."""
    import torch
    from paper_2309_05435_gb300 import build, qsel
    from paper_2309_05435_gb300 import cv as cvm
    build.build()
    if args.cv_params:
        net = qsel.qsel_cv_create(0)
        qsel.qsel_cv_set_params(net, np.load(args.cv_params))
        info = {"loaded": os.path.basename(args.cv_params)}
    else:
        net, info = train_control_variate(args)
    print(json.dumps({"cv_training": info}), flush=True)
    mesh = qi.grid_mesh(64)
    n_t = 128
    spec = cvm.ModelSpec(mesh, n_t, qi.obs_mask(4096 * n_t, 0.25, 6), 0.5, qi.balanced_slab_start(n_t, 8))
    rows = []
    for i, th in enumerate(cvm.sobol_thetas(args.cv_eval_thetas, seed=2)):
        # exact single-subdomain reference (mixed: its error, ~1e-4, is far below the target)
        ref = qsel.qsel_create(spec.n_s, n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val, spec.mask,
                               spec.sigma, th, n_parts=1, overlap=0, n_samples=1, precision=qsel.QSEL_MIXED)
        v_ex = qsel.qsel_diag_inv(ref)
        ref.close()

        def eps(v):
            return float(np.sqrt(np.mean(((v - v_ex) / v_ex) ** 2)))

        row = {"theta": [round(x, 4) for x in th], "target": args.target}
        kron = args.preconditioner == "kron"
        pl = cvm.solve_planned(spec, th, net, args.target, max_overlap=args.max_overlap, margin=args.margin,
                               preconditioner=qsel.QSEL_PRECOND_KRON if kron else qsel.QSEL_PRECOND_BLOCK_JACOBI,
                               cost_pcg=KRON_PCG_COST if kron else 0.0)
        row["planned_mixed"] = {"k": pl["k"], "part_overlap": pl["part_overlap"], "runs": len(pl["runs"]),
                                "samples": pl["samples_drawn"], "err_estimate": pl["err"],
                                "predicted_err": pl["plan"]["predicted_err"], "eps_vs_exact": eps(pl["v"]),
                                "plan_s": pl["plan_s"], "wall_s": pl["wall_s"], "met": pl["met"]}
        forms = [("plain_mixed", qsel.QSEL_MIXED)]
        if i < args.cv_fp64_thetas:
            forms.append(("plain_fp64", qsel.QSEL_FP64))
        for name, prec in forms:
            r = cvm.solve_plain(spec, th, args.target, overlap=2, precision=prec)
            row[name] = {"k_total": r["k"], "runs": len(r["runs"]), "samples": r["samples_drawn"],
                         "err_estimate": r["err"], "eps_vs_exact": eps(r["v"]), "wall_s": r["wall_s"],
                         "met": r["met"]}
        # the literal reading (estimate w_i^2 - c_hat_i, add c_hat_i back) is
        # the plain estimator for any prediction: the same runs, samples and
        # error as plain RBMC at the same settings
        row["literal_residual_form"] = {"same_as": "plain_mixed", "samples": row["plain_mixed"]["samples"],
                                        "wall_s": row["plain_mixed"]["wall_s"],
                                        "err_estimate": row["plain_mixed"]["err_estimate"]}
        if i < args.cv_controls:
            # control: plain RBMC at each fixed overlap (doubling k), the best
            # of them chosen in hindsight
            by_nl = {}
            for nl in (1, 2, 4, 8):
                r = cvm.solve_plain(spec, th, args.target, overlap=nl, precision=qsel.QSEL_MIXED)
                by_nl[nl] = {"samples": r["samples_drawn"], "runs": len(r["runs"]), "wall_s": r["wall_s"],
                             "device_ms": r["device_ms"], "err_estimate": r["err"], "eps_vs_exact": eps(r["v"]),
                             "met": r["met"]}
            best = min((v for v in by_nl.items() if v[1]["met"]), key=lambda kv: kv[1]["wall_s"], default=None)
            row["plain_mixed_by_overlap"] = by_nl
            if best is not None:
                row["best_fixed_overlap"] = {"overlap": best[0], "wall_s": best[1]["wall_s"],
                                             "speedup_planned_vs_best_fixed": best[1]["wall_s"] / pl["wall_s"]}
        row["speedup_vs_plain_mixed"] = row["plain_mixed"]["wall_s"] / pl["wall_s"]
        if "plain_fp64" in row:
            row["speedup_vs_plain_fp64"] = row["plain_fp64"]["wall_s"] / pl["wall_s"]
        print(json.dumps(row), flush=True)
        rows.append(row)
    summ = {"summary": "cv_eval", "thetas": len(rows),
            "planned_met": sum(r["planned_mixed"]["met"] for r in rows),
            "median_planned_wall_s": float(np.median([r["planned_mixed"]["wall_s"] for r in rows])),
            "median_plain_mixed_wall_s": float(np.median([r["plain_mixed"]["wall_s"] for r in rows])),
            "median_speedup_vs_plain_mixed": float(np.median([r["speedup_vs_plain_mixed"] for r in rows])),
            "planned_samples_total": int(sum(r["planned_mixed"]["samples"] for r in rows)),
            "plain_mixed_samples_total": int(sum(r["plain_mixed"]["samples"] for r in rows))}
    fp = [r for r in rows if "plain_fp64" in r]
    if fp:
        summ["speedup_vs_plain_fp64"] = [r["speedup_vs_plain_fp64"] for r in fp]
    ctl = [r for r in rows if "best_fixed_overlap" in r]
    if ctl:
        summ["speedup_vs_best_fixed_overlap"] = [r["best_fixed_overlap"]["speedup_planned_vs_best_fixed"] for r in ctl]
        summ["best_fixed_overlaps"] = [r["best_fixed_overlap"]["overlap"] for r in ctl]
    print(json.dumps(summ), flush=True)


def run_batch(args):
    """Uneven batch (grids 16x16 to 64x64, n_t 8 to 128, 2-8 parts, overlap 1,
    128 samples, mixed precision, PCG to 1e-8, theta per model): one captured
    graph over a stream pool, replayed; against the same models solved one
    after another by separate contexts with the same (tuned) settings.  Both
    sides time device work with CUDA events; the graph's W warm-up replays are
    untimed and its K replays are timed."""
    import torch
    from paper_2309_05435_gb300 import build, qsel
    build.build()
    specs = qi.uneven_batch(args.batch_models)
    meshes = {}
    models = []
    for b in specs:
        if b.m not in meshes:
            meshes[b.m] = qi.grid_mesh(b.m)
        me = meshes[b.m]
        models.append({"n_s": b.n_s, "n_t": b.n_t, "c_diag": me.c_diag, "g_rowptr": me.g_rowptr, "g_col": me.g_col,
                       "g_val": me.g_val, "obs_mask": b.mask(), "sigma": b.sigma})
    opts = dict(n_samples=128, seed=1000, precision=qsel.QSEL_MIXED, pcg_tol=1e-8, pcg_max_iter=20000)
    t0 = time.perf_counter()
    bt = qsel.qsel_create_batch(models, [b.theta for b in specs], [(b.n_parts, None) for b in specs],
                                [b.overlap for b in specs], n_streams=args.batch_streams,
                                autotune=not args.no_autotune, **opts)
    t_create = time.perf_counter() - t0
    for _ in range(max(1, args.warmup)):
        qsel.qsel_batch_run(bt)
    info0 = qsel.qsel_batch_info(bt)
    reps = []
    for _ in range(args.steps):
        qsel.qsel_batch_run(bt)
        reps.append(qsel.qsel_batch_info(bt)["ms_replay"])
    tuning = [qsel.qsel_batch_tuning(bt, i) for i in range(len(specs))]
    iters = [qsel.qsel_batch_stats(bt, i)["pcg_iterations"] for i in range(len(specs))]
    v_batch = [qsel.qsel_batch_diag_inv(bt, i) for i in range(min(4, len(specs)))]
    bt.close()
    torch.cuda.synchronize()
    # one model after another, same settings, device time per pipeline
    seq_ms, same = 0.0, True
    for i, (b, mdl) in enumerate(zip(specs, models)):
        tu = tuning[i]
        ctx = qsel.qsel_create(b.n_s, b.n_t, mdl["c_diag"], mdl["g_rowptr"], mdl["g_col"], mdl["g_val"],
                               mdl["obs_mask"], b.sigma, b.theta, n_parts=b.n_parts, overlap=b.overlap,
                               n_samples=128, seed=1000 + i, precision=qsel.QSEL_MIXED, pcg_tol=1e-8,
                               pcg_max_iter=20000, precond_block=tu["precond_block"],
                               tensor_passes=tu["tensor_passes"] if tu["tensor_passes"] > 0 else -1)
        v = ctx.diag_inv()
        seq_ms += ctx.stats()["ms_total"]
        if i < len(v_batch):
            same = same and bool(np.array_equal(v, v_batch[i]))
        ctx.close()
    replay_ms = float(np.median(reps))
    n_total = sum(b.n for b in specs)
    print(json.dumps({
        "mode": "batch", "models": len(specs), "nodes_total": int(n_total),
        "grid_sides": sorted({b.m for b in specs}), "n_t_range": [min(b.n_t for b in specs), max(b.n_t for b in specs)],
        "replay_ms": replay_ms, "replays": reps, "sequential_ms": seq_ms, "speedup_vs_sequential": seq_ms / replay_ms,
        "streams": info0["n_streams"], "capture_ms": info0["ms_capture"], "autotune_ms": info0["ms_autotune"],
        "create_s": t_create, "launches_per_replay": info0["launches_per_replay"],
        "pcg_iterations_max": int(max(iters)), "first_models_identical_to_separate_contexts": same,
        "tuning_counts": {f"{k}": sum(1 for t in tuning if (t["precond_block"], t["tensor_passes"]) == k)
                          for k in sorted({(t["precond_block"], t["tensor_passes"]) for t in tuning})},
    }), flush=True)


def run_lanczos_eval(args):
    """The preconditioned Krylov sampler (Algorithm 5.1) against the PCG
    perturbation sampler at the workload's fixed settings, mixed dense part:
    per Krylov dimension m, one pass after one warm-up (CUDA events), the
    sampler's share of it, and the RBMC error against the exact one-part
    result (the same error definitions as the bench line)."""
    import torch
    from paper_2309_05435_gb300 import build, qsel
    build.build()
    w = qi.workload(args.workload)
    mesh, mask = workload_inputs(w)
    stream = torch.cuda.current_stream()
    ref = qsel.qsel_create(w.n_s, w.n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val, mask, w.sigma,
                           w.theta, n_parts=1, overlap=0, n_samples=1, cuda_stream=stream.cuda_stream)
    v_ex = qsel.qsel_diag_inv(ref)
    t_ex = qsel.qsel_trace_grads(ref)
    ref.close()
    entries = [("pcg", 0)] + [("lanczos", int(m)) for m in args.lanczos_eval.split(",")]
    for name, m in entries:
        kw = dict(sampler=qsel.QSEL_SAMPLER_LANCZOS, lanczos_steps=m) if name == "lanczos" else {}
        ctx = qsel.qsel_create(w.n_s, w.n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val, mask, w.sigma,
                               w.theta, n_parts=w.n_parts, overlap=w.overlap, n_samples=w.n_samples, seed=2000,
                               precision=qsel.QSEL_MIXED, pcg_tol=w.pcg_tol, cuda_stream=stream.cuda_stream, **kw)
        for _ in range(2):
            qsel.qsel_set_theta(ctx, w.theta)
            v = qsel.qsel_diag_inv(ctx)
            g = qsel.qsel_trace_grads(ctx)
        st = qsel.qsel_stats(ctx)
        ctx.close()
        r = (v - v_ex) / v_ex
        print(json.dumps({"sampler": name, "lanczos_steps": m, "workload": w.name, "ms_total": st["ms_total"],
                          "ms_sampler": st["ms_rhs"] + st["ms_pcg"], "pcg_iterations": st["pcg_iterations"],
                          "eps_diag_rms": float(np.sqrt(np.mean(r ** 2))),
                          "eps_traces": [float(abs(a - b) / abs(b)) for a, b in zip(g, t_ex)]}), flush=True)


def run_hyper_eval(args):
    """Posterior mean and hyperparameter gradient (qsel_loglik_grad) at the
    workload: per precision one evaluation after one warm-up, CUDA events on
    the library's stream around set_theta + the gradient (pipeline, posterior
    mean, quadratic forms, prior term), then the posterior mean alone.  The
    data are seeded normal values on the observed nodes (the cost does not
    depend on them)."""
    import torch
    from paper_2309_05435_gb300 import build, qsel
    build.build()
    w = qi.workload(args.workload)
    mesh, mask = workload_inputs(w)
    stream = torch.cuda.current_stream()
    y = qi.seeded_normal((int(np.count_nonzero(mask)), 1), 7)[:, 0]
    out = {}
    for name, prec, pre in (("mixed", qsel.QSEL_MIXED, qsel.QSEL_PRECOND_KRON),
                            ("fp64", qsel.QSEL_FP64, qsel.QSEL_PRECOND_BLOCK_JACOBI)):
        ctx = qsel.qsel_create(w.n_s, w.n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val, mask, w.sigma,
                               w.theta, n_parts=w.n_parts, overlap=w.overlap, n_samples=w.n_samples, seed=3000,
                               precision=prec, pcg_tol=w.pcg_tol, cuda_stream=stream.cuda_stream, preconditioner=pre)
        qsel.qsel_set_data(ctx, y)
        qsel.qsel_set_theta(ctx, w.theta)
        qsel.qsel_loglik_grad(ctx)
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        qsel.qsel_set_theta(ctx, w.theta)
        g, (prior, tr, quad) = qsel.qsel_loglik_grad(ctx, with_terms=True)
        e1.record(stream)
        qsel.qsel_posterior_mean(ctx)
        e2.record(stream)
        torch.cuda.synchronize()
        st = qsel.qsel_stats(ctx)
        ctx.close()
        out[name] = {"grad_ms": e0.elapsed_time(e1), "pipeline_ms": st["ms_total"],
                     "posterior_mean_ms": e1.elapsed_time(e2), "grad": [float(x) for x in g],
                     "prior_logdet_grad": [float(x) for x in prior], "traces": [float(x) for x in tr],
                     "quadratic_forms": [float(x) for x in quad]}
    rel = [abs(a - b) / max(abs(b), 1e-300) for a, b in zip(out["mixed"]["grad"], out["fp64"]["grad"])]
    print(json.dumps({"mode": "hyper_eval", "workload": w.name, "n_parts": w.n_parts, "overlap": w.overlap,
                      "n_samples": w.n_samples, **out,
                      "speedup_mixed_vs_fp64": out["fp64"]["grad_ms"] / out["mixed"]["grad_ms"],
                      "grad_rel_diff_mixed_vs_fp64": rel,
                      "note": "same seed, so the same Philox noise and samples up to the solves' tolerance: the "
                              "difference is the mixed form's arithmetic"}), flush=True)


def main():
    args = parse_args()
    if args.oracle_sample:
        est, spent, _ = oracle_sample(qi.workload(args.workload))
        print(json.dumps({"est": est, "spent": spent}), flush=True)
        return
    if args.kron_apply:
        run_kron_apply(args)
        return
    if args.exact_pass:
        run_exact_pass(args)
        return
    if args.oracle_e2e is not None:
        run_oracle_e2e(args)
        return
    if args.hyper_eval:
        run_hyper_eval(args)
        return
    if args.lanczos_eval:
        run_lanczos_eval(args)
        return
    if args.batch:
        run_batch(args)
        return
    if args.cv_eval:
        run_cv_eval(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
