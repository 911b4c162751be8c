#!/usr/bin/env python
"""Benchmark: time to diag(Q^-1) + tr(Q^-1 dQ/dtheta_j) on one GB300.

One step = one pass of the whole hot path through the C ABI on a resident
context: qsel_set_theta (invalidates), qsel_diag_inv (perturbation RHS,
multi-RHS PCG, per-subdomain block factorisation + Takahashi, RB correction)
and qsel_trace_grads.  Workload: 64 x 64 grid (n_s = 4096), n_t = 64
(n = 262,144), kappa = 0.2, rho = 0.95, 25 % observed, 8 time subdomains,
overlap 2, 256 samples, PCG to 1e-10 -- synthetic, seeded.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

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
# DRAM bytes per FLOP of k_gemm64 from one ncu capture (profiles/k_gemm64_grid64_nt16_fp64.md)
GEMM64_DRAM_BYTES_PER_FLOP = 7.808e9 / 2.749e11
L2_BYTES = 126 * 2 ** 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", default="grid64_nt64")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


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
def oracle_sample(w):
    """Time the oracle's per-slab dense work at the workload's block size: block
    Cholesky and Takahashi of a 2-slab chain of Q's blocks.  The full oracle
    run needs sum_p T_p slab units of factor + Takahashi plus n_t units of
    factor for its direct sampler; returns (extrapolated seconds, sample
    seconds, description)."""
    from oracle import qsel_oracle as o
    mesh, mask = workload_inputs(w)
    model = o.model_from_csr(w.n_s, w.n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val, mask, w.sigma)
    Q = o.precision(model, w.theta)
    diag_b = [o.block(Q, w.n_s, t, t) for t in (0, 1)]
    sub_b = [o.block(Q, w.n_s, 1, 0)]
    t0 = time.perf_counter()
    L_diag, L_sub = o.block_cholesky(diag_b, sub_b)
    t1 = time.perf_counter()
    o.block_takahashi(L_diag, L_sub)
    t2 = time.perf_counter()
    chol, tak = (t1 - t0) / 2, (t2 - t1) / 2
    parts = o.partition(w.n_t, qi.balanced_slab_start(w.n_t, w.n_parts), w.overlap)
    units = sum(p.ext[1] - p.ext[0] for p in parts)
    est = units * (chol + tak) + w.n_t * chol
    desc = (f"oracle block Cholesky + Takahashi of a 2-slab chain of {w.n_s}x{w.n_s} blocks "
            f"({t2 - t0:.1f} s), extrapolated to {units} subdomain slabs + {w.n_t} sampler slabs; "
            "excludes the correction solves (lower bound)")
    return est, t2 - t0, desc


def cpu_cores():
    return os.cpu_count() or 1


# ----------------------------------------------------------------------------
# native arm
# ----------------------------------------------------------------------------
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

    w = qi.workload(args.workload)
    mesh, mask = workload_inputs(w)
    stream = torch.cuda.current_stream()
    seed = 1000 + rank
    ctx = qsel.qsel_create(w.n_s, w.n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val, mask, w.sigma,
                           w.theta, n_parts=w.n_parts, overlap=w.overlap, n_samples=w.n_samples, seed=seed,
                           pcg_tol=w.pcg_tol, cuda_stream=stream.cuda_stream, profile_kernels=1)
    out = torch.empty(w.n, dtype=torch.float64, device=f"cuda:{local}")
    grads = np.zeros(3)

    def step():
        qsel.qsel_set_theta(ctx, w.theta)
        qsel.qsel_diag_inv(ctx, out)
        g = qsel.qsel_trace_grads(ctx)
        grads[:] = g
        return qsel.qsel_stats(ctx)

    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        stats.append(step())
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms_local = e0.elapsed_time(e1)
    t = torch.tensor([ms_local], dtype=torch.float64, device=f"cuda:{local}")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_total = float(t.item())
    ms_per_step = ms_total / args.steps

    # end to end through the public API with host buffers
    e2e_s = None
    h2d = (mesh.c_diag.nbytes + mesh.g_rowptr.nbytes + mesh.g_col.nbytes + mesh.g_val.nbytes + mask.nbytes
           + 3 * 8 + 8)
    d2h = w.n * 8 + 3 * 8
    if args.e2e_steps > 0:
        c_pin = torch.from_numpy(mesh.c_diag).pin_memory().numpy()
        gv_pin = torch.from_numpy(mesh.g_val).pin_memory().numpy()
        rp_pin = torch.from_numpy(mesh.g_rowptr).pin_memory().numpy()
        gc_pin = torch.from_numpy(mesh.g_col).pin_memory().numpy()
        mk_pin = torch.from_numpy(mask).pin_memory().numpy()
        diag_host = torch.empty(w.n, dtype=torch.float64).pin_memory().numpy()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            c2 = qsel.qsel_create(w.n_s, w.n_t, c_pin, rp_pin, gc_pin, gv_pin, mk_pin, w.sigma, w.theta,
                                  n_parts=w.n_parts, overlap=w.overlap, n_samples=w.n_samples, seed=seed,
                                  pcg_tol=w.pcg_tol, cuda_stream=stream.cuda_stream)
            qsel.qsel_diag_inv(c2, diag_host)
            qsel.qsel_trace_grads(c2)
            c2.close()
        torch.cuda.synchronize()
        el = torch.tensor([time.perf_counter() - t0], dtype=torch.float64, device=f"cuda:{local}")
        if world > 1:
            dist.all_reduce(el, op=dist.ReduceOp.MAX)
        e2e_s = float(el.item()) / (args.e2e_steps * world)

    if rank != 0:
        ctx.close()
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    # dominant kernel: the FP64 dense tile GEMM
    gemm_ms = sum(s["gemm_ms"] for s in stats)
    gemm_flop = sum(s["gemm_flop"] for s in stats)
    gemm_launches = sum(s["gemm_launches"] for s in stats)
    sweep_ms = sum(s["sweep_ms"] for s in stats)
    spmm_ms = sum(s["spmm_ms"] for s in stats)
    achieved = gemm_flop / (gemm_ms * 1e-3) / 1e12 if gemm_ms > 0 else None
    st = stats[-1]

    accuracy = None
    if not args.no_accuracy:
        ref = qsel.qsel_create(w.n_s, w.n_t, mesh.c_diag, mesh.g_rowptr, mesh.g_col, mesh.g_val, mask, w.sigma,
                               w.theta, n_parts=1, overlap=0, n_samples=1, cuda_stream=stream.cuda_stream)
        v_ex = qsel.qsel_diag_inv(ref)
        t_ex = qsel.qsel_trace_grads(ref)
        ref.close()
        v = out.cpu().numpy()
        rel = (v - v_ex) / v_ex
        accuracy = {"reference": "exact single-subdomain FP64 selected inversion on the GPU (n_p = 1)",
                    "eps_diag_rms": float(np.sqrt(np.mean(rel ** 2))),
                    "eps_diag_p99": float(np.quantile(np.abs(rel), 0.99)),
                    "eps_diag_max": float(np.max(np.abs(rel))),
                    "eps_traces": [float(abs(a - b) / abs(b)) for a, b in zip(grads, t_ex)],
                    "seeds": 1}

    cpu = None
    if not args.no_cpu_baseline:
        est, spent, desc = oracle_sample(w)
        cpu = {"value": est, "unit": "s", "cores": cpu_cores(), "kind": "oracle", "sample": desc,
               "sample_seconds": spent}

    result = {
        "metric": METRIC,
        "value": ms_per_step / 1e3 / world,
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded grid FEM mesh, Philox noise)",
        "config": {"workload": f"{w.name}: {w.m}x{w.m} grid, n_t={w.n_t}, n={w.n}, kappa={w.kappa}, "
                               f"rho={w.rho}, {int(w.obs_frac * 100)}% observed",
                   "form": "plain FP64 RBMC", "n_parts": w.n_parts, "overlap": w.overlap,
                   "n_samples": w.n_samples, "pcg_tol": w.pcg_tol,
                   "l2": "inputs larger than L2 (samples alone %.2f GB)" % (w.n * 256 * 8 / 1e9),
                   "parallelism": f"replicas x{world}"},
        "roofline": {"kernel": "k_gemm64 (FP64 dense tile GEMM of the Takahashi recursion and the sweeps)",
                     "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS if achieved else None,
                     "traffic": (GEMM64_DRAM_BYTES_PER_FLOP * gemm_flop / gemm_launches) if gemm_launches else None,
                     "traffic_unit": "bytes per launch (ncu per-FLOP traffic scaled to the average timed launch)",
                     "peak_source": "nominal FP64 rate (recipe); probe measured 1.19 TFLOP/s"},
        "phases_ms": {"rhs": st["ms_rhs"], "pcg": st["ms_pcg"], "factor": st["ms_factor"],
                      "takahashi": st["ms_takahashi"], "correction": st["ms_correction"]},
        "kernel_ms_per_step": {"gemm": gemm_ms / args.steps, "sweep_update": sweep_ms / args.steps,
                               "spmm": spmm_ms / args.steps},
        "pcg_iterations": st["pcg_iterations"],
        "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
        "gemm_launches_per_step": gemm_launches // args.steps,
        "clocks": clk,
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "cpu_baseline": cpu,
        "accuracy": accuracy,
    }
    print(json.dumps(result), flush=True)
    ctx.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ----------------------------------------------------------------------------
# reference arm: the CPU oracle
# ----------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = qi.workload(args.workload)
    for _ in range(args.warmup):
        oracle_sample(w)
    vals, spent, desc = [], 0.0, ""
    for _ in range(args.steps):
        est, sp, desc = oracle_sample(w)
        vals.append(est)
        spent += sp
    v = float(np.mean(vals))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": spent / args.steps * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded grid FEM mesh)",
        "config": {"workload": w.name, "form": "CPU FP64 oracle"},
        "cpu_baseline": {"value": v, "unit": "s", "kind": "oracle", "cores": cpu_cores(), "sample": desc},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
