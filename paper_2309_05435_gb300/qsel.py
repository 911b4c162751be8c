"""ctypes binding of the C ABI in include/qsel.h (argument marshalling only).

Every computation happens in libqsel.so.  The functions keep the C names;
``Context`` wraps an opaque ``qsel_ctx*`` and owns it.  Loading fails loudly
when the library has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_float, c_int32, c_int64, c_uint8, c_uint64, c_void_p

import numpy as np

QSEL_FP64 = 0
QSEL_MIXED = 1
QSEL_SAMPLER_PCG = 0
QSEL_SAMPLER_LANCZOS = 1
QSEL_PRECOND_BLOCK_JACOBI = 0
QSEL_PRECOND_KRON = 1
QSEL_PIVOT_DOUBLE_FLOAT = 0
QSEL_PIVOT_FP64 = 1
QSEL_MODEL_SEPARABLE = 0
QSEL_MODEL_DIFFUSION = 1
QSEL_MODEL_BLOCK_TRIDIAGONAL = 2
QSEL_CHAIN_TWO_ENDED = 0
QSEL_CHAIN_FORWARD = 1

_STATUS = {0: "QSEL_OK", 1: "QSEL_EINVAL", 2: "QSEL_ENOMEM", 3: "QSEL_ECUDA", 4: "QSEL_ENOTSPD",
           5: "QSEL_ENOCONV", 6: "QSEL_ETIMEOUT", 7: "QSEL_ESTATE"}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libqsel.so")


class qsel_model(ctypes.Structure):
    _fields_ = [("n_s", c_int32), ("n_t", c_int32), ("c_diag", POINTER(c_double)),
                ("g_rowptr", POINTER(c_int32)), ("g_col", POINTER(c_int32)), ("g_val", POINTER(c_double)),
                ("obs_mask", POINTER(c_uint8)), ("sigma", c_double)]


class qsel_theta(ctypes.Structure):
    _fields_ = [("log_kappa", c_double), ("log_tau", c_double), ("logit_rho", c_double)]


class qsel_partition(ctypes.Structure):
    _fields_ = [("n_parts", c_int32), ("slab_start", POINTER(c_int32))]


class qsel_options(ctypes.Structure):
    _fields_ = [("n_samples", c_int32), ("seed", c_uint64), ("precision", c_int32), ("pcg_tol", c_double),
                ("pcg_max_iter", c_int32), ("precond_block", c_int32), ("control_variate", c_int32),
                ("cuda_stream", c_void_p), ("profile_kernels", c_int32), ("tensor_passes", c_int32),
                ("sampler", c_int32), ("lanczos_steps", c_int32), ("preconditioner", c_int32),
                ("part_overlap", POINTER(c_int32)), ("pivot_precision", c_int32), ("model", c_int32),
                ("chain", c_int32)]


class qsel_bt_model(ctypes.Structure):
    _fields_ = [("n_s", c_int32), ("n_t", c_int32), ("rowptr", POINTER(c_int32)), ("col", POINTER(c_int32)),
                ("diag_vals", POINTER(c_double)), ("off_vals", POINTER(c_double)), ("n_theta", c_int32),
                ("ddiag_vals", POINTER(c_double)), ("doff_vals", POINTER(c_double))]


class qsel_batch_info_t(ctypes.Structure):
    _fields_ = [("n_models", c_int32), ("n_streams", c_int32), ("ms_replay", c_double), ("ms_capture", c_double),
                ("ms_autotune", c_double), ("launches_per_replay", c_int64), ("max_pcg_iterations", c_int32)]


class qsel_cv_plan_options(ctypes.Structure):
    _fields_ = [("target_rel_err", c_double), ("max_overlap", c_int32), ("min_samples", c_int32),
                ("max_samples", c_int32), ("cost_pcg", c_double), ("cost_dense", c_double),
                ("cost_corr", c_double), ("part_counts", POINTER(c_int32)), ("n_part_counts", c_int32)]


class qsel_cv_plan_t(ctypes.Structure):
    _fields_ = [("n_samples", c_int32), ("feasible", c_int32), ("predicted_cost", c_double),
                ("predicted_err", c_double), ("single_part_cost", c_double), ("part_overlap", POINTER(c_int32)),
                ("part_pred_err", POINTER(c_double)), ("n_parts", c_int32), ("slab_start", POINTER(c_int32))]


class qsel_stats_t(ctypes.Structure):
    _fields_ = [("pcg_iterations", c_int32), ("pcg_max_rel_residual", c_double), ("ms_rhs", c_double),
                ("ms_pcg", c_double), ("ms_factor", c_double), ("ms_takahashi", c_double),
                ("ms_correction", c_double), ("ms_total", c_double), ("kernel_launches", c_int64),
                ("gemm_ms", c_double), ("gemm_flop", c_double), ("gemm_launches", c_int64),
                ("sweep_ms", c_double), ("sweep_flop", c_double), ("sweep_launches", c_int64),
                ("spmm_ms", c_double), ("spmm_bytes", c_double), ("spmm_launches", c_int64),
                ("class_ms", c_double * 11), ("class_launches", c_int64 * 11), ("class_work", c_double * 11)]


PROF_CLASSES = ("gemm", "sweep_update", "spmm", "pivot", "sweep_panel", "schur", "gather", "precond", "pcg_vec",
                "correction", "extract")


def _fields(s) -> dict:
    out = {}
    for name, _ in type(s)._fields_:
        v = getattr(s, name)
        out[name] = list(v) if hasattr(v, "_length_") else v
    return out


EXPORTED = ["qsel_create", "qsel_create_bt", "qsel_set_bt_values", "qsel_set_seed", "qsel_set_theta",
            "qsel_diag_inv", "qsel_trace_grads", "qsel_trace_grads_n", "qsel_stats",
            "qsel_set_data", "qsel_posterior_mean", "qsel_loglik_grad", "qsel_set_covariates",
            "qsel_fixed_effects",
            "qsel_debug_set_samples", "qsel_debug_get_samples", "qsel_debug_get_rhs",
            "qsel_debug_get_selinv_diag", "qsel_debug_get_lanczos", "qsel_debug_apply_precond",
            "qsel_spd_inverse_noalloc", "qsel_debug_tc_wait", "qsel_debug_sweep_schedule",
            "qsel_error_estimate",
            "qsel_cv_create", "qsel_cv_set_params", "qsel_cv_get_params", "qsel_cv_predict", "qsel_cv_grad",
            "qsel_cv_train", "qsel_cv_features", "qsel_cv_targets", "qsel_cv_plan",
            "qsel_cv_destroy", "qsel_create_batch", "qsel_batch_run", "qsel_batch_set_theta",
            "qsel_batch_diag_inv", "qsel_batch_trace_grads", "qsel_batch_stats", "qsel_batch_info",
            "qsel_batch_tuning", "qsel_batch_last_error", "qsel_batch_destroy", "qsel_last_error", "qsel_destroy"]
QSEL_NOALLOC_MAX_N = 1024
QSEL_CV_FEATURES = 14
QSEL_CV_PARAMS = 5185
QSEL_CV_PARAMS_ALL = 5213

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libqsel.so (raises if it is missing; nothing runs without it)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2309_05435_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P = POINTER
    lib.qsel_create.argtypes = [P(c_void_p), P(qsel_model), P(qsel_theta), P(qsel_partition), c_int32,
                                P(qsel_options)]
    lib.qsel_set_theta.argtypes = [c_void_p, P(qsel_theta)]
    lib.qsel_set_seed.argtypes = [c_void_p, c_uint64]
    lib.qsel_diag_inv.argtypes = [c_void_p, c_void_p, c_int32]
    lib.qsel_trace_grads.argtypes = [c_void_p, P(c_double)]
    lib.qsel_trace_grads_n.argtypes = [c_void_p, P(c_double), c_int32]
    lib.qsel_create_bt.argtypes = [P(c_void_p), P(qsel_bt_model), P(qsel_partition), c_int32, P(qsel_options)]
    lib.qsel_set_bt_values.argtypes = [c_void_p, P(c_double), P(c_double), P(c_double), P(c_double)]
    lib.qsel_set_data.argtypes = [c_void_p, P(c_double)]
    lib.qsel_posterior_mean.argtypes = [c_void_p, c_void_p, c_int32]
    lib.qsel_loglik_grad.argtypes = [c_void_p, P(c_double), P(c_double)]
    lib.qsel_set_covariates.argtypes = [c_void_p, c_int32, P(c_double), c_double]
    lib.qsel_fixed_effects.argtypes = [c_void_p, P(c_double), P(c_double), P(c_double), c_int32]
    lib.qsel_stats.argtypes = [c_void_p, P(qsel_stats_t)]
    lib.qsel_debug_set_samples.argtypes = [c_void_p, P(c_double), c_int32]
    lib.qsel_debug_get_samples.argtypes = [c_void_p, P(c_double), c_int32]
    lib.qsel_debug_get_rhs.argtypes = [c_void_p, P(c_double), c_int32]
    lib.qsel_debug_get_selinv_diag.argtypes = [c_void_p, P(c_double)]
    lib.qsel_debug_get_lanczos.argtypes = [c_void_p, P(c_double), P(c_double), c_int32]
    lib.qsel_debug_apply_precond.argtypes = [c_void_p, P(c_double), P(c_double), c_int32]
    lib.qsel_spd_inverse_noalloc.argtypes = [c_void_p, c_int32, c_int32, c_void_p]
    lib.qsel_debug_tc_wait.argtypes = [c_int32, c_int64]
    lib.qsel_debug_sweep_schedule.argtypes = [c_int32, c_int32, c_int32, c_int32]
    lib.qsel_error_estimate.argtypes = [c_void_p, P(c_double), P(c_double)]
    lib.qsel_cv_create.argtypes = [P(c_void_p), c_uint64, c_void_p]
    lib.qsel_cv_set_params.argtypes = [c_void_p, P(c_float)]
    lib.qsel_cv_get_params.argtypes = [c_void_p, P(c_float)]
    lib.qsel_cv_predict.argtypes = [c_void_p, c_void_p, c_void_p, c_int32]
    lib.qsel_cv_grad.argtypes = [c_void_p, c_void_p, c_void_p, c_int32, P(c_float), P(c_float)]
    lib.qsel_cv_train.argtypes = [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_float, c_int32, P(c_float)]
    lib.qsel_cv_features.argtypes = [c_void_p, c_int32, c_void_p]
    lib.qsel_cv_targets.argtypes = [P(c_void_p), c_int32, c_void_p]
    lib.qsel_cv_plan.argtypes = [c_void_p, c_void_p, P(qsel_cv_plan_options), P(qsel_cv_plan_t)]
    lib.qsel_cv_destroy.argtypes = [c_void_p]
    lib.qsel_cv_destroy.restype = None
    lib.qsel_create_batch.argtypes = [P(c_void_p), c_int32, P(qsel_model), P(qsel_theta), P(qsel_partition),
                                      P(c_int32), P(qsel_options), c_int32, c_int32]
    lib.qsel_batch_run.argtypes = [c_void_p]
    lib.qsel_batch_set_theta.argtypes = [c_void_p, c_int32, P(qsel_theta)]
    lib.qsel_batch_diag_inv.argtypes = [c_void_p, c_int32, c_void_p, c_int32]
    lib.qsel_batch_trace_grads.argtypes = [c_void_p, c_int32, P(c_double)]
    lib.qsel_batch_stats.argtypes = [c_void_p, c_int32, P(qsel_stats_t)]
    lib.qsel_batch_info.argtypes = [c_void_p, P(qsel_batch_info_t)]
    lib.qsel_batch_tuning.argtypes = [c_void_p, c_int32, P(c_int32), P(c_int32), P(c_int32)]
    lib.qsel_batch_last_error.argtypes = [c_void_p]
    lib.qsel_batch_last_error.restype = c_char_p
    lib.qsel_batch_destroy.argtypes = [c_void_p]
    lib.qsel_batch_destroy.restype = None
    lib.qsel_last_error.argtypes = [c_void_p]
    lib.qsel_last_error.restype = c_char_p
    lib.qsel_destroy.argtypes = [c_void_p]
    lib.qsel_destroy.restype = None
    for name in EXPORTED:
        if name not in ("qsel_cv_destroy", "qsel_last_error", "qsel_destroy", "qsel_batch_last_error",
                        "qsel_batch_destroy"):
            getattr(lib, name).restype = c_int32
    _lib = lib
    return lib


class QselError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(POINTER(ctype))


def _check(status: int, handle):
    if status != 0:
        msg = load_library().qsel_last_error(handle)
        raise QselError(status, msg.decode() if msg else "")


class Context:
    """Owner of one qsel_ctx*."""

    def __init__(self, handle, n: int, k: int, n_parts: int = 1):
        self.handle = handle
        self.n = n
        self.k = k
        self.n_parts = n_parts

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "handle", None):
            load_library().qsel_destroy(self.handle)
            self.handle = None

    # convenience methods with the same meaning as the free functions
    def diag_inv(self, out=None):
        return qsel_diag_inv(self, out)

    def trace_grads(self):
        return qsel_trace_grads(self)

    def stats(self):
        return qsel_stats(self)


def qsel_create(n_s, n_t, c_diag, g_rowptr, g_col, g_val, obs_mask, sigma, theta, n_parts=1,
                slab_start=None, overlap=0, n_samples=64, seed=0, precision=QSEL_FP64, pcg_tol=1e-10,
                pcg_max_iter=20000, precond_block=0, control_variate=0, cuda_stream=None,
                profile_kernels=0, tensor_passes=0, part_overlap=None, sampler=QSEL_SAMPLER_PCG,
                lanczos_steps=0, preconditioner=QSEL_PRECOND_BLOCK_JACOBI,
                pivot_precision=QSEL_PIVOT_DOUBLE_FLOAT, model=QSEL_MODEL_SEPARABLE,
                chain=QSEL_CHAIN_TWO_ENDED) -> Context:
    """Create a context from host arrays (copied by the library).  With
    model=QSEL_MODEL_DIFFUSION, theta = (log gamma_s, log gamma_t, log gamma_e)."""
    lib = load_library()
    c = np.ascontiguousarray(c_diag, dtype=np.float64)
    rp = np.ascontiguousarray(g_rowptr, dtype=np.int32)
    gc = np.ascontiguousarray(g_col, dtype=np.int32)
    gv = np.ascontiguousarray(g_val, dtype=np.float64)
    mk = np.ascontiguousarray(obs_mask, dtype=np.uint8)
    model_s = qsel_model(int(n_s), int(n_t), _ptr(c, c_double), _ptr(rp, c_int32), _ptr(gc, c_int32),
                         _ptr(gv, c_double), _ptr(mk, c_uint8), float(sigma))
    th = qsel_theta(*[float(x) for x in theta])
    ss = None
    if slab_start is not None:
        ss = np.ascontiguousarray(slab_start, dtype=np.int32)
    part = qsel_partition(int(n_parts), _ptr(ss, c_int32) if ss is not None else None)
    po = None
    if part_overlap is not None:
        po = np.ascontiguousarray(part_overlap, dtype=np.int32)
        if po.size != int(n_parts):
            raise ValueError("part_overlap needs one entry per part")
    opt = qsel_options(int(n_samples), int(seed), int(precision), float(pcg_tol), int(pcg_max_iter),
                       int(precond_block), int(control_variate),
                       c_void_p(int(cuda_stream)) if cuda_stream else None, int(profile_kernels),
                       int(tensor_passes), int(sampler), int(lanczos_steps), int(preconditioner),
                       _ptr(po, c_int32) if po is not None else None, int(pivot_precision), int(model),
                       int(chain))
    h = c_void_p()
    st = lib.qsel_create(ctypes.byref(h), ctypes.byref(model_s), ctypes.byref(th), ctypes.byref(part),
                         int(overlap), ctypes.byref(opt))
    _check(st, None)
    return Context(h, int(n_s) * int(n_t), int(n_samples), int(n_parts))


def qsel_create_bt(n_s, n_t, rowptr, col, diag_vals, off_vals, ddiag_vals=None, doff_vals=None, n_parts=1,
                   slab_start=None, overlap=0, n_samples=64, seed=0, precision=QSEL_FP64, pcg_tol=1e-10,
                   cuda_stream=None, sampler=QSEL_SAMPLER_LANCZOS, lanczos_steps=64, precond_block=0,
                   profile_kernels=0, tensor_passes=0, part_overlap=None,
                   pivot_precision=QSEL_PIVOT_DOUBLE_FLOAT, chain=QSEL_CHAIN_TWO_ENDED) -> Context:
    """Context for a user-given block-tridiagonal precision: the pattern in
    CSR (rowptr, col), diag_vals (n_t x nnz), off_vals ((n_t - 1) x nnz),
    and optional derivatives ddiag_vals (n_theta x n_t x nnz), doff_vals
    (n_theta x (n_t - 1) x nnz)."""
    lib = load_library()
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    dv = np.ascontiguousarray(diag_vals, dtype=np.float64)
    ov = np.ascontiguousarray(off_vals, dtype=np.float64)
    n_theta = 0 if ddiag_vals is None else int(np.asarray(ddiag_vals).shape[0])
    ddv = None if ddiag_vals is None else np.ascontiguousarray(ddiag_vals, dtype=np.float64)
    dov = None if doff_vals is None else np.ascontiguousarray(doff_vals, dtype=np.float64)
    m = qsel_bt_model(int(n_s), int(n_t), _ptr(rp, c_int32), _ptr(cl, c_int32), _ptr(dv, c_double),
                      _ptr(ov, c_double), n_theta, _ptr(ddv, c_double) if ddv is not None else None,
                      _ptr(dov, c_double) if dov is not None else None)
    ss = None if slab_start is None else np.ascontiguousarray(slab_start, dtype=np.int32)
    part = qsel_partition(int(n_parts), _ptr(ss, c_int32) if ss is not None else None)
    po = None if part_overlap is None else np.ascontiguousarray(part_overlap, dtype=np.int32)
    opt = qsel_options(int(n_samples), int(seed), int(precision), float(pcg_tol), 20000, int(precond_block), 0,
                       c_void_p(int(cuda_stream)) if cuda_stream else None, int(profile_kernels),
                       int(tensor_passes), int(sampler), int(lanczos_steps), QSEL_PRECOND_BLOCK_JACOBI,
                       _ptr(po, c_int32) if po is not None else None, int(pivot_precision),
                       QSEL_MODEL_BLOCK_TRIDIAGONAL, int(chain))
    h = c_void_p()
    _check(lib.qsel_create_bt(ctypes.byref(h), ctypes.byref(m), ctypes.byref(part), int(overlap),
                              ctypes.byref(opt)), None)
    ctx = Context(h, int(n_s) * int(n_t), int(n_samples), int(n_parts))
    ctx.n_theta = n_theta
    return ctx


def qsel_set_bt_values(ctx: Context, diag_vals, off_vals, ddiag_vals=None, doff_vals=None):
    """New block values on the pattern of a qsel_create_bt context."""
    dv = np.ascontiguousarray(diag_vals, dtype=np.float64)
    ov = np.ascontiguousarray(off_vals, dtype=np.float64)
    ddv = None if ddiag_vals is None else np.ascontiguousarray(ddiag_vals, dtype=np.float64)
    dov = None if doff_vals is None else np.ascontiguousarray(doff_vals, dtype=np.float64)
    _check(load_library().qsel_set_bt_values(ctx.handle, _ptr(dv, c_double), _ptr(ov, c_double),
                                             _ptr(ddv, c_double) if ddv is not None else None,
                                             _ptr(dov, c_double) if dov is not None else None), ctx.handle)


def qsel_trace_grads_n(ctx: Context, n: int) -> np.ndarray:
    """The n trace gradients of the context's hyperparameters."""
    out = np.zeros(max(1, int(n)), dtype=np.float64)
    _check(load_library().qsel_trace_grads_n(ctx.handle, _ptr(out, c_double), int(n)), ctx.handle)
    return out[:int(n)]


def qsel_set_data(ctx: Context, y_obs):
    """Data on the observed nodes, in increasing node order (n_obs values)."""
    y = np.ascontiguousarray(y_obs, dtype=np.float64)
    _check(load_library().qsel_set_data(ctx.handle, _ptr(y, c_double)), ctx.handle)


def qsel_posterior_mean(ctx: Context, out=None):
    """mu = Q^-1 A^T y / sigma^2 (numpy array, or into a device tensor `out`)."""
    lib = load_library()
    if out is not None:
        _check(lib.qsel_posterior_mean(ctx.handle, c_void_p(out.data_ptr()), 1), ctx.handle)
        return out
    mu = np.empty(ctx.n, dtype=np.float64)
    _check(lib.qsel_posterior_mean(ctx.handle, _ptr(mu, c_double), 0), ctx.handle)
    return mu


def qsel_set_covariates(ctx: Context, Z, beta_prec):
    """Fixed effects: Z (n_obs x n_beta, rows in the order of the data),
    beta ~ N(0, I / beta_prec); an empty Z removes them."""
    Zc = np.ascontiguousarray(Z, dtype=np.float64)
    nb = 0 if Zc.size == 0 else int(Zc.shape[1])
    _check(load_library().qsel_set_covariates(ctx.handle, nb, _ptr(Zc, c_double) if nb else None,
                                              float(beta_prec)), ctx.handle)


def qsel_fixed_effects(ctx: Context, n_beta: int):
    """(mu_beta, Var(beta), diag(W S^-1 W^T)) as numpy arrays."""
    mu = np.empty(n_beta)
    var = np.empty((n_beta, n_beta))
    corr = np.empty(ctx.n)
    _check(load_library().qsel_fixed_effects(ctx.handle, _ptr(mu, c_double), _ptr(var, c_double),
                                             _ptr(corr, c_double), 0), ctx.handle)
    return mu, var, corr


def qsel_loglik_grad(ctx: Context, with_terms=False):
    """Gradient of log p(y | theta); with_terms also returns (prior log-det
    derivatives, traces, quadratic forms), each of length 3."""
    g = np.zeros(3)
    t = np.zeros(9)
    _check(load_library().qsel_loglik_grad(ctx.handle, _ptr(g, c_double), _ptr(t, c_double)), ctx.handle)
    if with_terms:
        return g, (t[0:3].copy(), t[3:6].copy(), t[6:9].copy())
    return g


def qsel_set_seed(ctx: Context, seed: int):
    """New Philox key: the next run draws new samples."""
    _check(load_library().qsel_set_seed(ctx.handle, int(seed)), ctx.handle)


def qsel_set_theta(ctx: Context, theta):
    th = qsel_theta(*[float(x) for x in theta])
    _check(load_library().qsel_set_theta(ctx.handle, ctypes.byref(th)), ctx.handle)


def qsel_diag_inv(ctx: Context, out=None):
    """Estimate of diag(Q^-1).  ``out``: None (returns a new numpy array), a
    float64 numpy array (host), or a CUDA tensor / object with data_ptr()
    (device, written in place)."""
    lib = load_library()
    if out is None:
        out = np.empty(ctx.n, dtype=np.float64)
    if isinstance(out, np.ndarray):
        if out.dtype != np.float64 or out.size != ctx.n or not out.flags.c_contiguous:
            raise ValueError("out must be a contiguous float64 array of n entries")
        _check(lib.qsel_diag_inv(ctx.handle, out.ctypes.data_as(c_void_p), 0), ctx.handle)
    else:
        _check(lib.qsel_diag_inv(ctx.handle, c_void_p(out.data_ptr()), 1), ctx.handle)
    return out


def qsel_trace_grads(ctx: Context) -> np.ndarray:
    g = np.zeros(3, dtype=np.float64)
    _check(load_library().qsel_trace_grads(ctx.handle, _ptr(g, c_double)), ctx.handle)
    return g


def qsel_stats(ctx: Context) -> dict:
    s = qsel_stats_t()
    _check(load_library().qsel_stats(ctx.handle, ctypes.byref(s)), ctx.handle)
    return _fields(s)


def qsel_debug_set_samples(ctx: Context, X: np.ndarray):
    X = np.ascontiguousarray(X, dtype=np.float64)
    if X.shape != (ctx.n, ctx.k):
        raise ValueError(f"X must be {(ctx.n, ctx.k)}")
    _check(load_library().qsel_debug_set_samples(ctx.handle, _ptr(X, c_double), ctx.k), ctx.handle)


def qsel_debug_get_samples(ctx: Context) -> np.ndarray:
    X = np.empty((ctx.n, ctx.k), dtype=np.float64)
    _check(load_library().qsel_debug_get_samples(ctx.handle, _ptr(X, c_double), ctx.k), ctx.handle)
    return X


def qsel_debug_get_rhs(ctx: Context) -> np.ndarray:
    R = np.empty((ctx.n, ctx.k), dtype=np.float64)
    _check(load_library().qsel_debug_get_rhs(ctx.handle, _ptr(R, c_double), ctx.k), ctx.handle)
    return R


def qsel_debug_get_selinv_diag(ctx: Context) -> np.ndarray:
    d = np.empty(ctx.n, dtype=np.float64)
    _check(load_library().qsel_debug_get_selinv_diag(ctx.handle, _ptr(d, c_double)), ctx.handle)
    return d


def qsel_debug_get_lanczos(ctx: Context, steps: int):
    """(alpha, beta), each (steps, n_samples): the Lanczos coefficients of
    every column of the last run."""
    a = np.empty((steps, ctx.k), dtype=np.float64)
    b = np.empty((steps, ctx.k), dtype=np.float64)
    _check(load_library().qsel_debug_get_lanczos(ctx.handle, _ptr(a, c_double), _ptr(b, c_double), ctx.k),
           ctx.handle)
    return a, b


def qsel_debug_apply_precond(ctx: Context, R: np.ndarray) -> np.ndarray:
    """Z = M^-1 R with the context's PCG preconditioner (FP64 contexts)."""
    R = np.ascontiguousarray(R, dtype=np.float64)
    if R.shape != (ctx.n, ctx.k):
        raise ValueError(f"R must be {(ctx.n, ctx.k)}")
    Z = np.empty_like(R)
    _check(load_library().qsel_debug_apply_precond(ctx.handle, _ptr(R, c_double), _ptr(Z, c_double), ctx.k),
           ctx.handle)
    return Z


def qsel_spd_inverse_noalloc(a, n: int, lda: int | None = None, cuda_stream=None):
    """Invert the SPD matrix at device address ``a`` (a CUDA tensor or an
    integer pointer; n x n row-major, leading dimension lda) in place, without
    any allocation by the library; see qsel.h for the scratch-memory rules."""
    ptr = a.data_ptr() if hasattr(a, "data_ptr") else int(a)
    st = load_library().qsel_spd_inverse_noalloc(c_void_p(ptr), int(n), int(lda if lda is not None else n),
                                                  c_void_p(int(cuda_stream)) if cuda_stream else None)
    _check(st, None)


def qsel_debug_sweep_schedule(serial: bool, update_ctas: int = 0, update_stages: int = 0,
                              shared_pivot: bool = False):
    """Scheduling hook of the mixed sweep: serial runs each panel's update after
    the pivot chain on one stream; update_ctas > 0 caps the persistent update
    kernel's CTAs; update_stages (2 or 3) sets its shared-memory ring;
    shared_pivot lets the pivot CTAs share SMs with the update.
    qsel_debug_sweep_schedule(False) restores the default."""
    _check(load_library().qsel_debug_sweep_schedule(1 if serial else 0, int(update_ctas), int(update_stages),
                                                    1 if shared_pivot else 0), None)


def qsel_debug_tc_wait(skip_loads: bool, wait_cycles: int = 0):
    """Test hook of the tensor-core GEMM's bounded waits (see qsel.h);
    qsel_debug_tc_wait(False, 0) restores normal operation."""
    _check(load_library().qsel_debug_tc_wait(1 if skip_loads else 0, int(wait_cycles)), None)


def qsel_error_estimate(ctx: Context):
    """(per-part RMS relative standard error, global one) of the last
    diag(Q^-1) estimate, from the sample moments of w^2."""
    part = np.zeros(ctx.n_parts, dtype=np.float64)
    g = c_double(0.0)
    _check(load_library().qsel_error_estimate(ctx.handle, _ptr(part, c_double), ctypes.byref(g)), ctx.handle)
    return part, g.value


def _dev(a):
    """Device address of a CUDA tensor (or an integer pointer)."""
    return c_void_p(a.data_ptr() if hasattr(a, "data_ptr") else int(a))


class ControlVariate:
    """Owner of one qsel_cv* (the control-variate network)."""

    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "handle", None):
            load_library().qsel_cv_destroy(self.handle)
            self.handle = None


def qsel_cv_create(seed: int = 0, cuda_stream=None) -> ControlVariate:
    h = c_void_p()
    _check(load_library().qsel_cv_create(ctypes.byref(h), int(seed),
                                         c_void_p(int(cuda_stream)) if cuda_stream else None), None)
    return ControlVariate(h)


def qsel_cv_set_params(cv: ControlVariate, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.size != QSEL_CV_PARAMS_ALL:
        raise ValueError(f"params must hold {QSEL_CV_PARAMS_ALL} values")
    _check(load_library().qsel_cv_set_params(cv.handle, _ptr(p, c_float)), None)


def qsel_cv_get_params(cv: ControlVariate) -> np.ndarray:
    p = np.empty(QSEL_CV_PARAMS_ALL, dtype=np.float32)
    _check(load_library().qsel_cv_get_params(cv.handle, _ptr(p, c_float)), None)
    return p


def qsel_cv_predict(cv: ControlVariate, X_dev, y_dev, n: int):
    _check(load_library().qsel_cv_predict(cv.handle, _dev(X_dev), _dev(y_dev), int(n)), None)


def qsel_cv_grad(cv: ControlVariate, X_dev, y_dev, n: int):
    g = np.empty(QSEL_CV_PARAMS, dtype=np.float32)
    loss = c_float(0.0)
    _check(load_library().qsel_cv_grad(cv.handle, _dev(X_dev), _dev(y_dev), int(n), _ptr(g, c_float),
                                       ctypes.byref(loss)), None)
    return g, loss.value


def qsel_cv_train(cv: ControlVariate, X_dev, y_dev, n: int, steps: int, lr: float, set_input_stats: bool = False):
    loss = c_float(0.0)
    _check(load_library().qsel_cv_train(cv.handle, _dev(X_dev), _dev(y_dev), int(n), int(steps), float(lr),
                                        int(bool(set_input_stats)), ctypes.byref(loss)), None)
    return loss.value


def qsel_cv_features(ctx: Context, overlap: int, F_dev):
    _check(load_library().qsel_cv_features(ctx.handle, int(overlap), _dev(F_dev)), ctx.handle)


def qsel_cv_targets(ctxs, y_dev):
    arr = (c_void_p * len(ctxs))(*[c.handle.value if isinstance(c.handle, c_void_p) else c.handle for c in ctxs])
    _check(load_library().qsel_cv_targets(arr, len(ctxs), _dev(y_dev)), ctxs[0].handle)


def qsel_cv_plan(ctx: Context, cv: ControlVariate, target_rel_err: float, max_overlap: int = 4,
                 min_samples: int = 32, max_samples: int = 512, cost_pcg: float = 0.0, cost_dense: float = 0.0,
                 cost_corr: float = 0.0, part_counts=None) -> dict:
    """Plan (k, per-part overlaps) for the context's partition, or, with
    part_counts, also choose among balanced partitions (1 = exact one part)."""
    pc = None if not part_counts else np.ascontiguousarray(part_counts, dtype=np.int32)
    o = qsel_cv_plan_options(float(target_rel_err), int(max_overlap), int(min_samples), int(max_samples),
                             float(cost_pcg), float(cost_dense), float(cost_corr),
                             _ptr(pc, c_int32) if pc is not None else None, 0 if pc is None else len(pc))
    room = max(ctx.n_parts, int(pc.max()) if pc is not None else 0)
    po = np.zeros(room, dtype=np.int32)
    pe = np.zeros(room, dtype=np.float64)
    ss = np.zeros(room + 1, dtype=np.int32)
    plan = qsel_cv_plan_t(0, 0, 0.0, 0.0, 0.0, _ptr(po, c_int32), _ptr(pe, c_double), 0, _ptr(ss, c_int32))
    _check(load_library().qsel_cv_plan(ctx.handle, cv.handle, ctypes.byref(o), ctypes.byref(plan)), ctx.handle)
    npart = plan.n_parts
    return {"n_samples": plan.n_samples, "feasible": bool(plan.feasible), "predicted_cost": plan.predicted_cost,
            "predicted_err": plan.predicted_err, "single_part_cost": plan.single_part_cost,
            "n_parts": npart, "slab_start": ss[:npart + 1].copy(),
            "part_overlap": po[:npart].copy(), "part_pred_err": pe[:npart].copy()}


class Batch:
    """Owner of one qsel_batch* (independent models under one captured graph)."""

    def __init__(self, handle, sizes):
        self.handle = handle
        self.sizes = sizes          # n of every model

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "handle", None):
            load_library().qsel_batch_destroy(self.handle)
            self.handle = None


def _check_batch(status: int, b):
    if status != 0:
        msg = load_library().qsel_batch_last_error(b.handle if b is not None else None)
        raise QselError(status, msg.decode() if msg else "")


def qsel_create_batch(models, thetas, partitions, overlaps, n_samples=128, seed=0, precision=QSEL_MIXED,
                      pcg_tol=1e-8, pcg_max_iter=20000, precond_block=0, tensor_passes=0, cuda_stream=None,
                      n_streams=16, autotune=False) -> Batch:
    """models: list of dicts with n_s, n_t, c_diag, g_rowptr, g_col, g_val,
    obs_mask, sigma (host arrays); partitions: list of (n_parts, slab_start or
    None); overlaps: list of ints."""
    lib = load_library()
    n = len(models)
    keep = []
    M = (qsel_model * n)()
    for i, m in enumerate(models):
        arrs = [np.ascontiguousarray(m["c_diag"], dtype=np.float64), np.ascontiguousarray(m["g_rowptr"], np.int32),
                np.ascontiguousarray(m["g_col"], np.int32), np.ascontiguousarray(m["g_val"], np.float64),
                np.ascontiguousarray(m["obs_mask"], np.uint8)]
        keep += arrs
        M[i] = qsel_model(int(m["n_s"]), int(m["n_t"]), _ptr(arrs[0], c_double), _ptr(arrs[1], c_int32),
                          _ptr(arrs[2], c_int32), _ptr(arrs[3], c_double), _ptr(arrs[4], c_uint8),
                          float(m["sigma"]))
    TH = (qsel_theta * n)(*[qsel_theta(*[float(x) for x in th]) for th in thetas])
    PA = (qsel_partition * n)()
    for i, (n_parts, ss) in enumerate(partitions):
        if ss is not None:
            a = np.ascontiguousarray(ss, dtype=np.int32)
            keep.append(a)
            PA[i] = qsel_partition(int(n_parts), _ptr(a, c_int32))
        else:
            PA[i] = qsel_partition(int(n_parts), None)
    OV = np.ascontiguousarray(overlaps, dtype=np.int32)
    opt = qsel_options(int(n_samples), int(seed), int(precision), float(pcg_tol), int(pcg_max_iter),
                       int(precond_block), 0, c_void_p(int(cuda_stream)) if cuda_stream else None, 0,
                       int(tensor_passes), QSEL_SAMPLER_PCG, 0, QSEL_PRECOND_BLOCK_JACOBI, None,
                       QSEL_PIVOT_DOUBLE_FLOAT)
    h = c_void_p()
    st = lib.qsel_create_batch(ctypes.byref(h), n, M, TH, PA, _ptr(OV, c_int32), ctypes.byref(opt),
                               int(n_streams), int(bool(autotune)))
    _check_batch(st, None)
    return Batch(h, [int(m["n_s"]) * int(m["n_t"]) for m in models])


def qsel_batch_run(b: Batch):
    _check_batch(load_library().qsel_batch_run(b.handle), b)


def qsel_batch_set_theta(b: Batch, model: int, theta):
    th = qsel_theta(*[float(x) for x in theta])
    _check_batch(load_library().qsel_batch_set_theta(b.handle, int(model), ctypes.byref(th)), b)


def qsel_batch_diag_inv(b: Batch, model: int, out=None):
    lib = load_library()
    if out is None:
        out = np.empty(b.sizes[model], dtype=np.float64)
    if isinstance(out, np.ndarray):
        _check_batch(lib.qsel_batch_diag_inv(b.handle, int(model), out.ctypes.data_as(c_void_p), 0), b)
    else:
        _check_batch(lib.qsel_batch_diag_inv(b.handle, int(model), c_void_p(out.data_ptr()), 1), b)
    return out


def qsel_batch_trace_grads(b: Batch, model: int) -> np.ndarray:
    g = np.zeros(3, dtype=np.float64)
    _check_batch(load_library().qsel_batch_trace_grads(b.handle, int(model), _ptr(g, c_double)), b)
    return g


def qsel_batch_stats(b: Batch, model: int) -> dict:
    s = qsel_stats_t()
    _check_batch(load_library().qsel_batch_stats(b.handle, int(model), ctypes.byref(s)), b)
    return _fields(s)


def qsel_batch_info(b: Batch) -> dict:
    s = qsel_batch_info_t()
    _check_batch(load_library().qsel_batch_info(b.handle, ctypes.byref(s)), b)
    return {name: getattr(s, name) for name, _ in qsel_batch_info_t._fields_}


def qsel_batch_tuning(b: Batch, model: int) -> dict:
    pb, tp, st = c_int32(0), c_int32(0), c_int32(0)
    _check_batch(load_library().qsel_batch_tuning(b.handle, int(model), ctypes.byref(pb), ctypes.byref(tp),
                                                  ctypes.byref(st)), b)
    return {"precond_block": pb.value, "tensor_passes": tp.value, "stream": st.value}


def qsel_last_error(ctx: Context | None) -> str:
    msg = load_library().qsel_last_error(ctx.handle if ctx is not None else None)
    return msg.decode() if msg else ""


def qsel_destroy(ctx: Context):
    ctx.close()
