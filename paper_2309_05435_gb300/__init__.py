"""GB300-native overlapping RBMC selected inversion (diag(Q^-1) and log-det
gradients of space-time SPDE precisions).  The compute path is the CUDA
library libqsel.so (C ABI in include/qsel.h); ``qsel`` is its thin binding."""
from . import qsel  # noqa: F401
from .qsel import (QSEL_FP64, QSEL_MIXED, Batch, Context, ControlVariate, QselError, load_library,  # noqa: F401
                   qsel_batch_diag_inv, qsel_batch_info, qsel_batch_run, qsel_batch_set_theta, qsel_batch_stats,
                   qsel_batch_trace_grads, qsel_batch_tuning, qsel_create, qsel_create_batch, qsel_cv_create, qsel_cv_features, qsel_cv_get_params,
                   qsel_cv_grad, qsel_cv_plan, qsel_cv_predict, qsel_cv_set_params, qsel_cv_targets, qsel_cv_train,
                   qsel_error_estimate, qsel_debug_get_rhs, qsel_debug_get_samples,
                   qsel_debug_get_selinv_diag, qsel_debug_set_samples, qsel_destroy,
                   qsel_diag_inv, qsel_fixed_effects, qsel_last_error, qsel_loglik_grad, qsel_posterior_mean,
                   qsel_set_covariates, qsel_set_data, qsel_set_seed, qsel_set_theta, qsel_spd_inverse_noalloc,
                   qsel_stats,
                   qsel_trace_grads)
