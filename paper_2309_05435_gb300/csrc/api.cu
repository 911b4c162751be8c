// C ABI (include/qsel.h) and the host orchestration of the pipeline:
// perturbation samples -> multi-RHS PCG -> per-subdomain block factorisation
// and Takahashi selected inversion -> RB correction -> diag and traces.
#include <algorithm>
#include <chrono>
#include <type_traits>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "qsel.h"
#include "kernels.cuh"

namespace qsel {

Err cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
  Err err;
  err.code = QSEL_ECUDA;
  char buf[512];
  snprintf(buf, sizeof buf, "CUDA error %s (%s) in %s at %s:%d", cudaGetErrorName(e),
           cudaGetErrorString(e), what, file, line);
  err.msg = buf;
  return err;
}

static Err ok() { return Err{}; }
static Err fail(int code, const std::string &msg) {
  Err e;
  e.code = code;
  e.msg = msg;
  return e;
}

// One subdomain of the time partition (Algorithm 3 on whole slabs).
struct Subdomain {
  int s0, s1, e0, e1, T, lo, hi;
  int sep_left, sep_right;             // separator slabs or -1
  double *partial = nullptr;           // corr_grid x 3 trace partials
  int slot_base = 0;                   // first pattern-sum slot (2 T slots)
  // Two-ended factorisation of the one-part form: the reversed half numbers
  // its slabs from e1 - 1 down to e0 (its last local slab, e0, is the middle
  // slab that the forward half factors), and factors nfac = T - 1 of them.
  int rev = 0;
  int nfac = 0;
  int g(int tl) const { return rev ? e1 - 1 - tl : e0 + tl; }         // global slab of local tl
  int cpl(int tl) const { return rev ? e1 - 2 - tl : e0 + tl; }       // coupling block of tl, tl + 1
};

// Dense working set of one subdomain in flight; the wave holds up to
// kMaxBatch of them and is reused for the next wave.  Element type: double
// (FP64 path) or float (mixed path).
struct DenseSlot {
  std::vector<void *> Dinv;            // T_max pivot-block inverses
  void *SigA = nullptr, *SigB = nullptr, *Y = nullptr, *W = nullptr, *V = nullptr;
  void *P = nullptr, *U = nullptr, *Vs = nullptr, *Vk = nullptr;  // sweep scratch
  void *U2 = nullptr, *V2 = nullptr, *Wp = nullptr, *Wp2 = nullptr;  // tensor-core sweep panels
  void *Sp[4] = {nullptr, nullptr, nullptr, nullptr};  // the panel update's operands split into TF32 hi / lo
  void *Gs[4] = {nullptr, nullptr, nullptr, nullptr};  // Takahashi operands split into TF32 hi / lo (2 matrices)
  void *wbuf = nullptr;                // T_max x n_pad x ld correction samples
  void *tra = nullptr, *trb = nullptr; // ld x n_pad transposes (tensor-core correction products)
  void *ybuf = nullptr, *tmp = nullptr, *bright = nullptr;
};

}  // namespace qsel

using namespace qsel;

struct qsel_ctx {
  int n_s = 0, n_t = 0, n = 0, ld = 0, k = 0, n_pad = 0, n_l = 0, bsize = 64;
  bool mixed = false;
  int tc_passes = 0;                  // mixed path: 3 or 1 = tcgen05 TF32 GEMMs, 0 = CUDA-core FP32
  double sigma = 1.0, obs_w = 1.0;
  qsel_theta theta{};
  qsel_options opt{};
  cudaStream_t stream = nullptr;
  std::vector<int> slab_start;
  // spatial pattern
  SellPattern pat{};
  int n_ent = 0;
  double *d_c_pat = nullptr, *d_g_pat = nullptr, *d_h_pat = nullptr, *d_isqc_pat = nullptr;
  double *d_h3_pat = nullptr;          // H C^-1 G (diffusion model)
  double *d_qs = nullptr, *d_dqs = nullptr, *d_kc = nullptr;
  uint8_t *d_obs = nullptr;
  // posterior mean and hyperparameter gradient (qsel_set_data and after)
  double *d_cdiag = nullptr;           // lumped mass diagonal
  double *d_y = nullptr;               // data on the observed nodes
  double *d_mu = nullptr;              // posterior mean, n
  double *d_hyp = nullptr;             // quadratic forms (3), gradient (3), terms (9)
  double *d_K = nullptr, *d_Kp = nullptr, *d_Ku = nullptr, *d_Kv = nullptr;   // dense K, sweep scratch
  bool have_data = false;
  // fixed effects (qsel_set_covariates): Z (n_obs x n_beta), the observed
  // nodes in order, and S, m, S^-1, mu_beta, C, Schur traces (3), diag corr (n)
  int n_beta = 0;
  double beta_prec = 1.0;
  double *d_Z = nullptr, *d_fe = nullptr, *d_fecorr = nullptr;
  int32_t *d_obs_nodes = nullptr;
  double *fe_S() { return d_fe; }
  double *fe_m() { return d_fe + 64 * 64; }
  double *fe_Sinv() { return d_fe + 64 * 64 + 64; }
  double *fe_mu() { return d_fe + 2 * 64 * 64 + 64; }
  double *fe_C() { return d_fe + 2 * 64 * 64 + 128; }
  double *fe_trace() { return d_fe + 3 * 64 * 64 + 128; }
  int32_t *d_obs_index = nullptr;
  int n_obs = 0;
  TimeCoeffs tc{};
  // The precision and dQ/dtheta_j as the kernels read them (block values on
  // the pattern with per-block scales), set by set_model_views: the
  // separable model points at Q_s, dQ_s and the time coefficients; the
  // diffusion model and user-given matrices at per-block arrays.
  int model_kind = 0;                  // QSEL_MODEL_*
  BtModel mod{};
  DerivModels dmod{};
  // per-block arrays of the diffusion model and of user-given matrices:
  // A_t (n_t x n_ent), B_t ((n_t - 1) x n_ent), then per theta_j dA_j, dB_j
  double *d_blk = nullptr;
  double *d_blk_coef = nullptr;        // per-block scales of the diffusion model
  std::vector<int64_t> bt_slot;        // user-given matrix: SELL slot of every CSR entry
  std::vector<int64_t> bt_mirror;      // and the CSR position of its transpose entry
  // sampler: FP64 right-hand sides and samples; FP64 PCG vectors (FP64 path)
  // or FP32 PCG vectors plus FP64 residual buffers (mixed path)
  double *d_z1 = nullptr, *d_z2 = nullptr, *d_R = nullptr, *d_X = nullptr;
  double *d_r = nullptr, *d_zv = nullptr, *d_p = nullptr, *d_q = nullptr;
  float *f_x = nullptr, *f_r = nullptr, *f_z = nullptr, *f_p = nullptr, *f_q = nullptr;
  double *d_pa = nullptr, *d_pb = nullptr;
  void *d_pblk = nullptr;
  double *d_scal = nullptr;           // alpha, beta, rho, bb, rr (ld each) + max_rel
  int32_t *d_active = nullptr, *d_counters = nullptr;
  // estimator
  std::vector<Subdomain> parts;
  // one-part form factored from both ends: forward half (slabs 0..m) and
  // reversed half (slabs n_t-1..m+1, then the middle m), run as one wave
  bool twist = false;
  Subdomain half[2];
  std::vector<DenseSlot> slots;
  int wave = 1, T_max = 1;
  int slot_cap = kMaxBatch;            // at most this many subdomains in flight
  double *d_diag = nullptr, *d_selinv = nullptr, *d_corr = nullptr, *d_traces = nullptr, *d_sums = nullptr;
  double *d_corr4 = nullptr;           // (1/k) sum w^4 per node (error estimate)
  std::vector<int> part_nl;            // overlap of every part
  int32_t *d_slab_start = nullptr;     // n_parts + 1 slab offsets
  double *d_part_sums = nullptr;       // n_parts doubles of per-part reductions
  float *d_bnd = nullptr, *d_sepd = nullptr;  // feature distances: n_s nodes, n_t slabs
  float *d_cv_F = nullptr, *d_cv_y = nullptr; // planner scratch, allocated on first use
  double *d_cv_sums = nullptr;         // planner: per-slab sums (n_t)
  int32_t *d_cv_slabs = nullptr;       // planner: slab offsets 0 .. n_t
  // theta in device memory (read by the model kernel) and its pinned host copy
  double *d_theta = nullptr, *h_theta = nullptr;
  // graph mode: the pipeline is captured into a CUDA graph with device-driven
  // loops (conditional while nodes); no host synchronisation inside
  bool graph_mode = false;
  cudaStream_t body_stream[2] = {nullptr, nullptr};  // capture streams of loop bodies
  int32_t *d_loop = nullptr;           // loop state (see launch_loop_init)
  double *d_tol2 = nullptr;            // inner tolerance of the refinement, squared
  // Kronecker preconditioner (grid meshes)
  bool kron = false;
  int kron_m = 0;
  double *d_kV = nullptr, *d_klam = nullptr, *d_kdh = nullptr, *d_kU = nullptr, *d_kmu = nullptr;
  void *d_ktab = nullptr;              // the operator's tables in the sampler's element type
  double kron_rho = -2.0;              // rho of the temporal eigenpairs on the device
  bool kron_tc = true;                 // Kronecker apply on the tensor cores (mixed form)
  KronOperator kop{};
  // Lanczos sampler (allocated on first use)
  struct {
    double *vec[3] = {nullptr, nullptr, nullptr};   // v_{j-1}, v_j, w (rotated)
    double *u = nullptr, *q = nullptr, *xt = nullptr, *linv = nullptr;
    double *alpha = nullptr, *beta = nullptr, *coef = nullptr, *eta = nullptr, *zero = nullptr;
    double *partial = nullptr, *dwork = nullptr, *U = nullptr;
    bool ready = false, ran = false;
  } lz;
  double *d_partials = nullptr, *d_diag_scratch = nullptr;
  TraceSlab *d_slabs = nullptr;
  int n_trace_slabs = 0;
  int32_t *d_err = nullptr;
  // host staging
  int32_t *h_counters = nullptr;
  double *h_small = nullptr;
  cudaEvent_t ev[4]{};
  SweepStreams sweep_ss;               // look-ahead of the tensor-core sweep (mixed path)
  cudaStream_t pcg_stream = nullptr;   // the PCG sampler, beside the first wave's dense part
  cudaEvent_t ev_fork = nullptr, ev_samples = nullptr;
  std::vector<cudaEvent_t> phase_ev;   // pairs per (wave, phase)
  size_t phase_used = 0;
  Profiler prof;
  bool computed = false, injected = false, have_rhs = false;
  qsel_stats_t stats{};
  std::string last_error;
  std::vector<void *> allocs;

  Err alloc_bytes(void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(QSEL_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    allocs.push_back(*p);
    return ok();
  }
  template <typename T>
  Err alloc(T **p, size_t count) {
    return alloc_bytes(reinterpret_cast<void **>(p), count * sizeof(T));
  }
  cudaEvent_t phase_event() {
    if (phase_used == phase_ev.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      phase_ev.push_back(e);
    }
    return phase_ev[phase_used++];
  }
  ~qsel_ctx() {
    for (void *p : allocs) cudaFree(p);
    if (h_counters) cudaFreeHost(h_counters);
    if (h_small) cudaFreeHost(h_small);
    if (h_theta) cudaFreeHost(h_theta);
    for (auto &e : ev)
      if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : {sweep_ss.fork, sweep_ss.panel, sweep_ss.lookahead, sweep_ss.scatter})
      if (e) cudaEventDestroy(e);
    if (sweep_ss.hi) cudaStreamDestroy(sweep_ss.hi);
    if (sweep_ss.lo) cudaStreamDestroy(sweep_ss.lo);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_samples) cudaEventDestroy(ev_samples);
    if (pcg_stream) cudaStreamDestroy(pcg_stream);
    for (auto e : phase_ev) cudaEventDestroy(e);
  }
};

static thread_local std::string g_create_error;

namespace qsel {
void set_context_free_error(const std::string &msg) { g_create_error = msg; }
}  // namespace qsel

static qsel_status finish(qsel_ctx *ctx, const Err &e) {
  if (e.code != 0 && ctx) ctx->last_error = e.msg;
  return (qsel_status)e.code;
}

#define TRY(expr)                         \
  do {                                    \
    Err _err = (expr);                    \
    if (_err.code != 0) return _err;      \
  } while (0)

// ---------------------------------------------------------------------------
// Creation: validation, spatial pattern (union of C, G and G C^-1 G), SELL-32,
// partition (Algorithm 3 on whole slabs) and device allocation.
// ---------------------------------------------------------------------------
// Eigenpairs of a symmetric tridiagonal matrix (diagonal d, off-diagonal e,
// e[i] coupling i and i + 1) by the implicit QL algorithm with Wilkinson
// shifts; Z (row-major n x n) holds the eigenvectors as columns.
static bool host_tridiag_eig(int n, std::vector<double> d, std::vector<double> e, std::vector<double> &evals,
                             std::vector<double> &Z) {
  e.resize(n, 0.0);
  e[n - 1] = 0.0;
  Z.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Z[(size_t)i * n + i] = 1.0;
  for (int l = 0; l < n; ++l) {
    int iter = 0;
    for (;;) {
      int mm = l;
      for (; mm < n - 1; ++mm) {
        const double dd = std::fabs(d[mm]) + std::fabs(d[mm + 1]);
        if (std::fabs(e[mm]) <= 2.3e-16 * dd) break;
      }
      if (mm == l) break;
      if (++iter > 60) return false;
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = std::hypot(g, 1.0);
      g = d[mm] - d[l] + e[l] / (g + std::copysign(r, g));
      double sn = 1.0, cs = 1.0, p = 0.0;
      bool early = false;
      for (int i = mm - 1; i >= l; --i) {
        const double f = sn * e[i], b = cs * e[i];
        r = std::hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {
          d[i + 1] -= p;
          e[mm] = 0.0;
          early = true;
          break;
        }
        sn = f / r;
        cs = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * sn + 2.0 * cs * b;
        p = sn * r;
        d[i + 1] = g + p;
        g = cs * r - b;
        for (int k = 0; k < n; ++k) {
          const double z1 = Z[(size_t)k * n + i + 1], z0 = Z[(size_t)k * n + i];
          Z[(size_t)k * n + i + 1] = sn * z0 + cs * z1;
          Z[(size_t)k * n + i] = cs * z0 - sn * z1;
        }
      }
      if (early) continue;
      d[l] -= p;
      e[l] = g;
      e[mm] = 0.0;
    }
  }
  evals = d;
  return true;
}

// The mesh is the unit m x m grid of this library's FEM convention when
// G = T (x) D + D (x) T (1-D Neumann stiffness T, D = diag(1/2, 1, .., 1, 1/2),
// node index i m + j) and the lumped mass equals D (x) D away from the
// corners.  Returns m, or 0 for other meshes.
static int detect_grid(const qsel_model *m) {
  const int n_s = m->n_s;
  const int g = (int)std::lround(std::sqrt((double)n_s));
  if (g < 2 || g * g != n_s) return 0;
  auto D = [&](int i) { return (i == 0 || i == g - 1) ? 0.5 : 1.0; };
  auto T = [&](int i, int j) {
    if (i == j) return (i == 0 || i == g - 1) ? 1.0 : 2.0;
    return (std::abs(i - j) == 1) ? -1.0 : 0.0;
  };
  for (int r = 0; r < n_s; ++r) {
    const int i = r / g, j = r % g;
    const bool corner = (i == 0 || i == g - 1) && (j == 0 || j == g - 1);
    if (!corner && std::fabs(m->c_diag[r] - D(i) * D(j)) > 1e-12) return 0;
    std::map<int, double> want;
    for (int di = -1; di <= 1; ++di)
      for (int dj = -1; dj <= 1; ++dj) {
        const int i2 = i + di, j2 = j + dj;
        if (i2 < 0 || i2 >= g || j2 < 0 || j2 >= g) continue;
        const double v = T(i, i2) * (j == j2 ? D(j) : 0.0) + (i == i2 ? D(i) : 0.0) * T(j, j2);
        if (v != 0.0) want[i2 * g + j2] = v;
      }
    std::map<int, double> have;
    for (int p = m->g_rowptr[r]; p < m->g_rowptr[r + 1]; ++p) have[m->g_col[p]] += m->g_val[p];
    for (auto &kv : have)
      if (std::fabs(kv.second) > 1e-14 && !want.count(kv.first)) return 0;
    for (auto &kv : want) {
      auto it = have.find(kv.first);
      if (it == have.end() || std::fabs(it->second - kv.second) > 1e-12) return 0;
    }
  }
  return g;
}

static Err validate_options(int n_t, const qsel_partition *part, int32_t overlap, const qsel_options *opt);

static Err validate(const qsel_model *m, const qsel_theta *th, const qsel_partition *part,
                    int32_t overlap, const qsel_options *opt) {
  if (!m || !th || !opt) return fail(QSEL_EINVAL, "model, theta and options must not be NULL");
  if (m->n_s < 1 || m->n_t < 1) return fail(QSEL_EINVAL, "n_s and n_t must be >= 1");
  if ((int64_t)m->n_s * m->n_t > (int64_t)1 << 30) return fail(QSEL_EINVAL, "n_s * n_t too large");
  if (!m->c_diag || !m->g_rowptr || !m->g_col || !m->g_val || !m->obs_mask)
    return fail(QSEL_EINVAL, "model arrays must not be NULL");
  if (!(m->sigma > 0.0) || !std::isfinite(m->sigma)) return fail(QSEL_EINVAL, "sigma must be > 0");
  for (int i = 0; i < m->n_s; ++i)
    if (!(m->c_diag[i] > 0.0) || !std::isfinite(m->c_diag[i]))
      return fail(QSEL_EINVAL, "c_diag must be finite and > 0");
  if (m->g_rowptr[0] != 0) return fail(QSEL_EINVAL, "g_rowptr[0] must be 0");
  for (int i = 0; i < m->n_s; ++i) {
    if (m->g_rowptr[i + 1] < m->g_rowptr[i]) return fail(QSEL_EINVAL, "g_rowptr must be non-decreasing");
    for (int p = m->g_rowptr[i]; p < m->g_rowptr[i + 1]; ++p) {
      if (m->g_col[p] < 0 || m->g_col[p] >= m->n_s) return fail(QSEL_EINVAL, "g_col out of range");
      if (!std::isfinite(m->g_val[p])) return fail(QSEL_EINVAL, "g_val must be finite");
    }
  }
  if (!std::isfinite(th->log_kappa) || !std::isfinite(th->log_tau) || !std::isfinite(th->logit_rho))
    return fail(QSEL_EINVAL, "theta must be finite");
  if (std::fabs(th->logit_rho) > 36.0) return fail(QSEL_EINVAL, "rho too close to 0 or 1");
  if (opt->model != QSEL_MODEL_SEPARABLE && opt->model != QSEL_MODEL_DIFFUSION)
    return fail(QSEL_EINVAL, "model must be QSEL_MODEL_SEPARABLE or QSEL_MODEL_DIFFUSION");
  if (opt->model == QSEL_MODEL_DIFFUSION && opt->sampler != QSEL_SAMPLER_LANCZOS)
    return fail(QSEL_EINVAL, "the diffusion model has no factored form: it needs sampler = QSEL_SAMPLER_LANCZOS");
  if (opt->model == QSEL_MODEL_DIFFUSION && opt->preconditioner != QSEL_PRECOND_BLOCK_JACOBI)
    return fail(QSEL_EINVAL, "the diffusion model takes the block-Jacobi preconditioner");
  TRY(validate_options(m->n_t, part, overlap, opt));
  if (opt->preconditioner == QSEL_PRECOND_KRON && detect_grid(m) == 0)
    return fail(QSEL_EINVAL, "QSEL_PRECOND_KRON needs the m x m grid mesh (stiffness T (x) D + D (x) T, lumped mass "
                             "D (x) D away from the corners)");
  return ok();
}

// Partition and option checks shared by every model.
static Err validate_options(int n_t, const qsel_partition *part, int32_t overlap, const qsel_options *opt) {
  if (overlap < 0) return fail(QSEL_EINVAL, "overlap must be >= 0");
  const int np = part ? part->n_parts : 1;
  if (np < 1 || np > n_t) return fail(QSEL_EINVAL, "n_parts must be in [1, n_t]");
  if (part && part->slab_start) {
    if (part->slab_start[0] != 0 || part->slab_start[np] != n_t)
      return fail(QSEL_EINVAL, "slab_start must run from 0 to n_t");
    for (int p = 0; p < np; ++p)
      if (part->slab_start[p + 1] <= part->slab_start[p])
        return fail(QSEL_EINVAL, "slab_start must be strictly increasing");
  }
  if (opt->part_overlap)
    for (int p = 0; p < np; ++p)
      if (opt->part_overlap[p] < 0) return fail(QSEL_EINVAL, "part_overlap entries must be >= 0");
  if (opt->n_samples < 1 || opt->n_samples > 512) return fail(QSEL_EINVAL, "n_samples must be in [1, 512]");
  if (opt->precision != QSEL_FP64 && opt->precision != QSEL_MIXED)
    return fail(QSEL_EINVAL, "precision must be QSEL_FP64 or QSEL_MIXED");
  if (!(opt->pcg_tol > 0.0) || opt->pcg_max_iter < 1) return fail(QSEL_EINVAL, "pcg_tol > 0 and pcg_max_iter >= 1 required");
  if (opt->precond_block != 0 && opt->precond_block != 1 && opt->precond_block != 16 &&
      opt->precond_block != 32 && opt->precond_block != 64)
    return fail(QSEL_EINVAL, "precond_block must be 0, 1, 16, 32 or 64");
  if (opt->control_variate != 0) return fail(QSEL_EINVAL, "control_variate must be 0");
  if (opt->tensor_passes != 0 && opt->tensor_passes != 1 && opt->tensor_passes != 3 && opt->tensor_passes != -1)
    return fail(QSEL_EINVAL, "tensor_passes must be 0, 1, 3 or -1");
  if (opt->pivot_precision != QSEL_PIVOT_DOUBLE_FLOAT && opt->pivot_precision != QSEL_PIVOT_FP64)
    return fail(QSEL_EINVAL, "pivot_precision must be QSEL_PIVOT_DOUBLE_FLOAT or QSEL_PIVOT_FP64");
  if (opt->preconditioner != QSEL_PRECOND_BLOCK_JACOBI && opt->preconditioner != QSEL_PRECOND_KRON)
    return fail(QSEL_EINVAL, "preconditioner must be QSEL_PRECOND_BLOCK_JACOBI or QSEL_PRECOND_KRON");
  if (opt->chain != QSEL_CHAIN_TWO_ENDED && opt->chain != QSEL_CHAIN_FORWARD)
    return fail(QSEL_EINVAL, "chain must be QSEL_CHAIN_TWO_ENDED or QSEL_CHAIN_FORWARD");
  if (opt->sampler != QSEL_SAMPLER_PCG && opt->sampler != QSEL_SAMPLER_LANCZOS)
    return fail(QSEL_EINVAL, "sampler must be QSEL_SAMPLER_PCG or QSEL_SAMPLER_LANCZOS");
  if (opt->sampler == QSEL_SAMPLER_LANCZOS) {
    if (opt->lanczos_steps < 1 || opt->lanczos_steps > 1024)
      return fail(QSEL_EINVAL, "lanczos_steps must be in [1, 1024]");
    if (opt->precond_block != 0 && opt->precond_block != 16 && opt->precond_block != 32 && opt->precond_block != 64)
      return fail(QSEL_EINVAL, "the Lanczos sampler's block preconditioner takes blocks of 16, 32 or 64 rows");
  }
  return ok();
}

template <typename T>
static Err upload(qsel_ctx *c, T **dst, const std::vector<T> &src) {
  TRY(c->alloc(dst, src.size()));
  if (!src.empty()) QSEL_CUDA_TRY(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return ok();
}

static Err kron_setup(qsel_ctx *c, const qsel_model *m) {
  const int g = detect_grid(m);   // checked in validate
  // scaled 1-D stiffness D^-1/2 T D^-1/2: diagonal 2, off-diagonal -1 / sqrt(D_i D_i+1)
  std::vector<double> d(g, 2.0), e(g, 0.0), dh(g), lam, V;
  for (int i = 0; i < g; ++i) dh[i] = (i == 0 || i == g - 1) ? std::sqrt(2.0) : 1.0;
  for (int i = 0; i + 1 < g; ++i) e[i] = -dh[i] * dh[i + 1];
  if (!host_tridiag_eig(g, d, e, lam, V)) return fail(QSEL_EINVAL, "grid eigendecomposition did not converge");
  TRY(upload(c, &c->d_kV, V));
  TRY(upload(c, &c->d_klam, lam));
  TRY(upload(c, &c->d_kdh, dh));
  TRY(c->alloc(&c->d_kU, (size_t)c->n_t * c->n_t));
  TRY(c->alloc(&c->d_kmu, (size_t)c->n_t));
  {
    // V, V^T, U, U^T, dh dh^T, spec (KronOperator), then for the mixed
    // form's tensor-core passes V, V^T, U, U^T as TF32 hi and lo; each
    // segment 256-byte aligned
    const size_t esz = c->mixed ? sizeof(float) : sizeof(double);
    const size_t gg = (size_t)g * g, tt = (size_t)c->n_t * c->n_t;
    const size_t seg[14] = {gg, gg, tt, tt, gg, (size_t)c->n_t * g * g, gg, gg, gg, gg, tt, tt, tt, tt};
    const int nseg = c->mixed ? 14 : 6;
    size_t off[14], total = 0;
    for (int i = 0; i < nseg; ++i) {
      off[i] = total;
      total += (seg[i] * esz + 255) / 256 * 256;
    }
    TRY(c->alloc_bytes(&c->d_ktab, total));
    char *b = static_cast<char *>(c->d_ktab);
    void **dst[6] = {&c->kop.tV, &c->kop.tVT, &c->kop.tU, &c->kop.tUT, &c->kop.dhdh, &c->kop.spec};
    for (int i = 0; i < 6; ++i) *dst[i] = b + off[i];
    for (int q = 0; q < 4; ++q)
      for (int h = 0; h < 2; ++h)
        c->kop.split[q][h] = c->mixed ? reinterpret_cast<float *>(b + off[6 + 2 * q + h]) : nullptr;
  }
  c->kron = true;
  c->kron_m = g;
  return ok();
}

// Temporal eigenpairs of Q_t (recomputed when rho changes) and the scalars of
// the current theta.
static Err kron_prepare(qsel_ctx *c) {
  const double rho = 1.0 / (1.0 + std::exp(-c->theta.logit_rho));
  const int n_t = c->n_t;
  if (rho != c->kron_rho) {
    const double om = 1.0 - rho * rho;
    std::vector<double> d(n_t), e(n_t, 0.0), mu, U;
    for (int t = 0; t < n_t; ++t) {
      const double R = (n_t == 1) ? om : ((t == 0 || t == n_t - 1) ? 1.0 : 1.0 + rho * rho);
      d[t] = R / om;
      if (t + 1 < n_t) e[t] = -rho / om;
    }
    if (!host_tridiag_eig(n_t, d, e, mu, U)) return fail(QSEL_EINVAL, "temporal eigendecomposition did not converge");
    // stream-ordered uploads (the tables below read them on the same stream;
    // a plain cudaMemcpy would go through the legacy default stream, which
    // the sampler's non-blocking stream does not wait for)
    QSEL_CUDA_TRY(cudaMemcpyAsync(c->d_kU, U.data(), U.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    QSEL_CUDA_TRY(cudaMemcpyAsync(c->d_kmu, mu.data(), mu.size() * sizeof(double), cudaMemcpyHostToDevice,
                                  c->stream));
    QSEL_CUDA_TRY(cudaStreamSynchronize(c->stream));   // the host vectors go out of scope
    c->kron_rho = rho;
  }
  KronOperator &k = c->kop;
  k.m = c->kron_m;
  k.n_t = n_t;
  k.ld = c->ld;
  k.V = c->d_kV;
  k.U = c->d_kU;
  k.dh = c->d_kdh;
  k.lam = c->d_klam;
  k.mu = c->d_kmu;
  k.kappa2 = std::exp(2.0 * c->theta.log_kappa);
  k.tau = std::exp(c->theta.log_tau);
  k.omega = (double)c->n_obs / (double)c->n * c->obs_w;
  // the passes on the tensor cores in the mixed form with 3xTF32 products
  k.use_tc = (c->kron_tc && c->mixed && c->tc_passes == 3 && kron_tc_supported(k.m, c->ld) &&
              kron_tc_supported(n_t, c->ld))
                 ? 1
                 : 0;
  k.err = c->d_err;
  if (c->mixed)
    launch_kron_tables<float>(c->stream, k);
  else
    launch_kron_tables<double>(c->stream, k);
  QSEL_CUDA_TRY(cudaGetLastError());
  return ok();
}

static void set_separable_views(qsel_ctx *c);
static void set_diffusion_views(qsel_ctx *c);

// Rows of the spatial pattern: column -> up to four theta-free values (for
// the mesh models C, G, H = G C^-1 G and H3 = H C^-1 G).
using PatRows = std::vector<std::map<int, std::array<double, 4>>>;

struct RestInputs {
  const uint8_t *obs_mask = nullptr;       // n entries, or null: no observation term
  const double *c_diag = nullptr;          // n_s lumped mass (mesh models), or null
  std::vector<std::vector<int>> adj;       // spatial neighbours (boundary distance feature)
};
static Err build_rest(qsel_ctx *c, const RestInputs &in, const qsel_partition *part, int32_t overlap);
static Err build_pattern(qsel_ctx *c, const PatRows &rows, int n_arrays, std::vector<std::vector<double>> &sell);

static Err build(qsel_ctx *c, const qsel_model *m, const qsel_partition *part, int32_t overlap) {
  const int n_s = m->n_s;
  const bool diffusion = c->model_kind == QSEL_MODEL_DIFFUSION;
  // spatial pattern rows: col -> (C, G, H = G C^-1 G, H3 = H C^-1 G)
  PatRows rows(n_s);
  auto touch = [&](int i, int j) -> double * {
    auto &r = rows[i];
    auto it = r.find(j);
    if (it == r.end()) it = r.emplace(j, std::array<double, 4>{0.0, 0.0, 0.0, 0.0}).first;
    return it->second.data();
  };
  for (int i = 0; i < n_s; ++i) {
    touch(i, i)[0] = m->c_diag[i];
    for (int p = m->g_rowptr[i]; p < m->g_rowptr[i + 1]; ++p) {
      const int j = m->g_col[p];
      touch(i, j)[1] += m->g_val[p];
      const double gij = m->g_val[p] / m->c_diag[j];
      for (int q = m->g_rowptr[j]; q < m->g_rowptr[j + 1]; ++q) touch(i, m->g_col[q])[2] += gij * m->g_val[q];
    }
  }
  if (diffusion) {
    for (int i = 0; i < n_s; ++i) {
      std::vector<std::pair<int, double>> h;
      for (auto &kv : rows[i])
        if (kv.second[2] != 0.0) h.emplace_back(kv.first, kv.second[2]);
      for (auto &hj : h) {
        const int j = hj.first;
        const double hc = hj.second / m->c_diag[j];
        for (int q = m->g_rowptr[j]; q < m->g_rowptr[j + 1]; ++q) touch(i, m->g_col[q])[3] += hc * m->g_val[q];
      }
    }
  }
  std::vector<std::vector<double>> sell;
  TRY(build_pattern(c, rows, 4, sell));
  const int n_ent = c->n_ent;
  std::vector<double> isq(n_ent, 0.0);
  {
    std::vector<int32_t> col(n_ent);
    QSEL_CUDA_TRY(cudaMemcpy(col.data(), c->pat.col, n_ent * sizeof(int32_t), cudaMemcpyDeviceToHost));
    for (int e = 0; e < n_ent; ++e) isq[e] = 1.0 / std::sqrt(m->c_diag[col[e]]);
  }
  TRY(upload(c, &c->d_c_pat, sell[0]));
  TRY(upload(c, &c->d_g_pat, sell[1]));
  TRY(upload(c, &c->d_h_pat, sell[2]));
  if (diffusion) TRY(upload(c, &c->d_h3_pat, sell[3]));
  TRY(upload(c, &c->d_isqc_pat, isq));
  TRY(c->alloc(&c->d_qs, n_ent));
  TRY(c->alloc(&c->d_dqs, n_ent));
  TRY(c->alloc(&c->d_kc, n_ent));
  if (c->opt.preconditioner == QSEL_PRECOND_KRON) TRY(kron_setup(c, m));
  RestInputs in;
  in.obs_mask = m->obs_mask;
  in.c_diag = m->c_diag;
  in.adj.resize(n_s);
  for (int i = 0; i < n_s; ++i)
    for (int p = m->g_rowptr[i]; p < m->g_rowptr[i + 1]; ++p) in.adj[i].push_back(m->g_col[p]);
  return build_rest(c, in, part, overlap);
}

// SELL-32 layout of the rows' pattern (columns in increasing order within a
// row) and the first n_arrays value arrays in that layout; sets c->pat and
// c->n_ent.
static Err build_pattern(qsel_ctx *c, const PatRows &rows, int n_arrays, std::vector<std::vector<double>> &sell) {
  const int n_s = (int)rows.size();
  const int n_slices = (n_s + kSlice - 1) / kSlice;
  std::vector<int32_t> slice_ptr(n_slices + 1, 0), slice_width(n_slices, 0);
  int max_w = 0;
  for (int s = 0; s < n_slices; ++s) {
    int w = 0;
    for (int l = 0; l < kSlice; ++l) {
      const int i = s * kSlice + l;
      if (i < n_s) w = std::max(w, (int)rows[i].size());
    }
    slice_width[s] = w;
    slice_ptr[s + 1] = slice_ptr[s] + w * kSlice;
    max_w = std::max(max_w, w);
  }
  const int n_ent = slice_ptr[n_slices];
  std::vector<int32_t> col(n_ent, 0);
  sell.assign(n_arrays, std::vector<double>(n_ent, 0.0));
  for (int s = 0; s < n_slices; ++s) {
    for (int l = 0; l < kSlice; ++l) {
      const int i = s * kSlice + l;
      int slot = 0;
      if (i < n_s) {
        for (auto &kv : rows[i]) {
          const int e = slice_ptr[s] + slot * kSlice + l;
          col[e] = kv.first;
          for (int a = 0; a < n_arrays; ++a) sell[a][e] = kv.second[a];
          ++slot;
        }
      }
      for (; slot < slice_width[s]; ++slot) col[slice_ptr[s] + slot * kSlice + l] = (i < n_s) ? i : 0;
    }
  }
  int32_t *d_sp, *d_sw, *d_col;
  TRY(upload(c, &d_sp, slice_ptr));
  TRY(upload(c, &d_sw, slice_width));
  TRY(upload(c, &d_col, col));
  if (max_w > kMaxPatternWidth)
    return fail(QSEL_EINVAL, "the pattern of Q_s has a row with " + std::to_string(max_w) +
                                 " entries; at most " + std::to_string(kMaxPatternWidth) + " are supported");
  c->pat.n_rows = n_s;
  c->pat.n_slices = n_slices;
  c->pat.max_width = max_w;
  if (!configure_pattern_kernels(c->pat)) return fail(QSEL_ECUDA, "shared-memory opt-in of the gather kernels failed");
  c->pat.slice_ptr = d_sp;
  c->pat.slice_width = d_sw;
  c->pat.col = d_col;
  c->n_ent = n_ent;
  return ok();
}

// Everything after the spatial pattern: observations, time coefficients and
// the model views, partition, sampler buffers, subdomains, dense working sets.
static Err build_rest(qsel_ctx *c, const RestInputs &in, const qsel_partition *part, int32_t overlap) {
  const int n_s = c->n_s;
  const int n = c->n;
  {
    std::vector<uint8_t> mask(n, 0);
    std::vector<int32_t> oidx(n, -1);
    int n_obs = 0;
    for (int r = 0; r < n; ++r) {
      mask[r] = (in.obs_mask && in.obs_mask[r]) ? 1 : 0;
      if (mask[r]) oidx[r] = n_obs++;
    }
    c->n_obs = n_obs;
    TRY(upload(c, &c->d_obs, mask));
    TRY(upload(c, &c->d_obs_index, oidx));
    if (in.c_diag) TRY(upload(c, &c->d_cdiag, std::vector<double>(in.c_diag, in.c_diag + n_s)));
  }

  // time coefficients
  double *tcb;
  TRY(c->alloc(&tcb, (size_t)5 * c->n_t + 8));
  c->tc.a0 = tcb;
  c->tc.a1 = tcb + c->n_t;
  c->tc.r0 = tcb + 2 * c->n_t;
  c->tc.r1 = tcb + 3 * c->n_t;
  c->tc.bdiag = tcb + 4 * c->n_t;
  c->tc.scalars = tcb + 5 * c->n_t;
  QSEL_CUDA_TRY(cudaMemset(tcb, 0, ((size_t)5 * c->n_t + 8) * sizeof(double)));
  if (c->model_kind == QSEL_MODEL_SEPARABLE) {
    set_separable_views(c);
  } else if (c->model_kind == QSEL_MODEL_DIFFUSION) {
    TRY(c->alloc(&c->d_blk, (size_t)(4 * c->n_t + 2) * c->n_ent));
    TRY(c->alloc(&c->d_blk_coef, (size_t)3 * c->n_t));
    set_diffusion_views(c);
  }

  // partition
  const int np = part ? part->n_parts : 1;
  c->slab_start.resize(np + 1);
  if (part && part->slab_start) {
    for (int p = 0; p <= np; ++p) c->slab_start[p] = part->slab_start[p];
  } else {
    const int base = c->n_t / np, extra = c->n_t % np;
    c->slab_start[0] = 0;
    for (int p = 0; p < np; ++p) c->slab_start[p + 1] = c->slab_start[p] + base + (p < extra ? 1 : 0);
  }
  c->part_nl.assign(np, overlap);
  if (c->opt.part_overlap)
    for (int p = 0; p < np; ++p) c->part_nl[p] = c->opt.part_overlap[p];
  c->opt.part_overlap = nullptr;   // the caller's array is not kept
  c->n_l = *std::min_element(c->part_nl.begin(), c->part_nl.end());
  {
    std::vector<int32_t> ss(c->slab_start.begin(), c->slab_start.end());
    TRY(upload(c, &c->d_slab_start, ss));
  }
  TRY(c->alloc(&c->d_part_sums, (size_t)np));

  // graph distance of every spatial node to the mesh boundary (nodes with
  // fewer stiffness neighbours than the maximum), capped at 8: an input of
  // the control-variate features
  {
    std::vector<int> deg(n_s, 0), dist(n_s, -1), queue;
    for (int i = 0; i < n_s; ++i)
      for (int j : in.adj[i]) deg[i] += (j != i);
    const int dmax = *std::max_element(deg.begin(), deg.end());
    for (int i = 0; i < n_s; ++i)
      if (deg[i] < dmax) {
        dist[i] = 0;
        queue.push_back(i);
      }
    for (size_t h = 0; h < queue.size(); ++h) {
      const int i = queue[h];
      for (int j : in.adj[i]) {
        if (dist[j] < 0) {
          dist[j] = dist[i] + 1;
          queue.push_back(j);
        }
      }
    }
    std::vector<float> bnd(n_s);
    for (int i = 0; i < n_s; ++i) bnd[i] = queue.empty() ? 0.f : (float)std::min(std::max(dist[i], 0), 8);
    TRY(upload(c, &c->d_bnd, bnd));
    TRY(c->alloc(&c->d_sepd, (size_t)c->n_t));
  }

  // sampler buffers
  const size_t vec = (size_t)n * c->ld;
  TRY(c->alloc(&c->d_z1, vec));
  TRY(c->alloc(&c->d_z2, (size_t)std::max(c->n_obs, 1) * c->ld));
  TRY(c->alloc(&c->d_R, vec));
  TRY(c->alloc(&c->d_X, vec));
  if (c->mixed) {
    TRY(c->alloc(&c->d_q, vec));           // Q X for the refinement residual
    TRY(c->alloc(&c->f_x, vec));
    TRY(c->alloc(&c->f_r, vec));
    TRY(c->alloc(&c->f_z, vec));
    TRY(c->alloc(&c->f_p, vec));
    TRY(c->alloc(&c->f_q, vec));
  } else {
    TRY(c->alloc(&c->d_r, vec));
    TRY(c->alloc(&c->d_zv, vec));
    TRY(c->alloc(&c->d_p, vec));
    TRY(c->alloc(&c->d_q, vec));
  }
  const int n_tiles = (n + 63) / 64;
  const int n_pa = std::max(std::max(n_tiles, bt_spmm_grid(n)), residual_grid(n));
  TRY(c->alloc(&c->d_pa, (size_t)n_pa * c->ld));
  TRY(c->alloc(&c->d_pb, (size_t)n_pa * c->ld));
  const int nblk = (n + c->bsize - 1) / c->bsize;
  const size_t esz = c->mixed ? sizeof(float) : sizeof(double);
  TRY(c->alloc_bytes(&c->d_pblk, (size_t)nblk * c->bsize * c->bsize * esz));
  TRY(c->alloc(&c->d_scal, (size_t)5 * c->ld + 8));
  TRY(c->alloc(&c->d_active, (size_t)c->ld));
  TRY(c->alloc(&c->d_counters, 8));
  QSEL_CUDA_TRY(cudaMemset(c->d_X, 0, vec * sizeof(double)));

  // subdomains and trace bookkeeping: 2 pattern-sum slots per (subdomain,
  // local slab) for Sigma and 2 for Y
  const int n_pad = c->n_pad;
  int n_sums = 0;
  std::vector<TraceSlab> tslabs;
  c->T_max = 1;
  for (int p = 0; p < np; ++p) {
    Subdomain sd;
    sd.s0 = c->slab_start[p];
    sd.s1 = c->slab_start[p + 1];
    sd.e0 = std::max(0, sd.s0 - c->part_nl[p]);
    sd.e1 = std::min(c->n_t, sd.s1 + c->part_nl[p]);
    sd.T = sd.e1 - sd.e0;
    sd.lo = sd.s0 - sd.e0;
    sd.hi = sd.s1 - 1 - sd.e0;
    sd.sep_left = sd.e0 > 0 ? sd.e0 - 1 : -1;
    sd.sep_right = sd.e1 < c->n_t ? sd.e1 : -1;
    sd.slot_base = n_sums;
    sd.nfac = sd.T;
    n_sums += 2 * sd.T;
    for (int tl = sd.lo; tl <= sd.hi; ++tl) {
      TraceSlab ts;
      ts.t = sd.e0 + tl;
      ts.sd = sd.slot_base + tl;                                // Sigma_tl
      ts.sy = (tl + 1 < sd.T) ? sd.slot_base + sd.T + tl : -1;  // Y_tl
      ts.sym = (tl > 0) ? sd.slot_base + sd.T + tl - 1 : -1;    // Y_{tl-1}
      tslabs.push_back(ts);
    }
    c->T_max = std::max(c->T_max, sd.T);
    c->parts.push_back(sd);
  }
  // Two-ended form of the one-part factorisation: D_t by Schur complements
  // from slab 0 up to the middle slab m and from slab n_t - 1 down to m + 1;
  // D_m takes both neighbours' terms, so D_m^-1 = Sigma_mm, and the
  // selected inverse runs outward from m in both halves.  The halves' steps
  // are batched into the same launches, which halves the sequential chain.
  // The reversed half's last factor step (local m' - 1 with m' = n_t - 1 - m)
  // runs before the forward half's middle step (local m) because m' <= m.
  c->twist = np == 1 && c->opt.chain == QSEL_CHAIN_TWO_ENDED && c->n_t >= 3;
  if (c->twist) {
    const int m = c->n_t / 2;
    Subdomain &f = c->half[0], &r = c->half[1];
    f = c->parts[0];
    r = c->parts[0];
    f.e0 = 0;
    f.e1 = m + 1;
    f.s0 = 0;
    f.s1 = m + 1;
    f.T = f.nfac = m + 1;
    f.lo = 0;
    f.hi = m;
    f.rev = 0;
    f.slot_base = 0;
    r.e0 = m;
    r.e1 = c->n_t;
    r.s0 = m + 1;
    r.s1 = c->n_t;
    r.T = c->n_t - m;
    r.nfac = r.T - 1;
    r.lo = 0;
    r.hi = r.T - 2;
    r.rev = 1;
    r.slot_base = 2 * f.T;
    n_sums = 2 * (f.T + r.T);
    // per global slab: Sigma_tt, Y of the pair (t, t+1), Y of (t-1, t);
    // the reversed half's Y slot tl holds the pair (g(tl + 1), g(tl))
    tslabs.clear();
    for (int t = 0; t < c->n_t; ++t) {
      TraceSlab ts;
      ts.t = t;
      if (t <= m) {
        ts.sd = f.slot_base + t;
        ts.sy = (t < m) ? f.slot_base + f.T + t : r.slot_base + r.T + (r.T - 2);
        ts.sym = (t > 0) ? f.slot_base + f.T + t - 1 : -1;
      } else {
        const int tl = c->n_t - 1 - t;
        ts.sd = r.slot_base + tl;
        ts.sy = (tl >= 1) ? r.slot_base + r.T + tl - 1 : -1;
        ts.sym = r.slot_base + r.T + tl;
      }
      tslabs.push_back(ts);
    }
    c->T_max = f.T;
  }
  TRY(c->alloc(&c->d_partials, (size_t)np * corr_grid() * kMaxTheta));
  QSEL_CUDA_TRY(cudaMemset(c->d_partials, 0, (size_t)np * corr_grid() * kMaxTheta * sizeof(double)));
  for (int p = 0; p < np; ++p) c->parts[p].partial = c->d_partials + (size_t)p * corr_grid() * kMaxTheta;
  c->half[0].partial = c->half[1].partial = c->d_partials;
  TRY(c->alloc(&c->d_diag, (size_t)n));
  TRY(c->alloc(&c->d_selinv, (size_t)n));
  TRY(c->alloc(&c->d_corr, (size_t)n));
  TRY(c->alloc(&c->d_corr4, (size_t)n));
  TRY(c->alloc(&c->d_traces, 4));
  TRY(c->alloc(&c->d_err, 4));
  TRY(c->alloc_bytes(reinterpret_cast<void **>(&c->d_diag_scratch), extract_scratch_bytes(n_pad)));

  // dense working sets: as many subdomains per wave as fit in 85 % of the free
  // device memory (at most kMaxBatch)
  const size_t mat = (size_t)n_pad * n_pad * esz;
  const size_t svec = (size_t)n_pad * c->ld * esz;
  // sweep scratch: two sets of U, V and the column panel W (n_pad x
  // 64 kSweepPanel each), Vk (64 kSweepPanel x 64) and P (64 x 64)
  const size_t panel = (size_t)n_pad * 64 * kSweepPanel * esz;
  const bool split_panels = c->mixed && c->tc_passes == 3;
  auto slot_bytes = [&](int T) {
    return (size_t)(T + 5 + (split_panels ? 4 : 0)) * mat + (split_panels ? 10 : 6) * panel +
           (size_t)2 * kSweepPanel * (kSweepPanel + 1) * 64 * 64 * esz + (size_t)(T + 5) * svec + 4096;
  };
  size_t free_b = 0, total_b = 0;
  QSEL_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  const size_t budget = (size_t)(0.85 * (double)free_b);
  if (c->twist && budget / slot_bytes(c->T_max) < 2) {
    // the two halves' working sets do not fit: the one chain after all, with
    // the part's own bookkeeping
    c->twist = false;
    const Subdomain &sd = c->parts[0];
    tslabs.clear();
    n_sums = 2 * sd.T;
    for (int tl = sd.lo; tl <= sd.hi; ++tl)
      tslabs.push_back(TraceSlab{sd.e0 + tl, sd.slot_base + tl, (tl + 1 < sd.T) ? sd.slot_base + sd.T + tl : -1,
                                 (tl > 0) ? sd.slot_base + sd.T + tl - 1 : -1});
    c->T_max = sd.T;
  }
  const size_t per_slot = slot_bytes(c->T_max);
  const size_t fit = budget / per_slot;
  if (fit < 1)
    return fail(QSEL_ENOMEM, "one subdomain's dense working set (" + std::to_string(per_slot >> 20) +
                                 " MiB) does not fit in device memory");
  c->wave = (int)std::min<size_t>(std::min<size_t>(fit, (size_t)std::min(kMaxBatch, c->slot_cap)), (size_t)np);
  TRY(c->alloc(&c->d_sums, (size_t)kMaxTheta * std::max(n_sums, 1)));
  QSEL_CUDA_TRY(cudaMemset(c->d_sums, 0, (size_t)kMaxTheta * std::max(n_sums, 1) * sizeof(double)));
  c->n_trace_slabs = (int)tslabs.size();
  TRY(upload(c, &c->d_slabs, tslabs));
  c->slots.resize(c->twist ? 2 : c->wave);
  for (size_t i = 0; i < c->slots.size(); ++i) {
    DenseSlot &sl = c->slots[i];
    // the reversed half's last pivot block is the forward half's middle one
    const int own = c->twist ? c->half[i].nfac : c->T_max;
    sl.Dinv.resize(c->twist ? c->half[i].T : c->T_max);
    for (int t = 0; t < own; ++t) TRY(c->alloc_bytes(&sl.Dinv[t], mat));
    if (c->twist && i == 1) sl.Dinv[c->half[1].T - 1] = c->slots[0].Dinv[c->half[0].T - 1];
    TRY(c->alloc_bytes(&sl.SigA, mat));
    TRY(c->alloc_bytes(&sl.SigB, mat));
    TRY(c->alloc_bytes(&sl.Y, mat));
    TRY(c->alloc_bytes(&sl.W, mat));
    TRY(c->alloc_bytes(&sl.V, mat));
    TRY(c->alloc_bytes(&sl.P, (size_t)2 * kSweepPanel * 64 * 64 * esz));   // per panel parity and pivot
    TRY(c->alloc_bytes(&sl.U, panel));
    TRY(c->alloc_bytes(&sl.Vs, panel));
    TRY(c->alloc_bytes(&sl.Wp, panel));
    TRY(c->alloc_bytes(&sl.U2, panel));
    TRY(c->alloc_bytes(&sl.V2, panel));
    TRY(c->alloc_bytes(&sl.Wp2, panel));
    if (split_panels) {
      for (auto &sp : sl.Sp) TRY(c->alloc_bytes(&sp, panel));
      for (auto &gs : sl.Gs) TRY(c->alloc_bytes(&gs, mat));
    }
    TRY(c->alloc_bytes(&sl.Vk, (size_t)2 * kSweepPanel * kSweepPanel * 64 * 64 * esz));
    TRY(c->alloc_bytes(&sl.wbuf, (size_t)c->T_max * svec));
    TRY(c->alloc_bytes(&sl.ybuf, svec));
    TRY(c->alloc_bytes(&sl.tmp, svec));
    TRY(c->alloc_bytes(&sl.bright, svec));
    TRY(c->alloc_bytes(&sl.tra, svec));
    TRY(c->alloc_bytes(&sl.trb, svec));
  }
  QSEL_CUDA_TRY(cudaHostAlloc(&c->h_counters, 64, cudaHostAllocDefault));
  QSEL_CUDA_TRY(cudaHostAlloc(&c->h_small, 64 * sizeof(double), cudaHostAllocDefault));
  QSEL_CUDA_TRY(cudaHostAlloc(&c->h_theta, 4 * sizeof(double), cudaHostAllocDefault));
  TRY(c->alloc(&c->d_theta, 4));
  TRY(c->alloc(&c->d_loop, 4));
  TRY(c->alloc(&c->d_tol2, 1));
  QSEL_CUDA_TRY(cudaMemset(c->d_loop, 0, 4 * sizeof(int32_t)));
  for (auto &e : c->ev) QSEL_CUDA_TRY(cudaEventCreate(&e));
  QSEL_CUDA_TRY(cudaStreamCreateWithFlags(&c->pcg_stream, cudaStreamNonBlocking));
  QSEL_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  QSEL_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_samples, cudaEventDisableTiming));
  if (c->mixed) {
    // the sweep's panels on a high-priority stream, so that their few CTAs are
    // scheduled ahead of the pending tiles of the concurrent update
    int least = 0, greatest = 0;
    QSEL_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    QSEL_CUDA_TRY(cudaStreamCreateWithPriority(&c->sweep_ss.hi, cudaStreamNonBlocking, greatest));
    QSEL_CUDA_TRY(cudaStreamCreateWithPriority(&c->sweep_ss.lo, cudaStreamNonBlocking, least));
    for (cudaEvent_t *e : {&c->sweep_ss.fork, &c->sweep_ss.panel, &c->sweep_ss.lookahead, &c->sweep_ss.scatter})
      QSEL_CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  }
  return ok();
}

// The kernels' view of the separable model (Q = tau Q_t (x) Q_s + obs):
// every block is Q_s (or dQ_s/dlog kappa) scaled by a time coefficient.
static void set_separable_views(qsel_ctx *c) {
  c->mod.diag = BlockVals{c->d_qs, 0, c->tc.a0};
  c->mod.off = BlockVals{c->d_qs, 0, c->tc.a1};
  c->mod.obs = c->d_obs;
  c->mod.obs_w = c->obs_w;
  c->dmod.n = 3;
  c->dmod.diag[0] = BlockVals{c->d_dqs, 0, c->tc.a0};   // d/dlog kappa
  c->dmod.off[0] = BlockVals{c->d_dqs, 0, c->tc.a1};
  c->dmod.diag[1] = BlockVals{c->d_qs, 0, c->tc.a0};    // d/dlog tau
  c->dmod.off[1] = BlockVals{c->d_qs, 0, c->tc.a1};
  c->dmod.diag[2] = BlockVals{c->d_qs, 0, c->tc.r0};    // d/dlogit rho
  c->dmod.off[2] = BlockVals{c->d_qs, 0, c->tc.r1};
}

// The diffusion model's view: per-slab diagonal blocks, couplings K1 scaled
// per slab pair (layout of d_blk and d_blk_coef in model.cu).
static void set_diffusion_views(qsel_ctx *c) {
  const int64_t e = c->n_ent, tot = (int64_t)c->n_t * e;
  const double *K1 = c->d_blk + 4 * tot, *dK1 = K1 + e;
  const double *cB = c->d_blk_coef, *cBt = cB + c->n_t, *cBe = cB + 2 * c->n_t;
  c->mod.diag = BlockVals{c->d_blk, e, nullptr};
  c->mod.off = BlockVals{K1, 0, cB};
  c->mod.obs = c->d_obs;
  c->mod.obs_w = c->obs_w;
  c->dmod.n = 3;
  c->dmod.diag[0] = BlockVals{c->d_blk + tot, e, nullptr};       // d/dlog gamma_s
  c->dmod.off[0] = BlockVals{dK1, 0, cB};
  c->dmod.diag[1] = BlockVals{c->d_blk + 2 * tot, e, nullptr};   // d/dlog gamma_t
  c->dmod.off[1] = BlockVals{K1, 0, cBt};
  c->dmod.diag[2] = BlockVals{c->d_blk + 3 * tot, e, nullptr};   // d/dlog gamma_e
  c->dmod.off[2] = BlockVals{K1, 0, cBe};
}

// ---------------------------------------------------------------------------
// Pipeline
// ---------------------------------------------------------------------------
static Err run_model(qsel_ctx *c) {
  if (c->model_kind == QSEL_MODEL_BLOCK_TRIDIAGONAL) return ok();   // values set by the caller
  // theta goes through pinned host memory, so a captured graph picks up the
  // value set before each replay
  c->h_theta[0] = c->theta.log_kappa;
  c->h_theta[1] = c->theta.log_tau;
  c->h_theta[2] = c->theta.logit_rho;
  QSEL_CUDA_TRY(cudaMemcpyAsync(c->d_theta, c->h_theta, 3 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  if (c->model_kind == QSEL_MODEL_DIFFUSION) {
    launch_diffusion_values(c->stream, c->d_theta, c->n_t, c->n_ent, c->d_c_pat, c->d_g_pat, c->d_h_pat,
                            c->d_h3_pat, c->d_blk, c->d_blk_coef);
    QSEL_CUDA_TRY(cudaGetLastError());
    return ok();
  }
  launch_time_coeffs(c->stream, c->d_theta, c->n_t, c->tc);
  launch_qs_values(c->stream, c->n_ent, c->d_c_pat, c->d_g_pat, c->d_h_pat, c->d_isqc_pat,
                   c->tc.scalars, c->d_qs, c->d_dqs, c->d_kc);
  QSEL_CUDA_TRY(cudaGetLastError());
  return ok();
}

template <typename T>
static PcgVec<T> make_pcg(qsel_ctx *c, T *x, T *r, T *z, T *p, T *q) {
  PcgVec<T> v;
  v.n = c->n;
  v.ld = c->ld;
  v.n_blocks_dot = bt_spmm_grid(c->n);
  v.n_tiles = pcg_update_grid(c->n);
  v.x = x;
  v.r = r;
  v.z = z;
  v.p = p;
  v.q = q;
  v.partial_a = c->d_pa;
  v.partial_b = c->d_pb;
  v.alpha = c->d_scal;
  v.beta = c->d_scal + c->ld;
  v.rho = c->d_scal + 2 * c->ld;
  v.bb = c->d_scal + 3 * c->ld;
  v.rr = c->d_scal + 4 * c->ld;
  v.max_rel = c->d_scal + 5 * c->ld;
  v.active = c->d_active;
  v.counters = c->d_counters;
  return v;
}

// Multi-RHS block-Jacobi PCG from x = 0 on the right-hand sides held in v.r.
// Per-column stop ||r_c|| <= tol ||b_c|| (recursive residual), converged
// columns frozen; the host polls the active-column count every 8 iterations.
template <typename T>
static Err pcg_solve(qsel_ctx *c, const PcgVec<T> &v, const T *pblk, double tol, int max_iter, int *iters,
                     double *max_rel, bool *converged) {
  cudaStream_t s = c->stream;
  const size_t vbytes = (size_t)c->n * c->ld * sizeof(T);
  QSEL_CUDA_TRY(cudaMemsetAsync(v.x, 0, vbytes, s));
  QSEL_CUDA_TRY(cudaMemsetAsync(v.p, 0, vbytes, s));
  QSEL_CUDA_TRY(cudaMemsetAsync(v.alpha, 0, (size_t)c->ld * sizeof(double), s));
  launch_pcg_update<T>(s, v, pblk, c->bsize, c->kron ? &c->kop : nullptr);
  launch_pcg_reduce_beta<T>(s, v, tol, 1);
  launch_pcg_p_update<T>(s, v);
  BtSpmmArgs<T> a{};
  a.pat = c->pat;
  a.m = c->mod;
  a.n_s = c->n_s;
  a.n_t = c->n_t;
  a.ld = c->ld;
  a.x = v.p;
  a.y = v.q;
  a.dot_partial = c->d_pa;
  a.tmp = v.z;  // free while the SpMM runs (rewritten by the preconditioner)
  const int check_every = 8;
  int it = 0;
  bool done = false;
  QSEL_CUDA_TRY(cudaMemcpyAsync(c->h_counters, v.counters, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  QSEL_CUDA_TRY(cudaStreamSynchronize(s));
  if (c->h_counters[0] == 0) done = true;
  while (!done && it < max_iter) {
    const int batch = std::min(check_every, max_iter - it);
    for (int b = 0; b < batch; ++b) {
      launch_bt_spmm<T>(s, a);
      launch_pcg_reduce_alpha<T>(s, v);
      launch_pcg_update<T>(s, v, pblk, c->bsize, c->kron ? &c->kop : nullptr);
      launch_pcg_reduce_beta<T>(s, v, tol, 0);
      launch_pcg_p_update<T>(s, v);
    }
    it += batch;
    QSEL_CUDA_TRY(cudaGetLastError());
    QSEL_CUDA_TRY(cudaMemcpyAsync(c->h_counters, v.counters, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    QSEL_CUDA_TRY(cudaStreamSynchronize(s));
    if (c->h_counters[0] == 0) done = true;
  }
  QSEL_CUDA_TRY(cudaMemcpyAsync(c->h_small, v.max_rel, sizeof(double), cudaMemcpyDeviceToHost, s));
  QSEL_CUDA_TRY(cudaStreamSynchronize(s));
  *iters = it;
  *max_rel = c->h_small[0];
  *converged = done;
  return ok();
}

// Perturbation right-hand sides and the global samples X = Q^-1 R.
//   FP64: one PCG in double.
//   mixed: iterative refinement -- the true residual R - Q X in double, an
//   FP32 PCG for the correction to a loose inner tolerance, X += correction
//   in double -- until every column meets pcg_tol in double.
static Err solve_R(qsel_ctx *c);

static Err run_sampler(qsel_ctx *c) {
  cudaStream_t s = c->stream;
  launch_philox_normals(s, c->opt.seed, 0u, c->n, c->k, c->ld, c->d_z1);
  launch_philox_normals(s, c->opt.seed, 1u, c->n_obs, c->k, c->ld, c->d_z2);
  launch_perturbation_rhs(s, c->pat, c->d_kc, c->n_s, c->n_t, c->ld, c->tc.bdiag, c->tc.scalars,
                          c->d_z1, c->d_z2, c->d_obs_index, 1.0 / c->sigma, c->d_R);
  c->have_rhs = true;
  QSEL_CUDA_TRY(cudaEventRecord(c->ev[1], s));
  return solve_R(c);
}

// X = Q^-1 R for the right-hand sides in d_R (all ld columns; zero columns
// are inactive from the start): multi-RHS PCG in FP64, or FP32 PCG inside
// FP64 iterative refinement for the mixed form.  Records pcg_iterations and
// pcg_max_rel_residual.
static Err solve_R(qsel_ctx *c) {
  cudaStream_t s = c->stream;
  const size_t vec = (size_t)c->n * c->ld;
  if (c->kron) TRY(kron_prepare(c));
  if (!c->mixed) {
    double *pblk = static_cast<double *>(c->d_pblk);
    if (!c->kron)
      launch_jacobi_setup<double>(s, c->pat, c->mod, c->n_s, c->n_t,
                                  c->bsize, pblk, c->d_err);
    QSEL_CUDA_TRY(cudaMemcpyAsync(c->d_r, c->d_R, vec * sizeof(double), cudaMemcpyDeviceToDevice, s));
    PcgVec<double> v = make_pcg<double>(c, c->d_X, c->d_r, c->d_zv, c->d_p, c->d_q);
    int it = 0;
    double rel = 0.0;
    bool conv = false;
    TRY(pcg_solve<double>(c, v, pblk, c->opt.pcg_tol, c->opt.pcg_max_iter, &it, &rel, &conv));
    c->stats.pcg_iterations = it;
    c->stats.pcg_max_rel_residual = rel;
    if (!conv)
      return fail(QSEL_ENOCONV, "PCG did not reach pcg_tol within pcg_max_iter iterations (max relative residual " +
                                    std::to_string(rel) + ")");
    return ok();
  }
  float *pblk = static_cast<float *>(c->d_pblk);
  if (!c->kron)
    launch_jacobi_setup<float>(s, c->pat, c->mod, c->n_s, c->n_t,
                               c->bsize, pblk, c->d_err);
  PcgVec<float> v = make_pcg<float>(c, c->f_x, c->f_r, c->f_z, c->f_p, c->f_q);
  QSEL_CUDA_TRY(cudaMemsetAsync(c->d_X, 0, vec * sizeof(double), s));
  QSEL_CUDA_TRY(cudaMemsetAsync(c->d_q, 0, vec * sizeof(double), s));
  BtSpmmArgs<double> a{};
  a.pat = c->pat;
  a.m = c->mod;
  a.n_s = c->n_s;
  a.n_t = c->n_t;
  a.ld = c->ld;
  a.x = c->d_X;
  a.y = c->d_q;
  a.dot_partial = nullptr;
  a.tmp = c->d_z1;  // free until the residual that follows overwrites it
  // inner FP32 solves stop at the reduction still needed (with a margin),
  // floored at what FP32 CG reliably attains
  const double inner_floor = 3e-6;
  const int max_outer = 30;
  int total = 0;
  double rel = 1.0;
  for (int outer = 0;; ++outer) {
    if (outer > 0) launch_bt_spmm<double>(s, a);
    launch_residual(s, c->d_R, c->d_q, c->d_z1, c->f_r, c->n, c->ld, c->d_pa, c->d_pb);
    launch_residual_check(s, c->d_pa, c->d_pb, residual_grid(c->n), c->ld, c->opt.pcg_tol, c->d_counters,
                          c->d_scal + 5 * c->ld);
    QSEL_CUDA_TRY(cudaMemcpyAsync(c->h_counters, c->d_counters, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    QSEL_CUDA_TRY(cudaMemcpyAsync(c->h_small, c->d_scal + 5 * c->ld, sizeof(double), cudaMemcpyDeviceToHost, s));
    QSEL_CUDA_TRY(cudaStreamSynchronize(s));
    rel = c->h_small[0];
    if (c->h_counters[0] == 0) break;
    if (outer == max_outer || total >= c->opt.pcg_max_iter) {
      c->stats.pcg_iterations = total;
      c->stats.pcg_max_rel_residual = rel;
      return fail(QSEL_ENOCONV, "mixed-precision refinement did not reach pcg_tol (max relative residual " +
                                    std::to_string(rel) + ")");
    }
    int it = 0;
    double inner_rel = 0.0;
    bool conv = false;
    const double inner_tol = std::max(inner_floor, 0.5 * c->opt.pcg_tol / std::max(rel, 1e-300));
    TRY(pcg_solve<float>(c, v, pblk, inner_tol, c->opt.pcg_max_iter - total, &it, &inner_rel, &conv));
    total += it;
    launch_accumulate(s, c->d_X, c->f_x, (int64_t)vec);
  }
  c->stats.pcg_iterations = total;
  c->stats.pcg_max_rel_residual = rel;
  return ok();
}

// ---------------------------------------------------------------------------
// Graph mode: the sampler's loops become conditional while nodes of the
// captured graph.  capture_while adds the node at the capture position of s
// (after `init`, which must set the condition) and captures `body` into it
// on the body stream of the given depth; the body must end with a kernel
// that sets the condition.
// ---------------------------------------------------------------------------
template <class Init, class Body>
static Err capture_while(qsel_ctx *c, cudaStream_t s, int depth, Init init, Body body) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  QSEL_CUDA_TRY(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd));
  if (st != cudaStreamCaptureStatusActive) return fail(QSEL_ESTATE, "graph-mode loop outside a stream capture");
  cudaGraphConditionalHandle h;
  QSEL_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
  TRY(init(h));
  QSEL_CUDA_TRY(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd));
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  QSEL_CUDA_TRY(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
  cudaGraph_t body_graph = np.conditional.phGraph_out[0];
  QSEL_CUDA_TRY(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaStream_t b = c->body_stream[depth];
  QSEL_CUDA_TRY(cudaStreamBeginCaptureToGraph(b, body_graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  Err e = body(b, h);
  cudaGraph_t captured = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(b, &captured);
  if (e.code) return e;
  if (ce != cudaSuccess) return cuda_fail(ce, "capture of a loop body", __FILE__, __LINE__);
  return ok();
}

template <typename T>
static void pcg_start(qsel_ctx *c, cudaStream_t s, const PcgVec<T> &v, const T *pblk, double tol) {
  const size_t vbytes = (size_t)c->n * c->ld * sizeof(T);
  cudaMemsetAsync(v.x, 0, vbytes, s);
  cudaMemsetAsync(v.p, 0, vbytes, s);
  cudaMemsetAsync(v.alpha, 0, (size_t)c->ld * sizeof(double), s);
  launch_pcg_update<T>(s, v, pblk, c->bsize, c->kron ? &c->kop : nullptr);
  launch_pcg_reduce_beta<T>(s, v, tol, 1);
  launch_pcg_p_update<T>(s, v);
}

template <typename T>
static void pcg_steps(qsel_ctx *c, cudaStream_t s, const PcgVec<T> &v, const T *pblk, double tol, int count) {
  BtSpmmArgs<T> a{};
  a.pat = c->pat;
  a.m = c->mod;
  a.n_s = c->n_s;
  a.n_t = c->n_t;
  a.ld = c->ld;
  a.x = v.p;
  a.y = v.q;
  a.dot_partial = c->d_pa;
  a.tmp = v.z;  // free while the SpMM runs (rewritten by the preconditioner)
  for (int b = 0; b < count; ++b) {
    launch_bt_spmm<T>(s, a);
    launch_pcg_reduce_alpha<T>(s, v);
    launch_pcg_update<T>(s, v, pblk, c->bsize, c->kron ? &c->kop : nullptr);
    launch_pcg_reduce_beta<T>(s, v, tol, 0);
    launch_pcg_p_update<T>(s, v);
  }
}

constexpr int kGraphCheckEvery = 8;

// PCG with the device-driven stop: while (active columns and iterations <
// max_iter - loop[2]) run 8 iterations.
template <typename T>
static Err pcg_graph(qsel_ctx *c, cudaStream_t s, int depth, const PcgVec<T> &v, const T *pblk, double tol) {
  pcg_start<T>(c, s, v, pblk, tol);
  const int max_iter = c->opt.pcg_max_iter;
  return capture_while(
      c, s, depth,
      [&](cudaGraphConditionalHandle h) {
        launch_loop_init(s, h, v.counters, c->d_loop, max_iter);
        return ok();
      },
      [&](cudaStream_t b, cudaGraphConditionalHandle h) {
        pcg_steps<T>(c, b, v, pblk, tol, kGraphCheckEvery);
        launch_loop_ctl(b, h, v.counters, c->d_loop, kGraphCheckEvery, max_iter);
        QSEL_CUDA_TRY(cudaGetLastError());
        return ok();
      });
}

// The sampler of run_sampler, enqueued for capture (no host synchronisation).
static Err run_sampler_graph(qsel_ctx *c) {
  cudaStream_t s = c->stream;
  launch_philox_normals(s, c->opt.seed, 0u, c->n, c->k, c->ld, c->d_z1);
  launch_philox_normals(s, c->opt.seed, 1u, c->n_obs, c->k, c->ld, c->d_z2);
  launch_perturbation_rhs(s, c->pat, c->d_kc, c->n_s, c->n_t, c->ld, c->tc.bdiag, c->tc.scalars,
                          c->d_z1, c->d_z2, c->d_obs_index, 1.0 / c->sigma, c->d_R);
  const size_t vec = (size_t)c->n * c->ld;
  QSEL_CUDA_TRY(cudaMemsetAsync(c->d_loop, 0, 4 * sizeof(int32_t), s));
  if (!c->mixed) {
    double *pblk = static_cast<double *>(c->d_pblk);
    launch_jacobi_setup<double>(s, c->pat, c->mod, c->n_s, c->n_t,
                                c->bsize, pblk, c->d_err);
    QSEL_CUDA_TRY(cudaMemcpyAsync(c->d_r, c->d_R, vec * sizeof(double), cudaMemcpyDeviceToDevice, s));
    PcgVec<double> v = make_pcg<double>(c, c->d_X, c->d_r, c->d_zv, c->d_p, c->d_q);
    TRY(pcg_graph<double>(c, s, 0, v, pblk, c->opt.pcg_tol));
    launch_loop_status(s, v.counters, c->d_loop);
    QSEL_CUDA_TRY(cudaGetLastError());
    return ok();
  }
  float *pblk = static_cast<float *>(c->d_pblk);
  launch_jacobi_setup<float>(s, c->pat, c->mod, c->n_s, c->n_t,
                             c->bsize, pblk, c->d_err);
  PcgVec<float> v = make_pcg<float>(c, c->f_x, c->f_r, c->f_z, c->f_p, c->f_q);
  v.tol2_dev = c->d_tol2;
  QSEL_CUDA_TRY(cudaMemsetAsync(c->d_X, 0, vec * sizeof(double), s));
  QSEL_CUDA_TRY(cudaMemsetAsync(c->d_q, 0, vec * sizeof(double), s));
  BtSpmmArgs<double> a{};
  a.pat = c->pat;
  a.m = c->mod;
  a.n_s = c->n_s;
  a.n_t = c->n_t;
  a.ld = c->ld;
  a.x = c->d_X;
  a.y = c->d_q;
  a.dot_partial = nullptr;
  a.tmp = c->d_z1;  // free until the residual that follows overwrites it
  const double inner_floor = 3e-6;
  const int max_outer = 30;
  const double tol = c->opt.pcg_tol;
  double *max_rel = c->d_scal + 5 * c->ld;
  const int max_iter = c->opt.pcg_max_iter;
  return capture_while(
      c, s, 0,
      [&](cudaGraphConditionalHandle h) {
        launch_residual(s, c->d_R, c->d_q, c->d_z1, c->f_r, c->n, c->ld, c->d_pa, c->d_pb);
        launch_residual_check(s, c->d_pa, c->d_pb, residual_grid(c->n), c->ld, tol, c->d_counters, max_rel);
        launch_refine_ctl(s, h, c->d_counters, max_rel, c->d_loop, 1, max_outer, max_iter, tol, inner_floor,
                          c->d_tol2);
        return ok();
      },
      [&](cudaStream_t b, cudaGraphConditionalHandle h) {
        TRY(pcg_graph<float>(c, b, 1, v, pblk, 1.0));
        launch_accumulate(b, c->d_X, c->f_x, (int64_t)vec);
        launch_bt_spmm<double>(b, a);
        launch_residual(b, c->d_R, c->d_q, c->d_z1, c->f_r, c->n, c->ld, c->d_pa, c->d_pb);
        launch_residual_check(b, c->d_pa, c->d_pb, residual_grid(c->n), c->ld, tol, c->d_counters, max_rel);
        launch_refine_ctl(b, h, c->d_counters, max_rel, c->d_loop, 0, max_outer, max_iter, tol, inner_floor,
                          c->d_tol2);
        QSEL_CUDA_TRY(cudaGetLastError());
        return ok();
      });
}

// Preconditioned Krylov sampler (Algorithm 5.1), FP64: two passes of m
// Lanczos steps on L^-1 Q L^-T for all columns at once (see lanczos.cu).
static Err run_sampler_lanczos(qsel_ctx *c) {
  cudaStream_t s = c->stream;
  const int m = c->opt.lanczos_steps;
  const size_t vec = (size_t)c->n * c->ld;
  const int b = c->bsize;
  const int nblk = (c->n + b - 1) / b;
  if (!c->lz.ready) {
    for (auto &p : c->lz.vec) TRY(c->alloc(&p, vec));
    TRY(c->alloc(&c->lz.u, vec));
    TRY(c->alloc(&c->lz.q, vec));
    TRY(c->alloc(&c->lz.xt, vec));
    TRY(c->alloc(&c->lz.linv, (size_t)nblk * b * b));
    TRY(c->alloc(&c->lz.alpha, (size_t)m * c->ld));
    TRY(c->alloc(&c->lz.beta, (size_t)m * c->ld));
    TRY(c->alloc(&c->lz.coef, (size_t)m * c->ld));
    TRY(c->alloc(&c->lz.eta, (size_t)c->ld));
    TRY(c->alloc(&c->lz.zero, (size_t)c->ld));
    TRY(c->alloc(&c->lz.partial, (size_t)lz_grid(c->n) * c->ld));
    TRY(c->alloc(&c->lz.dwork, (size_t)2 * m * c->ld));
    TRY(c->alloc(&c->lz.U, (size_t)m * m * c->ld));
    QSEL_CUDA_TRY(cudaMemset(c->lz.zero, 0, (size_t)c->ld * sizeof(double)));
    c->lz.ready = true;
  }
  launch_philox_normals(s, c->opt.seed, 0u, c->n, c->k, c->ld, c->d_z1);
  QSEL_CUDA_TRY(cudaEventRecord(c->ev[1], s));
  launch_bj_cholinv(s, c->pat, c->mod, c->n_s, c->n_t, b, c->lz.linv,
                    c->d_err);
  LanczosArgs la{c->n, c->ld, c->k, m};
  BtSpmmArgs<double> sp{};
  sp.pat = c->pat;
  sp.m = c->mod;
  sp.n_s = c->n_s;
  sp.n_t = c->n_t;
  sp.ld = c->ld;
  sp.dot_partial = nullptr;
  for (int pass = 0; pass < 2; ++pass) {
    double *vp = c->lz.vec[0], *v = c->lz.vec[1], *w = c->lz.vec[2];
    // v_1 = z / eta
    QSEL_CUDA_TRY(cudaMemcpyAsync(v, c->d_z1, vec * sizeof(double), cudaMemcpyDeviceToDevice, s));
    QSEL_CUDA_TRY(cudaMemsetAsync(vp, 0, vec * sizeof(double), s));
    if (pass == 0) {
      launch_lz_vec(s, 2, la, nullptr, nullptr, v, nullptr, nullptr, nullptr, c->lz.partial);
      launch_lz_reduce(s, la, c->lz.partial, true, c->lz.eta, nullptr);
    } else {
      QSEL_CUDA_TRY(cudaMemsetAsync(c->lz.xt, 0, vec * sizeof(double), s));
    }
    launch_lz_scale(s, la, v, c->lz.eta);
    for (int j = 0; j < m; ++j) {
      const double *beta_prev = j == 0 ? c->lz.zero : c->lz.beta + (size_t)(j - 1) * c->ld;
      double *alpha_j = c->lz.alpha + (size_t)j * c->ld;
      double *beta_j = c->lz.beta + (size_t)j * c->ld;
      // w = L^-1 Q L^-T v  (the SpMM's time combination uses w as scratch)
      launch_block_apply(s, c->lz.linv, b, c->n, c->ld, v, c->lz.u, true);
      sp.x = c->lz.u;
      sp.y = c->lz.q;
      sp.tmp = w;
      launch_bt_spmm<double>(s, sp);
      launch_block_apply(s, c->lz.linv, b, c->n, c->ld, c->lz.q, w, false);
      if (pass == 0) {
        launch_lz_vec(s, 0, la, vp, v, w, nullptr, nullptr, beta_prev, c->lz.partial);
        launch_lz_reduce(s, la, c->lz.partial, false, alpha_j, nullptr);
        launch_lz_vec(s, 1, la, nullptr, v, w, nullptr, nullptr, alpha_j, c->lz.partial);
        launch_lz_reduce(s, la, c->lz.partial, true, beta_j, nullptr);
      } else {
        // the same vectors from the stored coefficients, accumulating x~
        launch_lz_vec(s, 0, la, vp, v, w, c->lz.xt, c->lz.coef + (size_t)j * c->ld, beta_prev, c->lz.partial);
        launch_lz_vec(s, 1, la, nullptr, v, w, nullptr, nullptr, alpha_j, c->lz.partial);
      }
      launch_lz_scale(s, la, w, beta_j);
      double *t = vp;
      vp = v;
      v = w;
      w = t;
    }
    if (pass == 0)
      launch_lz_quadrature(s, la, c->lz.alpha, c->lz.beta, c->lz.eta, c->lz.dwork, c->lz.U, c->lz.coef, c->d_err);
  }
  // rewind the preconditioner: x = L^-T x~
  launch_block_apply(s, c->lz.linv, b, c->n, c->ld, c->lz.xt, c->d_X, true);
  QSEL_CUDA_TRY(cudaGetLastError());
  c->stats.pcg_iterations = m;
  c->stats.pcg_max_rel_residual = 0.0;
  c->lz.ran = true;
  return ok();
}

// The pattern values of the derivative blocks whose inner products with a
// Sigma or Y block of global slab t the extraction forms.
template <typename T>
static void set_sum_vals(ExtractEntry<T> &xe, const BlockVals *bv, int n, int t) {
  for (int j = 0; j < kMaxTheta; ++j) xe.sv[j] = j < n ? bv[j].at(t) : nullptr;
}

static void phase_mark(qsel_ctx *c, std::vector<std::pair<cudaEvent_t, int>> &marks, int phase) {
  if (c->graph_mode) return;
  cudaEvent_t e = c->phase_event();
  cudaEventRecord(e, c->stream);
  marks.emplace_back(e, phase);
}

// Forward block factorisation, backward Takahashi recursion and RB correction
// for the subdomains [p0, p1) held in slots 0 .. p1-p0-1, in lockstep.
// stages: 1 = factorisation and Takahashi, 2 = correction (needs the samples).
template <typename T>
static Err run_wave(qsel_ctx *c, int p0, int p1, std::vector<std::pair<cudaEvent_t, int>> &marks, int stages = 3) {
  cudaStream_t s = c->stream;
  const int n_pad = c->n_pad, n_s = c->n_s, ld = c->ld;
  // the wave's parts: p0..p1 of the partition, or the two halves of the
  // one-part form factored from both ends
  if (c->twist) p1 = p0 + 2;
  auto part = [&](int p) -> Subdomain & { return c->twist ? c->half[p - p0] : c->parts[p]; };
  const size_t svec = (size_t)n_pad * ld;
  int maxT = 0;
  for (int p = p0; p < p1; ++p) maxT = std::max(maxT, part(p).T);
  auto slot = [&](int p) -> DenseSlot & { return c->slots[p - p0]; };
  auto Dinv = [&](int p, int t) { return static_cast<T *>(slot(p).Dinv[t]); };
  auto buf = [](void *x) { return static_cast<T *>(x); };
  if (stages & 1) {
  phase_mark(c, marks, -1);
  // ---- forward: D_t assembled (Schur), inverted in place, W_t = c_t Q_s D_t^-1
  for (int t = 0; t < maxT; ++t) {
    SchurBatch<T> sb{};
    SweepBatch<T> wb{};
    SpBatch<T, T> gb{};
    for (int p = p0; p < p1; ++p) {
      Subdomain &sd = part(p);
      if (t >= sd.nfac) continue;
      DenseSlot &sl = slot(p);
      const int tg = sd.g(t);
      SchurEntry<T> &se = sb.e[sb.count++];
      se.W = (t > 0) ? buf(sl.W) : nullptr;
      se.D = Dinv(p, t);
      se.dval = c->mod.diag.at(tg);
      se.a0 = c->mod.diag.scale_ptr(tg);
      se.cval = (t > 0) ? c->mod.off.at(sd.cpl(t - 1)) : nullptr;
      se.c = (t > 0) ? c->mod.off.scale_ptr(sd.cpl(t - 1)) : nullptr;
      se.obs = c->mod.obs ? c->mod.obs + (size_t)tg * n_s : nullptr;
      wb.pivot_fp64 = c->opt.pivot_precision == QSEL_PIVOT_FP64 ? 1 : 0;
      SweepEntry<T> &we = wb.e[wb.count++];
      we.A = Dinv(p, t);
      we.P = buf(sl.P);
      we.U = buf(sl.U);
      we.V = buf(sl.Vs);
      we.Up[0] = buf(sl.U);
      we.Vp[0] = buf(sl.Vs);
      we.Wp[0] = buf(sl.Wp);
      we.Up[1] = buf(sl.U2);
      we.Vp[1] = buf(sl.V2);
      we.Wp[1] = buf(sl.Wp2);
      we.Vk = buf(sl.Vk);
      for (int q = 0; q < 4; ++q) we.Sp[q] = buf(sl.Sp[q]);
      if (t + 1 < sd.T) {
        SpEntry<T, T> &ge = gb.e[gb.count++];
        ge.B = Dinv(p, t);
        ge.C = nullptr;
        ge.Out = buf(sl.W);
        ge.alpha_ptr = c->mod.off.scale_ptr(sd.cpl(t));
        ge.val = c->mod.off.at(sd.cpl(t));
        ge.alpha = 1.0;
        ge.beta = 0.0;
      }
    }
    launch_schur_assemble<T>(s, sb, c->pat, c->mod.obs_w, n_s, n_pad);
    if (c->twist && t == part(p0).T - 1) {
      // the middle slab m: its other neighbour's term - B_m W'^T, W' = B_m
      // D'^-1 of the reversed half's last factored slab m + 1
      const int m = part(p0).e1 - 1;
      SchurBatch<T> ab{};
      SchurEntry<T> &ae = ab.e[ab.count++];
      ae.W = buf(slot(p0 + 1).W);
      ae.D = Dinv(p0, t);
      ae.cval = c->mod.off.at(m);
      ae.c = c->mod.off.scale_ptr(m);
      ae.accumulate = 1;
      launch_schur_assemble<T>(s, ab, c->pat, c->mod.obs_w, n_s, n_pad);
    }
    spd_inverse<T>(s, wb, n_pad, c->d_err, c->tc_passes, c->mixed ? &c->sweep_ss : nullptr);
    launch_sp_rowgather<T, T>(s, gb, c->pat, n_s, n_pad, n_pad, n_pad, n_pad);
  }
  QSEL_CUDA_TRY(cudaGetLastError());
  phase_mark(c, marks, 0);
  // ---- backward: Sigma_{T-1} = D_{T-1}^-1, then Y_t, Sigma_t
  {
    ExtractBatch<T> xb{};
    for (int p = p0; p < p1; ++p) {
      Subdomain &sd = part(p);
      const int tl = sd.T - 1;
      if (tl < sd.lo || tl > sd.hi) continue;
      ExtractEntry<T> &xe = xb.e[xb.count++];
      xe.S = Dinv(p, tl);
      xe.diag_out = c->d_selinv + (size_t)sd.g(tl) * n_s;
      xe.sums = c->d_sums + kMaxTheta * (size_t)(sd.slot_base + tl);
      set_sum_vals(xe, c->dmod.diag, c->dmod.n, sd.g(tl));
      xe.D0 = nullptr;
      xe.V = nullptr;
    }
    launch_extract<T>(s, xb, c->pat, c->dmod.n, n_s, n_pad, c->d_diag_scratch);
  }
  std::vector<T *> sig_next(p1 - p0, nullptr);
  std::vector<int> flip(p1 - p0, 0);
  for (int p = p0; p < p1; ++p) sig_next[p - p0] = Dinv(p, part(p).T - 1);
  bool use_tc = false;
  if constexpr (std::is_same<T, float>::value) use_tc = c->tc_passes > 0;
  if (use_tc) {
    if constexpr (std::is_same<T, float>::value) {
      // Tensor-core form: Wt = c_t D_t^-1 Q_s (= W^T), Yt = Wt Sigma_{t+1} (= Y^T),
      // Sigma_t = D_t^-1 + Yt (Wt)^T; both products have K-major operands.
      for (int b = 0; b < maxT; ++b) {
        SpBatch<T, T> wb{};
        GemmBatch<T> yb{}, sgb{};
        SweepBatch<T> mb{};
        ExtractBatch<T> xy{}, xs{};
        DiagRowBatch<T> db{};
        std::vector<int> active;
        for (int p = p0; p < p1; ++p) {
          Subdomain &sd = part(p);
          DenseSlot &sl = slot(p);
          const int tl = sd.T - 2 - b;
          if (tl < std::max(sd.lo - 1, 0)) continue;
          active.push_back(p);
          const int tg = sd.g(tl), tc = sd.cpl(tl);
          SpEntry<T, T> &we = wb.e[wb.count++];
          we.B = Dinv(p, tl);
          we.C = nullptr;
          we.Out = buf(sl.W);
          we.alpha_ptr = c->mod.off.scale_ptr(tc);
          we.val = c->mod.off.at(tc);
          we.alpha = 1.0;
          we.beta = 0.0;
          GemmEntry<T> &ye = yb.e[yb.count++];
          ye.A = buf(sl.W);
          ye.B = sig_next[p - p0];
          ye.C0 = nullptr;
          ye.C = buf(sl.Y);
          ye.alpha = 1.0;
          ye.beta = 0.0;
          const bool y_needed = (tl >= sd.lo && tl <= sd.hi) || (tl + 1 >= sd.lo && tl + 1 <= sd.hi);
          if (y_needed) {
            ExtractEntry<T> &xe = xy.e[xy.count++];
            xe.S = buf(sl.Y);   // <M, Y> = <M, Y^T> for symmetric M
            xe.diag_out = nullptr;
            xe.sums = c->d_sums + kMaxTheta * (size_t)(sd.slot_base + sd.T + tl);
            set_sum_vals(xe, c->dmod.off, c->dmod.n, tc);
            xe.D0 = nullptr;
            xe.V = nullptr;
          }
          if (tl >= sd.lo) {
            T *sig_cur = buf(flip[p - p0] ? sl.SigB : sl.SigA);
            GemmEntry<T> &ge = sgb.e[sgb.count++];
            ge.A = buf(sl.Y);
            ge.B = buf(sl.W);
            ge.C0 = Dinv(p, tl);
            ge.C = sig_cur;
            ge.alpha = 1.0;
            ge.beta = 1.0;
            SweepEntry<T> &me = mb.e[mb.count++];
            me.A = sig_cur;
            if (tl <= sd.hi) {
              ExtractEntry<T> &xe = xs.e[xs.count++];
              xe.S = sig_cur;
              xe.diag_out = nullptr;
              xe.sums = c->d_sums + kMaxTheta * (size_t)(sd.slot_base + tl);
              set_sum_vals(xe, c->dmod.diag, c->dmod.n, tg);
              xe.D0 = nullptr;
              xe.V = nullptr;
              DiagRowEntry<T> &de = db.e[db.count++];
              de.D0 = Dinv(p, tl);
              de.P = buf(sl.Y);
              de.R = buf(sl.W);
              de.diag_out = c->d_selinv + (size_t)tg * n_s;
            }
          }
        }
        if (active.empty()) break;
        launch_sp_colgather<T>(s, wb, c->pat, n_s, n_pad);
        const int64_t mm = (int64_t)n_pad * n_pad;
        if (slot(active[0]).Gs[0] != nullptr) {
          // 3xTF32 on operands split once in HBM: W and Sigma_{t+1}, then
          // Y; the persistent 128 x 256-tile kernel
          SplitGemmBatch y2{}, s2{};
          {
            ProfScope ps_(s, PROF_GATHER);
            for (int q = 0; q < yb.count; ++q) {
              DenseSlot &sl = slot(active[q]);
              launch_split_tf32(s, yb.e[q].A, static_cast<float *>(sl.Gs[0]), static_cast<float *>(sl.Gs[1]), mm);
              launch_split_tf32(s, yb.e[q].B, static_cast<float *>(sl.Gs[2]), static_cast<float *>(sl.Gs[3]), mm);
              y2.e[y2.count++] = SplitGemmEntry{static_cast<float *>(sl.Gs[0]), static_cast<float *>(sl.Gs[1]),
                                                static_cast<float *>(sl.Gs[2]), static_cast<float *>(sl.Gs[3]),
                                                nullptr, yb.e[q].C, 1.0f, 0.0f};
            }
          }
          if (!launch_tc_gemm_split(s, y2, n_pad, n_pad, n_pad, n_pad, n_pad, n_pad, false, c->d_err))
            return fail(QSEL_ECUDA, "tensor-core GEMM: tensor map encoding failed");
          launch_extract<T>(s, xy, c->pat, c->dmod.n, n_s, n_pad, c->d_diag_scratch);
          {
            // the parts with a Sigma_t product (the first sgb.count active parts
            // in order); Y's parts replace Sigma_{t+1}'s
            ProfScope ps_(s, PROF_GATHER);
            int q = 0;
            for (int a = 0; a < (int)active.size() && q < sgb.count; ++a) {
              DenseSlot &sl = slot(active[a]);
              if (sgb.e[q].A != buf(sl.Y)) continue;
              launch_split_tf32(s, buf(sl.Y), static_cast<float *>(sl.Gs[2]), static_cast<float *>(sl.Gs[3]), mm);
              s2.e[s2.count++] = SplitGemmEntry{static_cast<float *>(sl.Gs[2]), static_cast<float *>(sl.Gs[3]),
                                                static_cast<float *>(sl.Gs[0]), static_cast<float *>(sl.Gs[1]),
                                                sgb.e[q].C0, sgb.e[q].C, 1.0f, 1.0f};
              ++q;
            }
          }
          if (!launch_tc_gemm_split(s, s2, n_pad, n_pad, n_pad, n_pad, n_pad, n_pad, true, c->d_err))
            return fail(QSEL_ECUDA, "tensor-core GEMM: tensor map encoding failed");
        } else {
          if (!launch_tc_gemm(s, yb, n_pad, n_pad, n_pad, n_pad, n_pad, n_pad, false, c->tc_passes, c->d_err))
            return fail(QSEL_ECUDA, "tensor-core GEMM: tensor map encoding failed");
          launch_extract<T>(s, xy, c->pat, c->dmod.n, n_s, n_pad, c->d_diag_scratch);
          if (!launch_tc_gemm(s, sgb, n_pad, n_pad, n_pad, n_pad, n_pad, n_pad, true, c->tc_passes, c->d_err))
            return fail(QSEL_ECUDA, "tensor-core GEMM: tensor map encoding failed");
        }
        launch_diag64_rows<T>(s, db, n_s, n_pad);
        launch_mirror<T>(s, mb, n_pad);
        launch_extract<T>(s, xs, c->pat, c->dmod.n, n_s, n_pad, c->d_diag_scratch);
        for (int p : active) {
          Subdomain &sd = part(p);
          DenseSlot &sl = slot(p);
          const int tl = sd.T - 2 - b;
          if (tl >= sd.lo) {
            sig_next[p - p0] = buf(flip[p - p0] ? sl.SigB : sl.SigA);
            flip[p - p0] ^= 1;
          }
        }
        QSEL_CUDA_TRY(cudaGetLastError());
      }
    }
  }
  for (int b = 0; !use_tc && b < maxT; ++b) {
    SpBatch<T, T> wb{}, vb{};
    GemmBatch<T> yb{}, sgb{};
    SweepBatch<T> mb{};
    ExtractBatch<T> xy{}, xs{};
    std::vector<int> active;
    for (int p = p0; p < p1; ++p) {
      Subdomain &sd = part(p);
      DenseSlot &sl = slot(p);
      const int tl = sd.T - 2 - b;
      if (tl < std::max(sd.lo - 1, 0)) continue;
      active.push_back(p);
      const int tg = sd.g(tl), tc = sd.cpl(tl);
      SpEntry<T, T> &we = wb.e[wb.count++];
      we.B = Dinv(p, tl);
      we.C = nullptr;
      we.Out = buf(sl.W);
      we.alpha_ptr = c->mod.off.scale_ptr(tc);
      we.val = c->mod.off.at(tc);
      we.alpha = 1.0;
      we.beta = 0.0;
      GemmEntry<T> &ye = yb.e[yb.count++];
      ye.A = sig_next[p - p0];
      ye.B = buf(sl.W);
      ye.C0 = nullptr;
      ye.C = buf(sl.Y);
      ye.alpha = 1.0;
      ye.beta = 0.0;
      const bool y_needed = (tl >= sd.lo && tl <= sd.hi) || (tl + 1 >= sd.lo && tl + 1 <= sd.hi);
      if (y_needed) {
        ExtractEntry<T> &xe = xy.e[xy.count++];
        xe.S = buf(sl.Y);
        xe.diag_out = nullptr;
        xe.sums = c->d_sums + kMaxTheta * (size_t)(sd.slot_base + sd.T + tl);
        set_sum_vals(xe, c->dmod.off, c->dmod.n, tc);
        xe.D0 = nullptr;
        xe.V = nullptr;
      }
      if (tl >= sd.lo) {
        T *sig_cur = buf(flip[p - p0] ? sl.SigB : sl.SigA);
        SpEntry<T, T> &ve = vb.e[vb.count++];
        ve.B = buf(sl.Y);
        ve.C = nullptr;
        ve.Out = buf(sl.V);
        ve.alpha_ptr = c->mod.off.scale_ptr(tc);
        ve.val = c->mod.off.at(tc);
        ve.alpha = 1.0;
        ve.beta = 0.0;
        GemmEntry<T> &ge = sgb.e[sgb.count++];
        ge.A = Dinv(p, tl);
        ge.B = buf(sl.V);
        ge.C0 = Dinv(p, tl);
        ge.C = sig_cur;
        ge.alpha = 1.0;
        ge.beta = 1.0;
        SweepEntry<T> &me = mb.e[mb.count++];
        me.A = sig_cur;
        if (tl <= sd.hi) {
          ExtractEntry<T> &xe = xs.e[xs.count++];
          xe.S = sig_cur;
          xe.diag_out = c->d_selinv + (size_t)tg * n_s;
          xe.sums = c->d_sums + kMaxTheta * (size_t)(sd.slot_base + tl);
          set_sum_vals(xe, c->dmod.diag, c->dmod.n, tg);
          // mixed path: the Takahashi diagonal accumulated in double
          xe.D0 = c->mixed ? Dinv(p, tl) : nullptr;
          xe.V = c->mixed ? buf(sl.V) : nullptr;
        }
      }
    }
    if (active.empty()) break;
    launch_sp_rowgather<T, T>(s, wb, c->pat, n_s, n_pad, n_pad, n_pad, n_pad);
    launch_gemm<T>(s, yb, n_pad, n_pad, n_pad, n_pad, n_pad, n_pad, false);
    launch_extract<T>(s, xy, c->pat, c->dmod.n, n_s, n_pad, c->d_diag_scratch);
    launch_sp_rowgather<T, T>(s, vb, c->pat, n_s, n_pad, n_pad, n_pad, n_pad);
    launch_gemm<T>(s, sgb, n_pad, n_pad, n_pad, n_pad, n_pad, n_pad, true);
    launch_mirror<T>(s, mb, n_pad);
    launch_extract<T>(s, xs, c->pat, c->dmod.n, n_s, n_pad, c->d_diag_scratch);
    for (int p : active) {
      Subdomain &sd = part(p);
      DenseSlot &sl = slot(p);
      const int tl = sd.T - 2 - b;
      if (tl >= sd.lo) {
        sig_next[p - p0] = buf(flip[p - p0] ? sl.SigB : sl.SigA);
        flip[p - p0] ^= 1;
      }
    }
    QSEL_CUDA_TRY(cudaGetLastError());
  }
  phase_mark(c, marks, 1);
  }  // stages & 1
  if (!(stages & 2)) return ok();
  // ---- RB correction: w = Q_{**}^-1 Q_{*S} x_S by the block LDL^T sweeps
  //   forward  y_0 = b_0, u_t = D_t^-1 y_t, y_{t+1} = b_{t+1} - c_t Q_s u_t
  //   backward w_{T-1} = u_{T-1}, w_t = u_t - D_t^-1 (c_t Q_s w_{t+1})
  std::vector<int> grp;
  for (int p = p0; p < p1; ++p)
    if (part(p).sep_left >= 0 || part(p).sep_right >= 0) grp.push_back(p);
  if (!grp.empty()) {
    SpBatch<double, T> bl{}, br{};
    for (int p : grp) {
      Subdomain &sd = part(p);
      DenseSlot &sl = slot(p);
      if (sd.sep_left >= 0) {
        SpEntry<double, T> &e = bl.e[bl.count++];
        e.B = c->d_X + (size_t)sd.sep_left * n_s * ld;
        e.C = nullptr;
        e.Out = buf(sl.ybuf);
        e.alpha_ptr = c->mod.off.scale_ptr(sd.sep_left);
        e.val = c->mod.off.at(sd.sep_left);
        e.alpha = 1.0;
        e.beta = 0.0;
      } else {
        QSEL_CUDA_TRY(cudaMemsetAsync(sl.ybuf, 0, svec * sizeof(T), s));
      }
      if (sd.sep_right >= 0) {
        SpEntry<double, T> &e = br.e[br.count++];
        e.B = c->d_X + (size_t)sd.sep_right * n_s * ld;
        e.C = nullptr;
        e.Out = buf(sl.bright);
        e.alpha_ptr = c->mod.off.scale_ptr(sd.sep_right - 1);
        e.val = c->mod.off.at(sd.sep_right - 1);
        e.alpha = 1.0;
        e.beta = 0.0;
      }
    }
    launch_sp_rowgather<double, T>(s, bl, c->pat, n_s, n_pad, ld, ld, ld);
    launch_sp_rowgather<double, T>(s, br, c->pat, n_s, n_pad, ld, ld, ld);
    // D_t^-1 times an n_pad x ld block: on the tensor cores in the mixed path
    // (through the transposed product, with each part's ld x n_pad scratch
    // tra / trb), else the tile GEMM
    void *bt[kMaxBatch], *pt[kMaxBatch];
    auto block_product = [&](const GemmBatch<T> &gb) -> Err {
      if constexpr (std::is_same<T, float>::value) {
        if (c->tc_passes > 0) {
          if (!launch_symm_block_tc(s, gb, reinterpret_cast<float *const *>(bt), reinterpret_cast<float *const *>(pt),
                                    n_pad, ld, c->tc_passes, c->d_err))
            return fail(QSEL_ECUDA, "tensor-core GEMM: tensor map encoding failed");
          return ok();
        }
      }
      launch_gemm<T>(s, gb, n_pad, ld, n_pad, n_pad, ld, ld, false);
      return ok();
    };
    for (int p : grp) {
      Subdomain &sd = part(p);
      DenseSlot &sl = slot(p);
      if (sd.T == 1 && sd.sep_right >= 0) launch_add<T>(s, buf(sl.ybuf), buf(sl.bright), (int64_t)svec);
    }
    for (int t = 0; t < maxT; ++t) {
      GemmBatch<T> ub{};
      SpBatch<T, T> yb{};
      for (int p : grp) {
        Subdomain &sd = part(p);
        DenseSlot &sl = slot(p);
        if (t >= sd.T) continue;
        bt[ub.count] = sl.tra;
        pt[ub.count] = sl.trb;
        GemmEntry<T> &g = ub.e[ub.count++];
        g.A = Dinv(p, t);
        g.B = buf(sl.ybuf);
        g.C0 = nullptr;
        g.C = buf(sl.wbuf) + (size_t)t * svec;
        g.alpha = 1.0;
        g.beta = 0.0;
        if (t + 1 < sd.T) {
          SpEntry<T, T> &e = yb.e[yb.count++];
          e.B = buf(sl.wbuf) + (size_t)t * svec;
          const bool add_right = (t + 1 == sd.T - 1) && sd.sep_right >= 0;
          e.C = add_right ? buf(sl.bright) : nullptr;
          e.Out = buf(sl.ybuf);
          e.alpha_ptr = c->mod.off.scale_ptr(sd.e0 + t);
          e.val = c->mod.off.at(sd.e0 + t);
          e.alpha = -1.0;
          e.beta = add_right ? 1.0 : 0.0;
        }
      }
      if (ub.count == 0) break;
      TRY(block_product(ub));
      launch_sp_rowgather<T, T>(s, yb, c->pat, n_s, n_pad, ld, ld, ld);
    }
    for (int b = 0; b < maxT; ++b) {
      SpBatch<T, T> tb{};
      GemmBatch<T> wb{};
      for (int p : grp) {
        Subdomain &sd = part(p);
        DenseSlot &sl = slot(p);
        const int t = sd.T - 2 - b;
        if (t < std::max(sd.lo - 1, 0)) continue;
        SpEntry<T, T> &e = tb.e[tb.count++];
        e.B = buf(sl.wbuf) + (size_t)(t + 1) * svec;
        e.C = nullptr;
        e.Out = buf(sl.tmp);
        e.alpha_ptr = c->mod.off.scale_ptr(sd.e0 + t);
        e.val = c->mod.off.at(sd.e0 + t);
        e.alpha = 1.0;
        e.beta = 0.0;
        bt[wb.count] = sl.tra;
        pt[wb.count] = sl.trb;
        GemmEntry<T> &g = wb.e[wb.count++];
        g.A = Dinv(p, t);
        g.B = buf(sl.tmp);
        g.C0 = buf(sl.wbuf) + (size_t)t * svec;
        g.C = buf(sl.wbuf) + (size_t)t * svec;
        g.alpha = -1.0;
        g.beta = 1.0;
      }
      if (tb.count == 0) break;
      launch_sp_rowgather<T, T>(s, tb, c->pat, n_s, n_pad, ld, ld, ld);
      TRY(block_product(wb));
    }
    CorrBatch<T> cb{};
    for (int p : grp) {
      Subdomain &sd = part(p);
      CorrEntry<T> &e = cb.e[cb.count++];
      e.w = buf(slot(p).wbuf);
      e.T_ = sd.T;
      e.lo = sd.lo;
      e.hi = sd.hi;
      e.e0 = sd.e0;
      e.corr_out = c->d_corr;
      e.corr4_out = c->d_corr4;
      e.partial = sd.partial;
    }
    launch_correction_terms<T>(s, cb, c->pat, c->dmod, n_s, n_pad, ld, c->k);
  }
  QSEL_CUDA_TRY(cudaGetLastError());
  phase_mark(c, marks, 2);
  return ok();
}

static Err run_pipeline_body(qsel_ctx *c);

static Err run_pipeline(qsel_ctx *c) {
  if (c->opt.profile_kernels) {
    c->prof.reset();
    g_prof = &c->prof;
  }
  Err e = run_pipeline_body(c);
  g_prof = nullptr;
  if (e.code == 0 && c->opt.profile_kernels) {
    static_assert(PROF_KINDS == QSEL_PROF_CLASSES, "profiler classes");
    double ms[PROF_KINDS] = {}, work[PROF_KINDS] = {};
    int64_t cnt[PROF_KINDS] = {};
    for (auto &r : c->prof.recs) {
      float t = 0.f;
      cudaEventElapsedTime(&t, r.a, r.b);
      ms[r.kind] += t;
      work[r.kind] += r.work;
      cnt[r.kind] += 1;
    }
    c->stats.gemm_ms = ms[PROF_GEMM];
    c->stats.gemm_flop = work[PROF_GEMM];
    c->stats.gemm_launches = cnt[PROF_GEMM];
    c->stats.sweep_ms = ms[PROF_SWEEP];
    c->stats.sweep_flop = work[PROF_SWEEP];
    c->stats.sweep_launches = cnt[PROF_SWEEP];
    c->stats.spmm_ms = ms[PROF_SPMM];
    c->stats.spmm_bytes = work[PROF_SPMM];
    c->stats.spmm_launches = cnt[PROF_SPMM];
    for (int q = 0; q < PROF_KINDS; ++q) {
      c->stats.class_ms[q] = ms[q];
      c->stats.class_launches[q] = cnt[q];
      c->stats.class_work[q] = work[q];
    }
  }
  return e;
}

static Err run_pipeline_body(qsel_ctx *c) {
  cudaStream_t s = c->stream;
  const int64_t launches0 = g_launch_count;
  c->phase_used = 0;
  QSEL_CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int32_t), s));
  QSEL_CUDA_TRY(cudaMemsetAsync(c->d_corr, 0, (size_t)c->n * sizeof(double), s));
  QSEL_CUDA_TRY(cudaMemsetAsync(c->d_corr4, 0, (size_t)c->n * sizeof(double), s));
  QSEL_CUDA_TRY(cudaEventRecord(c->ev[0], s));
  TRY(run_model(c));
  const bool need_samples = c->parts.size() > 1;
  c->stats.pcg_iterations = 0;
  c->stats.pcg_max_rel_residual = 0.0;
  c->lz.ran = false;
  std::vector<std::pair<cudaEvent_t, int>> marks;
  const int np = (int)c->parts.size();
  auto wave = [&](int p0, int p1, int stages) -> Err {
    return c->mixed ? run_wave<float>(c, p0, p1, marks, stages) : run_wave<double>(c, p0, p1, marks, stages);
  };
  int first = 0;   // first wave still to run in full
  if (c->mixed && !c->injected && need_samples && c->opt.sampler == QSEL_SAMPLER_PCG) {
    // The samples are needed only by the correction: the first wave's
    // factorisation and Takahashi recursion are enqueued on the context's
    // stream and run while the PCG (whose host loop synchronises only its
    // own stream) runs on pcg_stream.  Mixed form only: in FP64 both parts
    // run on the FP64 pipe, and sequential phases keep its phase times
    // (which the plain-FP64 time-to-target model scales) additive.
    QSEL_CUDA_TRY(cudaEventRecord(c->ev_fork, s));
    first = std::min(np, c->wave);
    TRY(wave(0, first, 1));
    QSEL_CUDA_TRY(cudaStreamWaitEvent(c->pcg_stream, c->ev_fork, 0));
    c->stream = c->pcg_stream;
    Err e = run_sampler(c);
    if (e.code == 0 && cudaEventRecord(c->ev[2], c->pcg_stream) != cudaSuccess)
      e = fail(QSEL_ECUDA, "event record failed");
    if (e.code == 0 && cudaEventRecord(c->ev_samples, c->pcg_stream) != cudaSuccess)
      e = fail(QSEL_ECUDA, "event record failed");
    c->stream = s;
    if (e.code) {
      cudaStreamSynchronize(s);   // leave no dense work of this call in flight
      return e;
    }
    QSEL_CUDA_TRY(cudaStreamWaitEvent(s, c->ev_samples, 0));
    TRY(wave(0, first, 2));
  } else {
    if (c->injected || !need_samples)
      QSEL_CUDA_TRY(cudaEventRecord(c->ev[1], s));
    else if (c->opt.sampler == QSEL_SAMPLER_LANCZOS)
      TRY(run_sampler_lanczos(c));
    else
      TRY(run_sampler(c));
    QSEL_CUDA_TRY(cudaEventRecord(c->ev[2], s));
  }
  for (int p0 = first; p0 < np; p0 += c->wave) TRY(wave(p0, std::min(np, p0 + c->wave), 3));
  launch_sum(s, c->d_diag, c->d_selinv, c->d_corr, c->n);
  launch_trace_combine(s, c->d_slabs, c->n_trace_slabs, c->d_sums, c->d_partials, np * corr_grid(), c->dmod,
                       c->d_traces);
  QSEL_CUDA_TRY(cudaEventRecord(c->ev[3], s));
  QSEL_CUDA_TRY(cudaStreamSynchronize(s));
  QSEL_CUDA_TRY(cudaGetLastError());
  int32_t err = 0;
  QSEL_CUDA_TRY(cudaMemcpy(&err, c->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost));
  // a timed-out GEMM leaves its output unwritten, so later pivots are
  // meaningless: the timeout is reported first
  if (err & 2) return fail(QSEL_ETIMEOUT, "a bounded device-side wait of the tensor-core GEMM gave up");
  if (err & 1) return fail(QSEL_ENOTSPD, "a pivot of a dense block factorisation was not positive");
  if (err & 8)
    return fail(QSEL_ENOCONV, "the Lanczos tridiagonal matrix could not be diagonalised or was not positive definite");
  float ms;
  auto el = [&](cudaEvent_t a, cudaEvent_t b) {
    cudaEventElapsedTime(&ms, a, b);
    return (double)ms;
  };
  c->stats.ms_rhs = (c->injected || !need_samples) ? 0.0 : el(c->ev[0], c->ev[1]);
  c->stats.ms_pcg = el(c->ev[1], c->ev[2]);
  double ph[3] = {0, 0, 0};
  for (size_t i = 1; i < marks.size(); ++i)
    if (marks[i].second >= 0) ph[marks[i].second] += el(marks[i - 1].first, marks[i].first);
  c->stats.ms_factor = ph[0];
  c->stats.ms_takahashi = ph[1];
  c->stats.ms_correction = ph[2];
  c->stats.ms_total = el(c->ev[0], c->ev[3]);
  c->stats.kernel_launches = g_launch_count - launches0;
  c->computed = true;
  return ok();
}

// The pipeline of run_pipeline_body, stream-ordered and free of host
// synchronisation and events, for capture into a graph (sampler loops as
// conditional while nodes).
static Err enqueue_pipeline_graph(qsel_ctx *c) {
  cudaStream_t s = c->stream;
  QSEL_CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int32_t), s));
  QSEL_CUDA_TRY(cudaMemsetAsync(c->d_corr, 0, (size_t)c->n * sizeof(double), s));
  QSEL_CUDA_TRY(cudaMemsetAsync(c->d_corr4, 0, (size_t)c->n * sizeof(double), s));
  TRY(run_model(c));
  if (c->parts.size() > 1) {
    TRY(run_sampler_graph(c));
  } else {
    QSEL_CUDA_TRY(cudaMemsetAsync(c->d_loop, 0, 4 * sizeof(int32_t), s));
  }
  std::vector<std::pair<cudaEvent_t, int>> marks;
  const int np = (int)c->parts.size();
  for (int p0 = 0; p0 < np; p0 += c->wave) {
    const int p1 = std::min(np, p0 + c->wave);
    if (c->mixed)
      TRY(run_wave<float>(c, p0, p1, marks));
    else
      TRY(run_wave<double>(c, p0, p1, marks));
  }
  launch_sum(s, c->d_diag, c->d_selinv, c->d_corr, c->n);
  launch_trace_combine(s, c->d_slabs, c->n_trace_slabs, c->d_sums, c->d_partials, np * corr_grid(), c->dmod,
                       c->d_traces);
  QSEL_CUDA_TRY(cudaGetLastError());
  return ok();
}

// After a replay of the graph: error flags, sampler status and statistics.
static Err collect_graph(qsel_ctx *c) {
  int32_t err = 0, loop[4] = {0, 0, 0, 0};
  double rel = 0.0;
  QSEL_CUDA_TRY(cudaMemcpy(&err, c->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost));
  QSEL_CUDA_TRY(cudaMemcpy(loop, c->d_loop, sizeof(loop), cudaMemcpyDeviceToHost));
  if (c->parts.size() > 1)
    QSEL_CUDA_TRY(cudaMemcpy(&rel, c->d_scal + 5 * c->ld, sizeof(double), cudaMemcpyDeviceToHost));
  c->stats = qsel_stats_t{};
  c->stats.pcg_iterations = loop[2];
  c->stats.pcg_max_rel_residual = rel;
  // a timed-out GEMM leaves its output unwritten, so later pivots are
  // meaningless: the timeout is reported first
  if (err & 2) return fail(QSEL_ETIMEOUT, "a bounded device-side wait of the tensor-core GEMM gave up");
  if (err & 1) return fail(QSEL_ENOTSPD, "a pivot of a dense block factorisation was not positive");
  if (loop[3] == QSEL_ENOCONV)
    return fail(QSEL_ENOCONV, "the sampler did not reach pcg_tol within its iteration limits (max relative residual " +
                                  std::to_string(rel) + ")");
  c->computed = true;
  return ok();
}

// ---------------------------------------------------------------------------
// Batch of independent models: one captured graph, one branch per model on a
// pool of streams (models placed longest-first on the least-loaded stream),
// the sampler loops device-driven.  An optional autotuner picks, per model
// size class, the block-Jacobi block and the dense tile path by timing them.
// ---------------------------------------------------------------------------
// subdomains in flight per batch model: the batch's concurrency comes from
// its many models, and two dense working sets per model keep 64 models of
// up to 64 x 64 x 128 within device memory
constexpr int kBatchSlots = 2;

struct qsel_batch {
  std::vector<qsel_ctx *> models;
  std::vector<int> stream_of;
  std::vector<double> cost;
  cudaStream_t main = nullptr;
  bool own_main = false;
  std::vector<cudaStream_t> pool;
  cudaStream_t body[2] = {nullptr, nullptr};
  cudaEvent_t fork = nullptr, t0 = nullptr, t1 = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t launches_per_replay = 0;
  double ms_last = 0.0, ms_capture = 0.0, ms_autotune = 0.0;
  bool computed = false;
  std::vector<std::array<int, 2>> tuned;   // per model: precond_block, tensor_passes
  std::string last_error;
  ~qsel_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (auto *c : models) qsel_destroy(c);
    for (auto st : pool) cudaStreamDestroy(st);
    for (auto st : body)
      if (st) cudaStreamDestroy(st);
    if (own_main && main) cudaStreamDestroy(main);
    for (auto e : join) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
  }
};

static qsel_status batch_fail(qsel_batch *b, const Err &e) {
  if (e.code && b) b->last_error = e.msg;
  return (qsel_status)e.code;
}

static Err batch_capture(qsel_batch *b) {
  const int64_t l0 = g_launch_count;
  const auto w0 = std::chrono::steady_clock::now();
  QSEL_CUDA_TRY(cudaStreamBeginCapture(b->main, cudaStreamCaptureModeRelaxed));
  Err e = ok();
  if (cudaEventRecord(b->fork, b->main) != cudaSuccess) e = fail(QSEL_ECUDA, "fork event");
  for (auto st : b->pool)
    if (e.code == 0 && cudaStreamWaitEvent(st, b->fork, 0) != cudaSuccess) e = fail(QSEL_ECUDA, "fork wait");
  std::vector<int> order(b->models.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return b->cost[x] > b->cost[y]; });
  for (int i : order) {
    if (e.code) break;
    qsel_ctx *c = b->models[i];
    c->stream = b->pool[b->stream_of[i]];
    c->body_stream[0] = b->body[0];
    c->body_stream[1] = b->body[1];
    c->graph_mode = true;
    e = enqueue_pipeline_graph(c);
    if (e.code) e.msg = "model " + std::to_string(i) + ": " + e.msg;
  }
  for (size_t j = 0; j < b->pool.size() && e.code == 0; ++j) {
    if (cudaEventRecord(b->join[j], b->pool[j]) != cudaSuccess ||
        cudaStreamWaitEvent(b->main, b->join[j], 0) != cudaSuccess)
      e = fail(QSEL_ECUDA, "join");
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(b->main, &g);
  if (e.code) {
    if (g) cudaGraphDestroy(g);
    return e;
  }
  if (ce != cudaSuccess) return cuda_fail(ce, "end of the batch capture", __FILE__, __LINE__);
  b->graph = g;
  // node priorities carry the sweep's high-priority panel stream into the graph
  QSEL_CUDA_TRY(cudaGraphInstantiate(&b->exec, g, cudaGraphInstantiateFlagUseNodePriority));
  b->ms_capture = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
  b->launches_per_replay = g_launch_count - l0;
  return ok();
}

// Modelled work of one model (dense slabs x n_pad^3 plus samples x n) for the
// stream placement.
static double model_cost(const qsel_ctx *c) {
  double slabs = 0.0;
  for (auto &sd : c->parts) slabs += sd.T;
  const double npad = (double)c->n_pad;
  return 1.10e-13 * slabs * npad * npad * npad + 1.53e-8 * (double)c->k * c->n;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

// Sizes and the option-derived settings of a new context.
static Err init_options(qsel_ctx *c, int n_s, int n_t, const qsel_options *opt, int slot_cap) {
  c->n_s = n_s;
  c->n_t = n_t;
  c->n = n_s * n_t;
  c->k = opt->n_samples;
  c->ld = round_up(opt->n_samples, kColPad);
  c->n_pad = round_up(n_s, kTile);
  c->opt = *opt;
  c->bsize = opt->precond_block == 0 ? 64 : opt->precond_block;
  c->mixed = opt->precision == QSEL_MIXED;
  if (c->mixed) {
    if (opt->tensor_passes == 0)
      c->tc_passes = tc_gemm_available() ? 3 : 0;
    else if (opt->tensor_passes > 0)
      c->tc_passes = opt->tensor_passes;
    if (c->tc_passes > 0 && !tc_gemm_available())
      return fail(QSEL_EINVAL, "tensor_passes requested but tcgen05 tensor-core GEMMs are not available on this device");
  }
  c->stream = reinterpret_cast<cudaStream_t>(opt->cuda_stream);
  c->slot_cap = slot_cap;
  return ok();
}

static qsel_status create_ctx(qsel_ctx **out, const qsel_model *model, const qsel_theta *theta,
                              const qsel_partition *partition, int32_t overlap, const qsel_options *opt,
                              int slot_cap) {
  if (!out) {
    g_create_error = "out must not be NULL";
    return QSEL_EINVAL;
  }
  *out = nullptr;
  Err e = validate(model, theta, partition, overlap, opt);
  if (e.code) {
    g_create_error = e.msg;
    return (qsel_status)e.code;
  }
  qsel_ctx *c = new (std::nothrow) qsel_ctx();
  if (!c) {
    g_create_error = "host allocation failed";
    return QSEL_ENOMEM;
  }
  c->sigma = model->sigma;
  c->obs_w = 1.0 / (model->sigma * model->sigma);
  c->theta = *theta;
  c->model_kind = opt->model;
  e = init_options(c, model->n_s, model->n_t, opt, slot_cap);
  if (e.code) {
    g_create_error = e.msg;
    delete c;
    return (qsel_status)e.code;
  }
  e = build(c, model, partition, overlap);
  if (e.code) {
    g_create_error = e.msg;
    delete c;
    return (qsel_status)e.code;
  }
  *out = c;
  return QSEL_OK;
}

qsel_status qsel_create(qsel_ctx **out, const qsel_model *model, const qsel_theta *theta,
                        const qsel_partition *partition, int32_t overlap, const qsel_options *opt) {
  return create_ctx(out, model, theta, partition, overlap, opt, kMaxBatch);
}

qsel_status qsel_set_theta(qsel_ctx *ctx, const qsel_theta *theta) {
  if (!ctx || !theta) return QSEL_EINVAL;
  if (ctx->model_kind == QSEL_MODEL_BLOCK_TRIDIAGONAL)
    return finish(ctx, fail(QSEL_EINVAL, "a user-given matrix has no theta: use qsel_set_bt_values"));
  if (!std::isfinite(theta->log_kappa) || !std::isfinite(theta->log_tau) ||
      !std::isfinite(theta->logit_rho) || std::fabs(theta->logit_rho) > 36.0)
    return finish(ctx, fail(QSEL_EINVAL, "theta must be finite with |logit rho| <= 36"));
  ctx->theta = *theta;
  ctx->computed = false;
  ctx->injected = false;
  ctx->have_rhs = false;
  return QSEL_OK;
}

// ---------------------------------------------------------------------------
// User-given block-tridiagonal precision
// ---------------------------------------------------------------------------
// Values of a user-given matrix in the SELL layout: every CSR entry of every
// block is copied to its slot (ctx->bt_slot), padding slots stay zero.
// Checks that every block is symmetric and finite.
static Err bt_upload_values(qsel_ctx *c, const double *diag_vals, const double *off_vals, const double *ddiag,
                            const double *doff) {
  const int n_t = c->n_t, n_theta = c->dmod.n;
  const int64_t nnz = (int64_t)c->bt_slot.size(), ne = c->n_ent;
  if (!diag_vals || (n_t > 1 && !off_vals) || (n_theta > 0 && (!ddiag || (n_t > 1 && !doff))))
    return fail(QSEL_EINVAL, "block value arrays must not be NULL");
  // blocks: A_t (n_t), B_t (n_t - 1), then per theta_j dA_j (n_t), dB_j (n_t - 1)
  const int64_t per_set = (int64_t)(2 * n_t - 1);
  std::vector<double> sell((size_t)(per_set * (1 + n_theta)) * ne, 0.0);
  auto put = [&](const double *src, int64_t nblk, int64_t dst_blk) -> bool {
    for (int64_t b = 0; b < nblk; ++b) {
      const double *v = src + b * nnz;
      for (int64_t q = 0; q < nnz; ++q) {
        const double w = v[c->bt_mirror[q]];
        if (!std::isfinite(v[q]) || std::fabs(v[q] - w) > 1e-12 * (std::fabs(v[q]) + std::fabs(w))) return false;
        sell[(size_t)((dst_blk + b) * ne + c->bt_slot[q])] = v[q];
      }
    }
    return true;
  };
  bool good = put(diag_vals, n_t, 0) && put(off_vals, n_t - 1, n_t);
  for (int j = 0; good && j < n_theta; ++j)
    good = put(ddiag + (int64_t)j * n_t * nnz, n_t, per_set * (1 + j)) &&
           put(doff + (int64_t)j * (n_t - 1) * nnz, n_t - 1, per_set * (1 + j) + n_t);
  if (!good) return fail(QSEL_EINVAL, "block values must be finite and every block symmetric (to 1e-12 relative)");
  QSEL_CUDA_TRY(cudaMemcpy(c->d_blk, sell.data(), sell.size() * sizeof(double), cudaMemcpyHostToDevice));
  return ok();
}

static Err build_bt(qsel_ctx *c, const qsel_bt_model *m, const qsel_partition *part, int32_t overlap) {
  const int n_s = m->n_s;
  const int64_t nnz = m->rowptr[n_s];
  // pattern rows (column -> CSR position) and the mirror position of every entry
  PatRows rows(n_s);
  std::vector<std::map<int, int64_t>> pos(n_s);
  for (int i = 0; i < n_s; ++i)
    for (int64_t q = m->rowptr[i]; q < m->rowptr[i + 1]; ++q) {
      const int j = m->col[q];
      if (pos[i].count(j)) return fail(QSEL_EINVAL, "the pattern repeats an entry");
      pos[i][j] = q;
      rows[i].emplace(j, std::array<double, 4>{(double)q, 0.0, 0.0, 0.0});
    }
  c->bt_mirror.assign((size_t)nnz, 0);
  for (int i = 0; i < n_s; ++i) {
    if (!pos[i].count(i)) return fail(QSEL_EINVAL, "every row of the pattern needs its diagonal entry");
    for (auto &kv : pos[i]) {
      auto it = pos[kv.first].find(i);
      if (it == pos[kv.first].end()) return fail(QSEL_EINVAL, "the pattern must be symmetric");
      c->bt_mirror[(size_t)kv.second] = it->second;
    }
  }
  std::vector<std::vector<double>> sell;
  TRY(build_pattern(c, rows, 1, sell));   // sell[0][slot] = CSR position (or 0 for padding)
  c->bt_slot.assign((size_t)nnz, 0);
  {
    std::vector<int32_t> col(c->n_ent);
    QSEL_CUDA_TRY(cudaMemcpy(col.data(), c->pat.col, c->n_ent * sizeof(int32_t), cudaMemcpyDeviceToHost));
    std::vector<int32_t> sp(c->pat.n_slices + 1), sw(c->pat.n_slices);
    QSEL_CUDA_TRY(cudaMemcpy(sp.data(), c->pat.slice_ptr, sp.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    QSEL_CUDA_TRY(cudaMemcpy(sw.data(), c->pat.slice_width, sw.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    for (int i = 0; i < n_s; ++i) {
      const int sl = i / kSlice, li = i % kSlice;
      int slot = 0;
      for (auto &kv : pos[i]) c->bt_slot[(size_t)kv.second] = sp[sl] + (slot++) * kSlice + li;
    }
  }
  const int n_theta = m->n_theta;
  const int64_t per_set = (int64_t)(2 * c->n_t - 1) * c->n_ent;
  TRY(c->alloc(&c->d_blk, (size_t)(per_set * (1 + n_theta))));
  c->dmod.n = n_theta;
  c->mod.diag = BlockVals{c->d_blk, c->n_ent, nullptr};
  c->mod.off = BlockVals{c->d_blk + (int64_t)c->n_t * c->n_ent, c->n_ent, nullptr};
  c->mod.obs = nullptr;
  c->mod.obs_w = 0.0;
  for (int j = 0; j < n_theta; ++j) {
    double *base = c->d_blk + per_set * (1 + j);
    c->dmod.diag[j] = BlockVals{base, c->n_ent, nullptr};
    c->dmod.off[j] = BlockVals{base + (int64_t)c->n_t * c->n_ent, c->n_ent, nullptr};
  }
  TRY(bt_upload_values(c, m->diag_vals, m->off_vals, m->ddiag_vals, m->doff_vals));
  RestInputs in;
  in.adj.resize(n_s);
  for (int i = 0; i < n_s; ++i)
    for (auto &kv : pos[i]) in.adj[i].push_back(kv.first);
  return build_rest(c, in, part, overlap);
}

qsel_status qsel_create_bt(qsel_ctx **out, const qsel_bt_model *model, const qsel_partition *partition,
                           int32_t overlap, const qsel_options *opt) {
  if (!out) {
    g_create_error = "out must not be NULL";
    return QSEL_EINVAL;
  }
  *out = nullptr;
  auto bad = [&](const std::string &msg) {
    g_create_error = "qsel_create_bt: " + msg;
    return QSEL_EINVAL;
  };
  if (!model || !opt) return bad("model and options must not be NULL");
  if (model->n_s < 1 || model->n_t < 1) return bad("n_s and n_t must be >= 1");
  if ((int64_t)model->n_s * model->n_t > (int64_t)1 << 30) return bad("n_s * n_t too large");
  if (!model->rowptr || !model->col) return bad("the pattern arrays must not be NULL");
  if (model->n_theta < 0 || model->n_theta > kMaxTheta) return bad("n_theta must be in [0, 4]");
  if (model->rowptr[0] != 0) return bad("rowptr[0] must be 0");
  for (int i = 0; i < model->n_s; ++i) {
    if (model->rowptr[i + 1] < model->rowptr[i]) return bad("rowptr must be non-decreasing");
    for (int32_t q = model->rowptr[i]; q < model->rowptr[i + 1]; ++q)
      if (model->col[q] < 0 || model->col[q] >= model->n_s) return bad("col out of range");
  }
  if (opt->sampler != QSEL_SAMPLER_LANCZOS) return bad("a user-given matrix needs sampler = QSEL_SAMPLER_LANCZOS");
  if (opt->preconditioner != QSEL_PRECOND_BLOCK_JACOBI) return bad("a user-given matrix takes block Jacobi");
  Err e = validate_options(model->n_t, partition, overlap, opt);
  if (e.code) {
    g_create_error = "qsel_create_bt: " + e.msg;
    return (qsel_status)e.code;
  }
  qsel_ctx *c = new (std::nothrow) qsel_ctx();
  if (!c) {
    g_create_error = "host allocation failed";
    return QSEL_ENOMEM;
  }
  c->model_kind = QSEL_MODEL_BLOCK_TRIDIAGONAL;
  e = init_options(c, model->n_s, model->n_t, opt, kMaxBatch);
  if (e.code == 0) e = build_bt(c, model, partition, overlap);
  if (e.code) {
    g_create_error = "qsel_create_bt: " + e.msg;
    delete c;
    return (qsel_status)e.code;
  }
  *out = c;
  return QSEL_OK;
}

qsel_status qsel_set_bt_values(qsel_ctx *ctx, const double *diag_vals, const double *off_vals,
                               const double *ddiag_vals, const double *doff_vals) {
  if (!ctx) return QSEL_EINVAL;
  if (ctx->model_kind != QSEL_MODEL_BLOCK_TRIDIAGONAL)
    return finish(ctx, fail(QSEL_EINVAL, "qsel_set_bt_values needs a context made by qsel_create_bt"));
  Err e = bt_upload_values(ctx, diag_vals, off_vals, ddiag_vals, doff_vals);
  if (e.code) return finish(ctx, e);
  ctx->computed = false;
  ctx->injected = false;
  ctx->have_rhs = false;
  return QSEL_OK;
}

qsel_status qsel_set_seed(qsel_ctx *ctx, uint64_t seed) {
  if (!ctx) return QSEL_EINVAL;
  ctx->opt.seed = seed;
  ctx->computed = false;
  ctx->injected = false;
  ctx->have_rhs = false;
  return QSEL_OK;
}

static Err ensure(qsel_ctx *c) {
  if (c->computed) return ok();
  return run_pipeline(c);
}

qsel_status qsel_diag_inv(qsel_ctx *ctx, double *diag_out, int32_t out_is_device) {
  if (!ctx) return QSEL_EINVAL;
  if (!diag_out) return finish(ctx, fail(QSEL_EINVAL, "diag_out must not be NULL"));
  Err e = ensure(ctx);
  if (e.code) return finish(ctx, e);
  cudaError_t ce = cudaMemcpyAsync(diag_out, ctx->d_diag, (size_t)ctx->n * sizeof(double),
                                   out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                   ctx->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
  if (ce != cudaSuccess) return finish(ctx, cuda_fail(ce, "copy of diag", __FILE__, __LINE__));
  return QSEL_OK;
}

static qsel_status trace_grads(qsel_ctx *ctx, double *grads_out, int n) {
  if (!ctx) return QSEL_EINVAL;
  if (!grads_out) return finish(ctx, fail(QSEL_EINVAL, "grads_out must not be NULL"));
  if (n != ctx->dmod.n)
    return finish(ctx, fail(QSEL_EINVAL, "the context has " + std::to_string(ctx->dmod.n) + " trace gradients"));
  if (ctx->n_l < 1 && ctx->parts.size() > 1)
    return finish(ctx, fail(QSEL_EINVAL, "trace gradients need overlap >= 1 when there are several parts"));
  Err e = ensure(ctx);
  if (e.code) return finish(ctx, e);
  if (n == 0) return QSEL_OK;
  cudaError_t ce = cudaMemcpyAsync(ctx->h_small, ctx->d_traces, n * sizeof(double), cudaMemcpyDeviceToHost,
                                   ctx->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
  if (ce != cudaSuccess) return finish(ctx, cuda_fail(ce, "copy of traces", __FILE__, __LINE__));
  for (int j = 0; j < n; ++j) grads_out[j] = ctx->h_small[j];
  return QSEL_OK;
}

qsel_status qsel_trace_grads(qsel_ctx *ctx, double grads_out[3]) { return trace_grads(ctx, grads_out, 3); }

qsel_status qsel_trace_grads_n(qsel_ctx *ctx, double *grads_out, int32_t n) { return trace_grads(ctx, grads_out, n); }

// ---------------------------------------------------------------------------
// Posterior mean and the gradient of the hyperparameter marginal (hyper.cu).
// ---------------------------------------------------------------------------
qsel_status qsel_set_data(qsel_ctx *ctx, const double *y_obs) {
  if (ctx && ctx->model_kind != QSEL_MODEL_SEPARABLE)
    return finish(ctx, fail(QSEL_EINVAL, "the posterior-mean and hyperparameter calls serve the separable model"));
  if (!ctx) return QSEL_EINVAL;
  qsel_ctx *c = ctx;
  if (!y_obs) return finish(c, fail(QSEL_EINVAL, "y_obs must not be NULL"));
  if (c->n_obs < 1) return finish(c, fail(QSEL_EINVAL, "the model has no observed nodes"));
  Err e = ok();
  if (!c->d_y) e = c->alloc(&c->d_y, (size_t)c->n_obs);
  if (e.code == 0) {
    const cudaError_t ce = cudaMemcpy(c->d_y, y_obs, (size_t)c->n_obs * sizeof(double), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) e = cuda_fail(ce, "copy of the data", __FILE__, __LINE__);
  }
  if (e.code) return finish(c, e);
  c->have_data = true;
  return QSEL_OK;
}

qsel_status qsel_set_covariates(qsel_ctx *ctx, int32_t n_beta, const double *Z, double beta_prec) {
  if (ctx && ctx->model_kind != QSEL_MODEL_SEPARABLE)
    return finish(ctx, fail(QSEL_EINVAL, "the posterior-mean and hyperparameter calls serve the separable model"));
  if (!ctx) return QSEL_EINVAL;
  qsel_ctx *c = ctx;
  if (n_beta < 0 || n_beta > 63 || n_beta + 1 > c->ld)
    return finish(c, fail(QSEL_EINVAL, "n_beta must lie in [0, 63]"));
  if (n_beta > 0 && (!Z || !(beta_prec > 0.0) || !std::isfinite(beta_prec)))
    return finish(c, fail(QSEL_EINVAL, "fixed effects need Z and a finite beta_prec > 0"));
  if (n_beta > 0 && c->n_obs < 1) return finish(c, fail(QSEL_EINVAL, "the model has no observed nodes"));
  Err e = ok();
  if (n_beta > 0) {
    if (!c->d_fe) e = c->alloc(&c->d_fe, (size_t)3 * 64 * 64 + 128 + 8);
    if (e.code == 0 && !c->d_fecorr) e = c->alloc(&c->d_fecorr, (size_t)c->n);
    if (e.code == 0 && !c->d_obs_nodes) {
      // the observed nodes in increasing order (host index bookkeeping)
      std::vector<int32_t> nodes;
      nodes.reserve(c->n_obs);
      std::vector<uint8_t> mask(c->n);
      const cudaError_t ce = cudaMemcpy(mask.data(), c->d_obs, c->n, cudaMemcpyDeviceToHost);
      if (ce != cudaSuccess) e = cuda_fail(ce, "copy of the observation mask", __FILE__, __LINE__);
      for (int r = 0; e.code == 0 && r < c->n; ++r)
        if (mask[r]) nodes.push_back(r);
      if (e.code == 0) e = upload(c, &c->d_obs_nodes, nodes);
    }
    if (e.code == 0 && !c->d_Z) e = c->alloc(&c->d_Z, (size_t)c->n_obs * 63);   // room for any n_beta
    if (e.code == 0) {
      const cudaError_t ce =
          cudaMemcpy(c->d_Z, Z, (size_t)c->n_obs * n_beta * sizeof(double), cudaMemcpyHostToDevice);
      if (ce != cudaSuccess) e = cuda_fail(ce, "copy of the covariates", __FILE__, __LINE__);
    }
  }
  if (e.code) return finish(c, e);
  c->n_beta = n_beta;
  c->beta_prec = n_beta > 0 ? beta_prec : 1.0;
  return QSEL_OK;
}

// mu = Q^-1 A^T y / sigma^2 with the sampler's solver, into d_mu; leaves mu
// in column 0 of d_X (the other columns zero).  The sampler's right-hand
// sides and samples are overwritten; the statistics of the last
// qsel_diag_inv are kept.
static Err compute_mean(qsel_ctx *c) {
  if (!c->have_data) return fail(QSEL_ESTATE, "no data: call qsel_set_data first");
  cudaStream_t s = c->stream;
  if (!c->d_mu) TRY(c->alloc(&c->d_mu, (size_t)c->n));
  TRY(run_model(c));
  QSEL_CUDA_TRY(cudaMemsetAsync(c->d_R, 0, (size_t)c->n * c->ld * sizeof(double), s));
  const double inv_s2 = 1.0 / (c->sigma * c->sigma);
  launch_data_rhs(s, c->d_R, c->ld, c->d_obs, c->d_obs_index, c->d_y, c->n, inv_s2);
  if (c->n_beta > 0) launch_fe_rhs(s, c->d_R, c->ld, c->d_obs_nodes, c->d_Z, c->n_obs, c->n_beta, inv_s2);
  c->have_rhs = false;
  c->injected = false;   // injected samples, if any, are overwritten: later runs sample afresh
  const int it0 = c->stats.pcg_iterations;
  const double rel0 = c->stats.pcg_max_rel_residual;
  Err e = solve_R(c);
  c->stats.pcg_iterations = it0;
  c->stats.pcg_max_rel_residual = rel0;
  TRY(e);
  if (c->n_beta > 0) {
    // fixed effects: S, m over the observed nodes, S^-1 and mu_beta, then
    // mu_u = X[:, 0] - W mu_beta (written back to X[:, 0]) and diag(W S^-1 W^T)
    QSEL_CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int32_t), s));
    launch_fe_schur(s, c->d_X, c->ld, c->d_obs_nodes, c->d_Z, c->d_y, c->n_obs, c->n_beta, inv_s2, c->beta_prec,
                    c->fe_S(), c->fe_m());
    launch_fe_solve(s, c->fe_S(), c->fe_m(), c->n_beta, c->fe_Sinv(), c->fe_mu(), c->d_err);
    launch_fe_mean(s, c->d_X, c->ld, c->n, c->n_beta, c->fe_mu(), c->fe_Sinv(), c->d_mu, c->d_fecorr);
    QSEL_CUDA_TRY(cudaMemcpyAsync(c->h_counters, c->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    QSEL_CUDA_TRY(cudaStreamSynchronize(s));
    if (c->h_counters[0] & 1) return fail(QSEL_ENOTSPD, "the Schur complement of the fixed effects was not positive");
  } else {
    QSEL_CUDA_TRY(cudaMemcpy2DAsync(c->d_mu, sizeof(double), c->d_X, (size_t)c->ld * sizeof(double), sizeof(double),
                                    (size_t)c->n, cudaMemcpyDeviceToDevice, s));
  }
  QSEL_CUDA_TRY(cudaGetLastError());
  return ok();
}

qsel_status qsel_posterior_mean(qsel_ctx *ctx, double *mu_out, int32_t out_is_device) {
  if (!ctx) return QSEL_EINVAL;
  qsel_ctx *c = ctx;
  if (!mu_out) return finish(c, fail(QSEL_EINVAL, "mu_out must not be NULL"));
  Err e = compute_mean(c);
  if (e.code) return finish(c, e);
  cudaError_t ce = cudaMemcpyAsync(mu_out, c->d_mu, (size_t)c->n * sizeof(double),
                                   out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
  if (ce != cudaSuccess) return finish(c, cuda_fail(ce, "copy of the posterior mean", __FILE__, __LINE__));
  return QSEL_OK;
}

qsel_status qsel_fixed_effects(qsel_ctx *ctx, double *mu_beta_out, double *var_beta_out, double *var_u_corr_out,
                               int32_t corr_is_device) {
  if (!ctx) return QSEL_EINVAL;
  qsel_ctx *c = ctx;
  if (c->n_beta < 1) return finish(c, fail(QSEL_ESTATE, "no fixed effects: call qsel_set_covariates first"));
  Err e = compute_mean(c);
  if (e.code) return finish(c, e);
  const int nb = c->n_beta;
  cudaStream_t s = c->stream;
  cudaError_t ce = cudaSuccess;
  std::vector<double> mu(nb), sinv((size_t)nb * nb);
  ce = cudaMemcpyAsync(mu.data(), c->fe_mu(), nb * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(sinv.data(), c->fe_Sinv(), (size_t)nb * nb * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess && var_u_corr_out)
    ce = cudaMemcpyAsync(var_u_corr_out, c->d_fecorr, (size_t)c->n * sizeof(double),
                         corr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return finish(c, cuda_fail(ce, "copy of the fixed effects", __FILE__, __LINE__));
  if (mu_beta_out) std::copy(mu.begin(), mu.end(), mu_beta_out);
  if (var_beta_out) std::copy(sinv.begin(), sinv.end(), var_beta_out);
  return QSEL_OK;
}

qsel_status qsel_loglik_grad(qsel_ctx *ctx, double grad_out[3], double terms_out[9]) {
  if (!ctx) return QSEL_EINVAL;
  qsel_ctx *c = ctx;
  if (!grad_out) return finish(c, fail(QSEL_EINVAL, "grad_out must not be NULL"));
  if (c->n_l < 1 && c->parts.size() > 1)
    return finish(c, fail(QSEL_EINVAL, "trace gradients need overlap >= 1 when there are several parts"));
  if (!c->have_data) return finish(c, fail(QSEL_ESTATE, "no data: call qsel_set_data first"));
  // tr(Q^-1 dQ_j) of the current theta (the RBMC estimate), then mu
  Err e = ensure(c);
  if (e.code == 0) e = compute_mean(c);
  if (e.code) return finish(c, e);
  cudaStream_t s = c->stream;
  const int n_pad = c->n_pad;
  if (!c->d_hyp) e = c->alloc(&c->d_hyp, 15);
  if (e.code == 0 && !c->d_K) e = c->alloc(&c->d_K, (size_t)n_pad * n_pad);
  if (e.code == 0 && !c->d_Kp) e = c->alloc(&c->d_Kp, 64 * 64);
  if (e.code == 0 && !c->d_Ku) e = c->alloc(&c->d_Ku, (size_t)n_pad * 64);
  if (e.code == 0 && !c->d_Kv) e = c->alloc(&c->d_Kv, (size_t)n_pad * 64);
  if (e.code) return finish(c, e);
  // mu^T dQ_j mu: dQ_j mu by the block-tridiagonal SpMM with the derivative's
  // coefficients (no observation term), its per-column dot partials with mu
  BtSpmmArgs<double> a{};
  a.pat = c->pat;
  a.n_s = c->n_s;
  a.n_t = c->n_t;
  a.ld = c->ld;
  a.x = c->d_X;
  a.y = c->d_q;
  a.dot_partial = c->d_pa;
  a.tmp = c->d_z1;
  for (int j = 0; j < 3; ++j) {
    a.m.diag = c->dmod.diag[j];   // dQ_j: no observation term
    a.m.off = c->dmod.off[j];
    launch_bt_spmm<double>(s, a);
    launch_column_sum(s, c->d_pa, bt_spmm_grid(c->n), c->ld, 0, c->d_hyp + j);
    // fixed effects: tr(S^-1 W^T dQ_j W) from the same product
    if (c->n_beta > 0)
      launch_fe_schur_trace(s, c->d_X, c->d_q, c->ld, c->n, c->n_beta, c->fe_Sinv(), c->fe_C(), c->fe_trace() + j);
  }
  // tr(K^-1 C) for the prior's log-determinant: K^-1 by the blocked sweep
  cudaError_t ce = cudaMemsetAsync(c->d_err, 0, sizeof(int32_t), s);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(c->d_K, 0, (size_t)n_pad * n_pad * sizeof(double), s);
  if (ce != cudaSuccess) return finish(c, cuda_fail(ce, "memset", __FILE__, __LINE__));
  launch_dense_K(s, c->d_K, n_pad, c->pat, c->d_c_pat, c->d_g_pat, c->d_theta, c->n_s);
  SweepBatch<double> kb{};
  kb.count = 1;
  kb.e[0].A = c->d_K;
  kb.e[0].P = c->d_Kp;
  kb.e[0].U = c->d_Ku;
  kb.e[0].V = c->d_Kv;
  spd_inverse<double>(s, kb, n_pad, c->d_err, 0);
  launch_loglik_combine(s, c->d_K, n_pad, c->d_cdiag, c->n_s, c->n_t, c->d_theta, c->d_traces,
                        c->n_beta > 0 ? c->fe_trace() : nullptr, c->d_hyp, c->d_hyp + 3, c->d_hyp + 6);
  int32_t err = 0;
  ce = cudaMemcpyAsync(c->h_small, c->d_hyp + 3, 12 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(c->h_counters, c->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce == cudaSuccess) ce = cudaGetLastError();
  if (ce != cudaSuccess) return finish(c, cuda_fail(ce, "hyperparameter gradient", __FILE__, __LINE__));
  err = c->h_counters[0];
  if (err & 1) return finish(c, fail(QSEL_ENOTSPD, "K = kappa^2 C + G was not positive definite"));
  for (int j = 0; j < 3; ++j) grad_out[j] = c->h_small[j];
  if (terms_out)
    for (int j = 0; j < 9; ++j) terms_out[j] = c->h_small[3 + j];
  return QSEL_OK;
}

qsel_status qsel_stats(const qsel_ctx *ctx, qsel_stats_t *stats) {
  if (!ctx || !stats) return QSEL_EINVAL;
  *stats = ctx->stats;
  return QSEL_OK;
}

static Err copy_rows(double *dst_host, int ldh, const double *src_dev, int n, int ld, int k,
                     cudaStream_t s, bool to_device) {
  const size_t spitch = (size_t)ld * sizeof(double), dpitch = (size_t)ldh * sizeof(double);
  if (!to_device)
    QSEL_CUDA_TRY(cudaMemcpy2DAsync(dst_host, dpitch, src_dev, spitch, (size_t)k * sizeof(double), n,
                                    cudaMemcpyDeviceToHost, s));
  QSEL_CUDA_TRY(cudaStreamSynchronize(s));
  return ok();
}

qsel_status qsel_debug_set_samples(qsel_ctx *ctx, const double *X, int32_t ld) {
  if (!ctx) return QSEL_EINVAL;
  if (!X || ld < ctx->k) return finish(ctx, fail(QSEL_EINVAL, "X must not be NULL and ld >= n_samples"));
  cudaStream_t s = ctx->stream;
  cudaError_t ce = cudaMemsetAsync(ctx->d_X, 0, (size_t)ctx->n * ctx->ld * sizeof(double), s);
  if (ce == cudaSuccess)
    ce = cudaMemcpy2DAsync(ctx->d_X, (size_t)ctx->ld * sizeof(double), X, (size_t)ld * sizeof(double),
                           (size_t)ctx->k * sizeof(double), ctx->n, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return finish(ctx, cuda_fail(ce, "upload of samples", __FILE__, __LINE__));
  ctx->injected = true;
  ctx->have_rhs = false;
  ctx->computed = false;
  return QSEL_OK;
}

qsel_status qsel_debug_get_samples(const qsel_ctx *ctx, double *X, int32_t ld) {
  if (!ctx) return QSEL_EINVAL;
  qsel_ctx *c = const_cast<qsel_ctx *>(ctx);
  if (!X || ld < ctx->k) return finish(c, fail(QSEL_EINVAL, "X must not be NULL and ld >= n_samples"));
  if (!ctx->computed && !ctx->injected) return finish(c, fail(QSEL_ESTATE, "no samples yet"));
  Err e = copy_rows(X, ld, ctx->d_X, ctx->n, ctx->ld, ctx->k, ctx->stream, false);
  return finish(c, e);
}

qsel_status qsel_debug_get_rhs(const qsel_ctx *ctx, double *R, int32_t ld) {
  if (!ctx) return QSEL_EINVAL;
  qsel_ctx *c = const_cast<qsel_ctx *>(ctx);
  if (!R || ld < ctx->k) return finish(c, fail(QSEL_EINVAL, "R must not be NULL and ld >= n_samples"));
  if (!ctx->have_rhs) return finish(c, fail(QSEL_ESTATE, "no right-hand sides: the samples were injected or not yet drawn"));
  Err e = copy_rows(R, ld, ctx->d_R, ctx->n, ctx->ld, ctx->k, ctx->stream, false);
  return finish(c, e);
}

qsel_status qsel_debug_get_selinv_diag(const qsel_ctx *ctx, double *diag_out) {
  if (!ctx) return QSEL_EINVAL;
  qsel_ctx *c = const_cast<qsel_ctx *>(ctx);
  if (!diag_out) return finish(c, fail(QSEL_EINVAL, "diag_out must not be NULL"));
  if (!ctx->computed) return finish(c, fail(QSEL_ESTATE, "pipeline has not run"));
  cudaError_t ce = cudaMemcpyAsync(diag_out, ctx->d_selinv, (size_t)ctx->n * sizeof(double),
                                   cudaMemcpyDeviceToHost, ctx->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
  if (ce != cudaSuccess) return finish(c, cuda_fail(ce, "copy of selected inverse", __FILE__, __LINE__));
  return QSEL_OK;
}

qsel_status qsel_error_estimate(qsel_ctx *ctx, double *part_err, double *global_err) {
  if (!ctx) return QSEL_EINVAL;
  if (ctx->k < 2) return finish(ctx, fail(QSEL_EINVAL, "the error estimate needs n_samples >= 2"));
  if (!ctx->computed) return finish(ctx, fail(QSEL_ESTATE, "pipeline has not run"));
  const int np = (int)ctx->parts.size();
  launch_part_error_sums(ctx->stream, ctx->d_corr, ctx->d_corr4, ctx->d_diag, ctx->d_slab_start, np, ctx->n_s,
                         ctx->k, ctx->d_part_sums);
  std::vector<double> sums(np);
  cudaError_t ce = cudaMemcpyAsync(sums.data(), ctx->d_part_sums, np * sizeof(double), cudaMemcpyDeviceToHost,
                                   ctx->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
  if (ce != cudaSuccess) return finish(ctx, cuda_fail(ce, "error estimate", __FILE__, __LINE__));
  double tot = 0.0;
  for (int p = 0; p < np; ++p) {
    const double rows = (double)(ctx->slab_start[p + 1] - ctx->slab_start[p]) * ctx->n_s;
    if (part_err) part_err[p] = std::sqrt(sums[p] / rows);
    tot += sums[p];
  }
  if (global_err) *global_err = std::sqrt(tot / (double)ctx->n);
  return QSEL_OK;
}

// Time distance (capped at 16) from slab t of part [s0, s1) to the nearest
// separator slab of the part extended by `overlap` slabs; 16 when it has none.
static float sep_distance(int t, int s0, int s1, int overlap, int n_t) {
  const int e0 = std::max(0, s0 - overlap), e1 = std::min(n_t, s1 + overlap);
  float d = 16.f;
  if (e0 > 0) d = std::min(d, (float)(t - (e0 - 1)));
  if (e1 < n_t) d = std::min(d, (float)(e1 - t));
  return d;
}

static Err cv_features_sepd(qsel_ctx *c, const std::vector<float> &sepd, float *F_dev);

// Control-variate features of the current theta with every part extended by
// `overlap` slabs (see qsel.h for the definition).
static Err cv_features(qsel_ctx *c, int overlap, float *F_dev) {
  const int np = (int)c->parts.size();
  std::vector<float> sepd(c->n_t, 16.f);
  for (int p = 0; p < np; ++p)
    for (int t = c->slab_start[p]; t < c->slab_start[p + 1]; ++t)
      sepd[t] = sep_distance(t, c->slab_start[p], c->slab_start[p + 1], overlap, c->n_t);
  return cv_features_sepd(c, sepd, F_dev);
}

// Features with the given separator distance of every slab.
static Err cv_features_sepd(qsel_ctx *c, const std::vector<float> &sepd, float *F_dev) {
  TRY(run_model(c));
  QSEL_CUDA_TRY(cudaMemcpyAsync(c->d_sepd, sepd.data(), c->n_t * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  const double th[3] = {c->theta.log_kappa, c->theta.log_tau, c->theta.logit_rho};
  launch_cv_features(c->stream, c->pat, c->mod, c->n_s, c->n_t, c->d_sepd,
                     c->d_bnd, th, F_dev);
  QSEL_CUDA_TRY(cudaStreamSynchronize(c->stream));   // sepd is a host vector
  QSEL_CUDA_TRY(cudaGetLastError());
  return ok();
}

qsel_status qsel_cv_features(qsel_ctx *ctx, int32_t overlap, float *F_dev) {
  if (!ctx) return QSEL_EINVAL;
  if (!F_dev || overlap < 0) return finish(ctx, fail(QSEL_EINVAL, "F_dev must not be NULL and overlap >= 0"));
  return finish(ctx, cv_features(ctx, overlap, F_dev));
}

qsel_status qsel_cv_targets(qsel_ctx *const *ctxs, int32_t count, float *y_dev) {
  if (!ctxs || count < 1 || count > kCvMaxTargets || !y_dev) {
    set_context_free_error("qsel_cv_targets: need 1..8 contexts and a target buffer");
    return QSEL_EINVAL;
  }
  CvTargetArgs a{};
  a.count = count;
  for (int q = 0; q < count; ++q) {
    if (!ctxs[q] || !ctxs[q]->computed || ctxs[q]->n != ctxs[0]->n) {
      set_context_free_error("qsel_cv_targets: every context must have run on a model of the same size");
      return ctxs[q] ? QSEL_ESTATE : QSEL_EINVAL;
    }
    a.corr[q] = ctxs[q]->d_corr;
  }
  qsel_ctx *c = ctxs[0];
  launch_cv_targets(c->stream, a, c->d_selinv, c->n, y_dev);
  cudaError_t ce = cudaStreamSynchronize(c->stream);
  if (ce != cudaSuccess) return finish(c, cuda_fail(ce, "control-variate targets", __FILE__, __LINE__));
  return QSEL_OK;
}

qsel_status qsel_cv_plan(qsel_ctx *ctx, const qsel_cv *cv, const qsel_cv_plan_options *o, qsel_cv_plan_t *plan) {
  if (!ctx) return QSEL_EINVAL;
  if (!cv || !o || !plan || !plan->part_overlap) return finish(ctx, fail(QSEL_EINVAL, "NULL argument"));
  if (!(o->target_rel_err > 0.0) || o->max_overlap < 1 || o->min_samples < 32 || o->max_samples > 512 ||
      o->min_samples > o->max_samples)
    return finish(ctx, fail(QSEL_EINVAL, "plan options: target > 0, max_overlap >= 1, 32 <= min <= max <= 512"));
  qsel_ctx *c = ctx;
  const int n_t = c->n_t;
  if (o->n_part_counts < 0 || (o->n_part_counts > 0 && !o->part_counts))
    return finish(c, fail(QSEL_EINVAL, "plan options: part_counts must hold n_part_counts entries"));
  for (int q = 0; q < o->n_part_counts; ++q)
    if (o->part_counts[q] < 1 || o->part_counts[q] > n_t)
      return finish(c, fail(QSEL_EINVAL, "plan options: every part count must be in 1..n_t"));
  if (!c->d_cv_F) {
    Err e = c->alloc(&c->d_cv_F, (size_t)c->n * QSEL_CV_FEATURES);
    if (e.code == 0) e = c->alloc(&c->d_cv_y, (size_t)c->n);
    if (e.code == 0) e = c->alloc(&c->d_cv_sums, (size_t)n_t);
    if (e.code == 0) {
      std::vector<int32_t> every(n_t + 1);
      for (int t = 0; t <= n_t; ++t) every[t] = t;
      e = upload(c, &c->d_cv_slabs, every);
    }
    if (e.code) return finish(c, e);
  }
  // S[d][t]: sum over the nodes of slab t of the predicted (c_i / v_i)^2 when
  // the slab lies d slabs from the nearest separator (d = 1..16, the feature's
  // cap).  Every plan below is a lookup in this table.
  constexpr int kMaxD = 16;
  std::vector<double> S((size_t)(kMaxD + 1) * n_t, 0.0);
  for (int d = 1; d <= kMaxD; ++d) {
    Err e = cv_features_sepd(c, std::vector<float>(n_t, (float)d), c->d_cv_F);
    if (e.code) return finish(c, e);
    qsel_status st = qsel_cv_predict(cv, c->d_cv_F, c->d_cv_y, c->n);
    if (st) return finish(c, fail(st, std::string("planner prediction: ") + qsel_last_error(nullptr)));
    launch_cv_part_m2(c->stream, c->d_cv_y, c->d_cv_slabs, n_t, c->n_s, c->d_cv_sums);
    cudaError_t ce = cudaMemcpyAsync(S.data() + (size_t)d * n_t, c->d_cv_sums, n_t * sizeof(double),
                                     cudaMemcpyDeviceToHost, c->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
    if (ce != cudaSuccess) return finish(c, cuda_fail(ce, "planner reduction", __FILE__, __LINE__));
  }
  const double cp = o->cost_pcg > 0 ? o->cost_pcg : 1.53e-8;
  const double cd = o->cost_dense > 0 ? o->cost_dense : 1.10e-13;
  const double cc = o->cost_corr > 0 ? o->cost_corr : 2.2e-13;
  const double npad = (double)c->n_pad;
  const double single_cost = cd * (double)n_t * npad * npad * npad;
  // candidate partitions: balanced ones of the requested part counts, or the
  // context's own
  std::vector<std::vector<int>> cands;
  if (o->n_part_counts > 0) {
    for (int q = 0; q < o->n_part_counts; ++q) {
      const int np = o->part_counts[q];
      std::vector<int> ss(np + 1, 0);
      for (int p = 0; p < np; ++p) ss[p + 1] = ss[p] + n_t / np + (p < n_t % np ? 1 : 0);
      cands.push_back(ss);
    }
  } else {
    cands.push_back(c->slab_start);
  }
  struct Choice {
    double cost = -1.0;
    int k = 0;
    std::vector<int> ss, nl;
    std::vector<double> err;
  };
  Choice best, fallback;
  for (const auto &ss : cands) {
    const int np = (int)ss.size() - 1;
    if (np == 1) {   // exact one-part form: no separator, no samples
      if (best.cost < 0 || single_cost < best.cost) {
        best.cost = single_cost;
        best.k = 0;
        best.ss = ss;
        best.nl.assign(1, 0);
        best.err.assign(1, 0.0);
      }
      continue;
    }
    // m2[nl][p]: mean over Omega_p of the predicted squared ratio
    std::vector<std::vector<double>> m2(o->max_overlap + 1, std::vector<double>(np, 0.0));
    for (int nl = 1; nl <= o->max_overlap; ++nl)
      for (int p = 0; p < np; ++p) {
        const int s0 = ss[p], s1 = ss[p + 1];
        if (std::max(0, s0 - nl) == 0 && std::min(n_t, s1 + nl) == n_t) continue;   // no separator: exact
        double acc = 0.0;
        for (int t = s0; t < s1; ++t) {
          const int d = (int)sep_distance(t, s0, s1, nl, n_t);
          acc += S[(size_t)d * n_t + t];
        }
        m2[nl][p] = acc / ((double)(s1 - s0) * c->n_s);
      }
    auto slabs = [&](int p, int nl) { return std::min(n_t, ss[p + 1] + nl) - std::max(0, ss[p] - nl); };
    auto err = [&](int p, int nl, int k) { return std::sqrt(2.0 * m2[nl][p] / k); };
    for (int k = round_up(o->min_samples, 32); k <= o->max_samples; k += 32) {
      double cost = cp * (double)k * c->n;
      std::vector<int> pick(np, -1);
      bool feasible = true;
      for (int p = 0; p < np && feasible; ++p) {
        for (int nl = 1; nl <= o->max_overlap && pick[p] < 0; ++nl)
          if (err(p, nl, k) <= o->target_rel_err) pick[p] = nl;
        feasible = pick[p] > 0;
        if (feasible) cost += slabs(p, pick[p]) * (cd * npad * npad * npad + cc * k * npad * npad);
      }
      if (feasible && (best.cost < 0 || cost < best.cost)) {
        best.cost = cost;
        best.k = k;
        best.ss = ss;
        best.nl = pick;
        best.err.resize(np);
        for (int p = 0; p < np; ++p) best.err[p] = err(p, pick[p], k);
      }
    }
    if (fallback.cost < 0) {   // best effort at the limits, first candidate
      fallback.k = o->max_samples;
      fallback.cost = cp * (double)fallback.k * c->n;
      fallback.ss = ss;
      fallback.nl.assign(np, o->max_overlap);
      fallback.err.resize(np);
      for (int p = 0; p < np; ++p) {
        fallback.cost += slabs(p, o->max_overlap) * (cd * npad * npad * npad + cc * fallback.k * npad * npad);
        fallback.err[p] = err(p, o->max_overlap, fallback.k);
      }
    }
  }
  plan->feasible = best.cost >= 0 ? 1 : 0;
  const Choice &ch = best.cost >= 0 ? best : fallback;
  const int np = (int)ch.ss.size() - 1;
  plan->n_samples = ch.k;
  plan->predicted_cost = ch.cost;
  plan->single_part_cost = single_cost;
  plan->n_parts = np;
  plan->predicted_err = 0.0;
  for (int p = 0; p < np; ++p) {
    plan->part_overlap[p] = ch.nl[p];
    if (plan->part_pred_err) plan->part_pred_err[p] = ch.err[p];
    plan->predicted_err = std::max(plan->predicted_err, ch.err[p]);
  }
  if (plan->slab_start)
    for (int p = 0; p <= np; ++p) plan->slab_start[p] = ch.ss[p];
  return QSEL_OK;
}

qsel_status qsel_create_batch(qsel_batch **out, int32_t n_models, const qsel_model *models,
                              const qsel_theta *thetas, const qsel_partition *partitions, const int32_t *overlaps,
                              const qsel_options *opt, int32_t n_streams, int32_t autotune) {
  if (!out) {
    g_create_error = "out must not be NULL";
    return QSEL_EINVAL;
  }
  *out = nullptr;
  if (n_models < 1 || !models || !thetas || !partitions || !overlaps || !opt || n_streams < 1 || n_streams > 64) {
    g_create_error = "qsel_create_batch: n_models >= 1, non-NULL arrays and 1 <= n_streams <= 64 required";
    return QSEL_EINVAL;
  }
  if (opt->profile_kernels || opt->part_overlap || opt->sampler != QSEL_SAMPLER_PCG ||
      opt->preconditioner != QSEL_PRECOND_BLOCK_JACOBI) {
    g_create_error = "qsel_create_batch: profile_kernels, part_overlap, the Lanczos sampler and the Kronecker "
                     "preconditioner are not available in a batch";
    return QSEL_EINVAL;
  }
  for (int i = 0; i < n_models; ++i) {
    Err e = validate(&models[i], &thetas[i], &partitions[i], overlaps[i], opt);
    if (e.code) {
      g_create_error = "model " + std::to_string(i) + ": " + e.msg;
      return (qsel_status)e.code;
    }
  }
  qsel_batch *b = new (std::nothrow) qsel_batch();
  if (!b) {
    g_create_error = "host allocation failed";
    return QSEL_ENOMEM;
  }
  auto bail = [&](qsel_status st, const std::string &m) {
    g_create_error = m;
    delete b;
    return st;
  };
  b->tuned.assign(n_models, {opt->precond_block, opt->tensor_passes});
  if (autotune) {
    // per grid size (n_s): time every (block-Jacobi block, dense path) pair on
    // the smallest model of that size, keep the fastest
    const auto w0 = std::chrono::steady_clock::now();
    std::map<int, int> rep;
    for (int i = 0; i < n_models; ++i) {
      auto it = rep.find(models[i].n_s);
      if (it == rep.end() || (int64_t)models[i].n_t * partitions[i].n_parts <
                                 (int64_t)models[it->second].n_t * partitions[it->second].n_parts)
        rep[models[i].n_s] = i;
    }
    std::vector<std::array<int, 2>> cands;
    for (int pb : {16, 32, 64}) {
      if (opt->precision == QSEL_MIXED && tc_gemm_available()) {
        cands.push_back({pb, 3});
        cands.push_back({pb, -1});
      } else {
        cands.push_back({pb, 0});
      }
    }
    std::map<int, std::array<int, 2>> best;
    for (auto &kv : rep) {
      // one context per size (block-Jacobi storage for the largest block);
      // the candidates switch its block size and dense path between runs
      const int i = kv.second;
      qsel_options o = *opt;
      o.precond_block = 64;
      o.tensor_passes = cands[0][1];
      o.seed = opt->seed + (uint64_t)i;
      qsel_ctx *t = nullptr;
      qsel_status st = create_ctx(&t, &models[i], &thetas[i], &partitions[i], overlaps[i], &o, kBatchSlots);
      if (st) return bail(st, "autotune: " + g_create_error);
      Err e = run_pipeline(t);                       // warm-up
      double best_ms = 1e300;
      for (auto cd : cands) {
        if (e.code) break;
        t->bsize = cd[0];
        if (t->mixed) t->tc_passes = cd[1] > 0 ? cd[1] : 0;
        t->computed = false;
        e = run_pipeline(t);
        const double ms = t->stats.ms_total;
        if (e.code == 0 && ms < best_ms) {
          best_ms = ms;
          best[kv.first] = cd;
        }
      }
      qsel_destroy(t);
      if (e.code) return bail((qsel_status)e.code, "autotune: " + e.msg);
    }
    for (int i = 0; i < n_models; ++i) b->tuned[i] = best[models[i].n_s];
    b->ms_autotune = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
  }
  if (opt->cuda_stream) {
    b->main = reinterpret_cast<cudaStream_t>(opt->cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) != cudaSuccess)
      return bail(QSEL_ECUDA, "stream creation failed");
    b->own_main = true;
  }
  b->pool.resize(std::min(n_streams, n_models));
  for (auto &st : b->pool)
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
      return bail(QSEL_ECUDA, "stream creation failed");
  for (auto &st : b->body)
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
      return bail(QSEL_ECUDA, "stream creation failed");
  b->join.resize(b->pool.size());
  for (auto &e : b->join)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return bail(QSEL_ECUDA, "event");
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&b->t0) != cudaSuccess || cudaEventCreate(&b->t1) != cudaSuccess)
    return bail(QSEL_ECUDA, "event creation failed");
  for (int i = 0; i < n_models; ++i) {
    qsel_options o = *opt;
    o.precond_block = b->tuned[i][0];
    o.tensor_passes = b->tuned[i][1];
    o.seed = opt->seed + (uint64_t)i;
    o.cuda_stream = nullptr;
    qsel_ctx *c = nullptr;
    qsel_status st = create_ctx(&c, &models[i], &thetas[i], &partitions[i], overlaps[i], &o, kBatchSlots);
    if (st) return bail(st, "model " + std::to_string(i) + ": " + g_create_error);
    b->models.push_back(c);
    b->cost.push_back(model_cost(c));
  }
  // longest first onto the least-loaded stream
  std::vector<int> order(n_models);
  for (int i = 0; i < n_models; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return b->cost[x] > b->cost[y]; });
  std::vector<double> load(b->pool.size(), 0.0);
  b->stream_of.assign(n_models, 0);
  for (int i : order) {
    const int j = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->stream_of[i] = j;
    load[j] += b->cost[i];
  }
  *out = b;
  return QSEL_OK;
}

qsel_status qsel_batch_run(qsel_batch *b) {
  if (!b) return QSEL_EINVAL;
  if (!b->exec) {
    Err e = batch_capture(b);
    if (e.code) return batch_fail(b, e);
  }
  cudaError_t ce = cudaEventRecord(b->t0, b->main);
  if (ce == cudaSuccess) ce = cudaGraphLaunch(b->exec, b->main);
  if (ce == cudaSuccess) ce = cudaEventRecord(b->t1, b->main);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->main);
  if (ce != cudaSuccess) return batch_fail(b, cuda_fail(ce, "batch graph launch", __FILE__, __LINE__));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, b->t0, b->t1);
  b->ms_last = ms;
  for (size_t i = 0; i < b->models.size(); ++i) {
    Err e = collect_graph(b->models[i]);
    if (e.code) {
      e.msg = "model " + std::to_string(i) + ": " + e.msg;
      b->models[i]->last_error = e.msg;
      return batch_fail(b, e);
    }
  }
  b->computed = true;
  return QSEL_OK;
}

qsel_status qsel_batch_set_theta(qsel_batch *b, int32_t model, const qsel_theta *theta) {
  if (!b) return QSEL_EINVAL;
  if (model < 0 || model >= (int)b->models.size() || !theta)
    return batch_fail(b, fail(QSEL_EINVAL, "model index out of range or theta NULL"));
  qsel_ctx *c = b->models[model];
  qsel_status st = qsel_set_theta(c, theta);
  if (st) return batch_fail(b, fail(st, c->last_error));
  // the captured copy reads the pinned host theta at every replay
  c->h_theta[0] = theta->log_kappa;
  c->h_theta[1] = theta->log_tau;
  c->h_theta[2] = theta->logit_rho;
  b->computed = false;
  return QSEL_OK;
}

static qsel_status batch_model(qsel_batch *b, int32_t model, qsel_ctx **c) {
  if (model < 0 || model >= (int)b->models.size())
    return batch_fail(b, fail(QSEL_EINVAL, "model index out of range"));
  if (!b->computed) {
    qsel_status st = qsel_batch_run(b);
    if (st) return st;
  }
  *c = b->models[model];
  return QSEL_OK;
}

qsel_status qsel_batch_diag_inv(qsel_batch *b, int32_t model, double *diag_out, int32_t out_is_device) {
  if (!b) return QSEL_EINVAL;
  if (!diag_out) return batch_fail(b, fail(QSEL_EINVAL, "diag_out must not be NULL"));
  qsel_ctx *c = nullptr;
  qsel_status st = batch_model(b, model, &c);
  if (st) return st;
  cudaError_t ce = cudaMemcpy(diag_out, c->d_diag, (size_t)c->n * sizeof(double),
                              out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
  if (ce != cudaSuccess) return batch_fail(b, cuda_fail(ce, "copy of diag", __FILE__, __LINE__));
  return QSEL_OK;
}

qsel_status qsel_batch_trace_grads(qsel_batch *b, int32_t model, double grads_out[3]) {
  if (!b) return QSEL_EINVAL;
  if (!grads_out) return batch_fail(b, fail(QSEL_EINVAL, "grads_out must not be NULL"));
  qsel_ctx *c = nullptr;
  qsel_status st = batch_model(b, model, &c);
  if (st) return st;
  if (c->n_l < 1 && c->parts.size() > 1)
    return batch_fail(b, fail(QSEL_EINVAL, "trace gradients need overlap >= 1 when there are several parts"));
  cudaError_t ce = cudaMemcpy(grads_out, c->d_traces, 3 * sizeof(double), cudaMemcpyDeviceToHost);
  if (ce != cudaSuccess) return batch_fail(b, cuda_fail(ce, "copy of traces", __FILE__, __LINE__));
  return QSEL_OK;
}

qsel_status qsel_batch_stats(const qsel_batch *b, int32_t model, qsel_stats_t *stats) {
  if (!b || !stats || model < 0 || model >= (int)b->models.size()) return QSEL_EINVAL;
  *stats = b->models[model]->stats;
  return QSEL_OK;
}

qsel_status qsel_batch_info(const qsel_batch *b, qsel_batch_info_t *info) {
  if (!b || !info) return QSEL_EINVAL;
  qsel_batch_info_t t{};
  t.n_models = (int32_t)b->models.size();
  t.n_streams = (int32_t)b->pool.size();
  t.ms_replay = b->ms_last;
  t.ms_capture = b->ms_capture;
  t.ms_autotune = b->ms_autotune;
  t.launches_per_replay = b->launches_per_replay;
  for (auto *c : b->models) t.max_pcg_iterations = std::max(t.max_pcg_iterations, c->stats.pcg_iterations);
  *info = t;
  return QSEL_OK;
}

qsel_status qsel_batch_tuning(const qsel_batch *b, int32_t model, int32_t *precond_block, int32_t *tensor_passes,
                              int32_t *stream) {
  if (!b || model < 0 || model >= (int)b->models.size()) return QSEL_EINVAL;
  if (precond_block) *precond_block = b->models[model]->bsize;
  if (tensor_passes) *tensor_passes = b->models[model]->mixed ? b->models[model]->tc_passes : 0;
  if (stream) *stream = b->stream_of[model];
  return QSEL_OK;
}

const char *qsel_batch_last_error(const qsel_batch *b) {
  if (!b) return g_create_error.c_str();
  return b->last_error.c_str();
}

void qsel_batch_destroy(qsel_batch *b) {
  if (!b) return;
  if (b->main) cudaStreamSynchronize(b->main);
  delete b;
}

qsel_status qsel_debug_apply_precond(qsel_ctx *ctx, const double *R, double *Z, int32_t ld) {
  if (!ctx) return QSEL_EINVAL;
  qsel_ctx *c = ctx;
  if (!R || !Z || ld < c->k) return finish(c, fail(QSEL_EINVAL, "NULL buffer or ld < n_samples"));
  cudaStream_t s = c->stream;
  Err e = run_model(c);
  if (e.code == 0 && c->kron) e = kron_prepare(c);
  if (e.code) return finish(c, e);
  cudaError_t ce0 = cudaMemsetAsync(c->d_err, 0, sizeof(int32_t), s);
  if (ce0 != cudaSuccess) return finish(c, cuda_fail(ce0, "error flag", __FILE__, __LINE__));
  if (c->mixed) {
    // the mixed form's binary32 preconditioner: R rounded to float, Z widened
    const size_t vec = (size_t)c->n * c->ld;
    std::vector<float> hr(vec, 0.0f), hz(vec);
    for (int i = 0; i < c->n; ++i)
      for (int j = 0; j < c->k; ++j) hr[(size_t)i * c->ld + j] = (float)R[(size_t)i * ld + j];
    float *pblk = static_cast<float *>(c->d_pblk);
    if (!c->kron) launch_jacobi_setup<float>(s, c->pat, c->mod, c->n_s, c->n_t, c->bsize, pblk, c->d_err);
    cudaError_t ce = cudaMemcpyAsync(c->f_r, hr.data(), vec * sizeof(float), cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(c->d_scal, 0, (size_t)c->ld * sizeof(double), s);   // alpha = 0
    if (ce != cudaSuccess) return finish(c, cuda_fail(ce, "preconditioner input", __FILE__, __LINE__));
    PcgVec<float> v = make_pcg<float>(c, c->f_x, c->f_r, c->f_z, c->f_p, c->f_q);
    launch_pcg_update<float>(s, v, pblk, c->bsize, c->kron ? &c->kop : nullptr);
    ce = cudaMemcpyAsync(hz.data(), c->f_z, vec * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return finish(c, cuda_fail(ce, "preconditioner output", __FILE__, __LINE__));
    int32_t err = 0;
    ce = cudaMemcpy(&err, c->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return finish(c, cuda_fail(ce, "error flag", __FILE__, __LINE__));
    if (err & 2) return finish(c, fail(QSEL_ETIMEOUT, "a bounded device-side wait of the tensor-core pass gave up"));
    for (int i = 0; i < c->n; ++i)
      for (int j = 0; j < c->k; ++j) Z[(size_t)i * ld + j] = (double)hz[(size_t)i * c->ld + j];
    return QSEL_OK;
  }
  double *pblk = static_cast<double *>(c->d_pblk);
  if (!c->kron)
    launch_jacobi_setup<double>(s, c->pat, c->mod, c->n_s, c->n_t,
                                c->bsize, pblk, c->d_err);
  const size_t vec = (size_t)c->n * c->ld;
  cudaError_t ce = cudaMemsetAsync(c->d_r, 0, vec * sizeof(double), s);
  if (ce == cudaSuccess)
    ce = cudaMemcpy2DAsync(c->d_r, (size_t)c->ld * sizeof(double), R, (size_t)ld * sizeof(double),
                           (size_t)c->k * sizeof(double), c->n, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(c->d_scal, 0, (size_t)c->ld * sizeof(double), s);   // alpha = 0
  if (ce != cudaSuccess) return finish(c, cuda_fail(ce, "preconditioner input", __FILE__, __LINE__));
  PcgVec<double> v = make_pcg<double>(c, c->d_X, c->d_r, c->d_zv, c->d_p, c->d_q);
  launch_pcg_update<double>(s, v, pblk, c->bsize, c->kron ? &c->kop : nullptr);
  ce = cudaMemcpy2DAsync(Z, (size_t)ld * sizeof(double), c->d_zv, (size_t)c->ld * sizeof(double),
                         (size_t)c->k * sizeof(double), c->n, cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return finish(c, cuda_fail(ce, "preconditioner output", __FILE__, __LINE__));
  return QSEL_OK;
}

qsel_status qsel_debug_get_lanczos(const qsel_ctx *ctx, double *alpha, double *beta, int32_t ld) {
  if (!ctx) return QSEL_EINVAL;
  qsel_ctx *c = const_cast<qsel_ctx *>(ctx);
  if (!alpha || !beta || ld < ctx->k) return finish(c, fail(QSEL_EINVAL, "NULL output or ld < n_samples"));
  if (!ctx->lz.ran) return finish(c, fail(QSEL_ESTATE, "the last run did not use the Lanczos sampler"));
  const int m = ctx->opt.lanczos_steps;
  cudaError_t ce = cudaMemcpy2D(alpha, (size_t)ld * sizeof(double), ctx->lz.alpha, (size_t)ctx->ld * sizeof(double),
                                (size_t)ctx->k * sizeof(double), m, cudaMemcpyDeviceToHost);
  if (ce == cudaSuccess)
    ce = cudaMemcpy2D(beta, (size_t)ld * sizeof(double), ctx->lz.beta, (size_t)ctx->ld * sizeof(double),
                      (size_t)ctx->k * sizeof(double), m, cudaMemcpyDeviceToHost);
  if (ce != cudaSuccess) return finish(c, cuda_fail(ce, "copy of Lanczos coefficients", __FILE__, __LINE__));
  return QSEL_OK;
}

const char *qsel_last_error(const qsel_ctx *ctx) {
  if (!ctx) return g_create_error.c_str();
  return ctx->last_error.c_str();
}

void qsel_destroy(qsel_ctx *ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  delete ctx;
}

}  // extern "C"
