// C ABI (include/qsel.h) and the host orchestration of the pipeline:
// perturbation samples -> multi-RHS PCG -> per-subdomain block factorisation
// and Takahashi selected inversion -> RB correction -> diag and traces.
#include <algorithm>
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

struct Subdomain {
  int s0, s1, e0, e1, T, lo, hi;
  int sep_left, sep_right;             // separator slabs or -1
  std::vector<double *> Dinv;          // T dense pivot-block inverses
  double *SigA = nullptr, *SigB = nullptr, *Y = nullptr, *W = nullptr, *V = nullptr;
  double *P = nullptr, *U = nullptr, *Vs = nullptr;  // sweep scratch
  double *wbuf = nullptr;              // T x n_pad x ld correction samples
  double *ybuf = nullptr, *tmp = nullptr, *bright = nullptr;
  double *partial = nullptr;           // corr_grid x 3
};

}  // namespace qsel

using namespace qsel;

struct qsel_ctx {
  int n_s = 0, n_t = 0, n = 0, ld = 0, k = 0, n_pad = 0, n_l = 0, bsize = 64;
  double sigma = 1.0, obs_w = 1.0;
  qsel_theta theta{};
  qsel_options opt{};
  cudaStream_t stream = nullptr;
  std::vector<int> slab_start;
  // spatial pattern
  SellPattern pat{};
  int n_ent = 0;
  double *d_c_pat = nullptr, *d_g_pat = nullptr, *d_h_pat = nullptr, *d_isqc_pat = nullptr;
  double *d_qs = nullptr, *d_dqs = nullptr, *d_kc = nullptr;
  uint8_t *d_obs = nullptr;
  int32_t *d_obs_index = nullptr;
  int n_obs = 0;
  TimeCoeffs tc{};
  // sampler
  double *d_z1 = nullptr, *d_z2 = nullptr, *d_R = nullptr, *d_X = nullptr;
  double *d_r = nullptr, *d_zv = nullptr, *d_p = nullptr, *d_q = nullptr;
  double *d_pa = nullptr, *d_pb = nullptr, *d_pblk = nullptr;
  double *d_scal = nullptr;           // alpha, beta, rho, bb, rr (ld each) + max_rel
  int32_t *d_active = nullptr, *d_counters = nullptr;
  // estimator
  std::vector<Subdomain> parts;
  double *d_diag = nullptr, *d_selinv = nullptr, *d_traces = nullptr, *d_sums = nullptr;
  double *d_partials = nullptr;
  TraceSlab *d_slabs = nullptr;
  int n_trace_slabs = 0;
  int32_t *d_err = nullptr;
  // host staging
  int32_t *h_counters = nullptr;
  double *h_small = nullptr;
  cudaEvent_t ev[8]{};
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
  ~qsel_ctx() {
    for (void *p : allocs) cudaFree(p);
    if (h_counters) cudaFreeHost(h_counters);
    if (h_small) cudaFreeHost(h_small);
    for (auto &e : ev)
      if (e) cudaEventDestroy(e);
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
  if (overlap < 0) return fail(QSEL_EINVAL, "overlap must be >= 0");
  const int np = part ? part->n_parts : 1;
  if (np < 1 || np > m->n_t) return fail(QSEL_EINVAL, "n_parts must be in [1, n_t]");
  if (part && part->slab_start) {
    if (part->slab_start[0] != 0 || part->slab_start[np] != m->n_t)
      return fail(QSEL_EINVAL, "slab_start must run from 0 to n_t");
    for (int p = 0; p < np; ++p)
      if (part->slab_start[p + 1] <= part->slab_start[p])
        return fail(QSEL_EINVAL, "slab_start must be strictly increasing");
  }
  if (opt->n_samples < 1 || opt->n_samples > 512) return fail(QSEL_EINVAL, "n_samples must be in [1, 512]");
  if (opt->precision != QSEL_FP64) return fail(QSEL_EINVAL, "precision: only QSEL_FP64 is available in this build");
  if (!(opt->pcg_tol > 0.0) || opt->pcg_max_iter < 1) return fail(QSEL_EINVAL, "pcg_tol > 0 and pcg_max_iter >= 1 required");
  if (opt->precond_block != 0 && opt->precond_block != 1 && opt->precond_block != 16 &&
      opt->precond_block != 32 && opt->precond_block != 64)
    return fail(QSEL_EINVAL, "precond_block must be 0, 1, 16, 32 or 64");
  if (opt->control_variate != 0) return fail(QSEL_EINVAL, "control_variate must be 0");
  return ok();
}

template <typename T>
static Err upload(qsel_ctx *c, T **dst, const std::vector<T> &src) {
  TRY(c->alloc(dst, src.size()));
  if (!src.empty()) QSEL_CUDA_TRY(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return ok();
}

static Err build(qsel_ctx *c, const qsel_model *m, const qsel_partition *part, int32_t overlap) {
  const int n_s = m->n_s;
  // spatial pattern rows: col -> (C, G, H = G C^-1 G)
  std::vector<std::map<int, std::array<double, 3>>> rows(n_s);
  for (int i = 0; i < n_s; ++i) {
    auto &r = rows[i];
    auto touch = [&](int j) -> double * {
      auto it = r.find(j);
      if (it == r.end()) it = r.emplace(j, std::array<double, 3>{0.0, 0.0, 0.0}).first;
      return it->second.data();
    };
    touch(i)[0] = m->c_diag[i];
    for (int p = m->g_rowptr[i]; p < m->g_rowptr[i + 1]; ++p) {
      const int j = m->g_col[p];
      touch(j)[1] += m->g_val[p];
      const double gij = m->g_val[p] / m->c_diag[j];
      for (int q = m->g_rowptr[j]; q < m->g_rowptr[j + 1]; ++q) touch(m->g_col[q])[2] += gij * m->g_val[q];
    }
  }
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
  std::vector<double> cp(n_ent, 0.0), gp(n_ent, 0.0), hp(n_ent, 0.0), isq(n_ent, 0.0);
  for (int s = 0; s < n_slices; ++s) {
    for (int l = 0; l < kSlice; ++l) {
      const int i = s * kSlice + l;
      int slot = 0;
      if (i < n_s) {
        for (auto &kv : rows[i]) {
          const int e = slice_ptr[s] + slot * kSlice + l;
          col[e] = kv.first;
          cp[e] = kv.second[0];
          gp[e] = kv.second[1];
          hp[e] = kv.second[2];
          isq[e] = 1.0 / std::sqrt(m->c_diag[kv.first]);
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
  c->pat.n_rows = n_s;
  c->pat.n_slices = n_slices;
  c->pat.max_width = max_w;
  c->pat.slice_ptr = d_sp;
  c->pat.slice_width = d_sw;
  c->pat.col = d_col;
  c->n_ent = n_ent;
  TRY(upload(c, &c->d_c_pat, cp));
  TRY(upload(c, &c->d_g_pat, gp));
  TRY(upload(c, &c->d_h_pat, hp));
  TRY(upload(c, &c->d_isqc_pat, isq));
  TRY(c->alloc(&c->d_qs, n_ent));
  TRY(c->alloc(&c->d_dqs, n_ent));
  TRY(c->alloc(&c->d_kc, n_ent));

  // observations
  const int n = c->n;
  std::vector<uint8_t> mask(m->obs_mask, m->obs_mask + n);
  std::vector<int32_t> oidx(n, -1);
  int n_obs = 0;
  for (int r = 0; r < n; ++r) {
    mask[r] = mask[r] ? 1 : 0;
    if (mask[r]) oidx[r] = n_obs++;
  }
  c->n_obs = n_obs;
  TRY(upload(c, &c->d_obs, mask));
  TRY(upload(c, &c->d_obs_index, oidx));

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
  c->n_l = overlap;

  // sampler buffers
  const size_t vec = (size_t)n * c->ld;
  TRY(c->alloc(&c->d_z1, vec));
  TRY(c->alloc(&c->d_z2, (size_t)std::max(n_obs, 1) * c->ld));
  TRY(c->alloc(&c->d_R, vec));
  TRY(c->alloc(&c->d_X, vec));
  TRY(c->alloc(&c->d_r, vec));
  TRY(c->alloc(&c->d_zv, vec));
  TRY(c->alloc(&c->d_p, vec));
  TRY(c->alloc(&c->d_q, vec));
  const int n_tiles = (n + 63) / 64;
  const int n_pa = std::max(n_tiles, bt_spmm_grid(n));
  TRY(c->alloc(&c->d_pa, (size_t)n_pa * c->ld));
  TRY(c->alloc(&c->d_pb, (size_t)n_tiles * c->ld));
  const int nblk = (n + c->bsize - 1) / c->bsize;
  TRY(c->alloc(&c->d_pblk, (size_t)nblk * c->bsize * c->bsize));
  TRY(c->alloc(&c->d_scal, (size_t)5 * c->ld + 8));
  TRY(c->alloc(&c->d_active, (size_t)c->ld));
  TRY(c->alloc(&c->d_counters, 8));
  QSEL_CUDA_TRY(cudaMemset(c->d_X, 0, vec * sizeof(double)));

  // subdomains
  const int n_pad = c->n_pad;
  const size_t mat = (size_t)n_pad * n_pad;
  const size_t svec = (size_t)n_pad * c->ld;
  int n_sums = 0;
  std::vector<TraceSlab> tslabs;
  for (int p = 0; p < np; ++p) {
    Subdomain sd;
    sd.s0 = c->slab_start[p];
    sd.s1 = c->slab_start[p + 1];
    sd.e0 = std::max(0, sd.s0 - overlap);
    sd.e1 = std::min(c->n_t, sd.s1 + overlap);
    sd.T = sd.e1 - sd.e0;
    sd.lo = sd.s0 - sd.e0;
    sd.hi = sd.s1 - 1 - sd.e0;
    sd.sep_left = sd.e0 > 0 ? sd.e0 - 1 : -1;
    sd.sep_right = sd.e1 < c->n_t ? sd.e1 : -1;
    sd.Dinv.resize(sd.T);
    for (int t = 0; t < sd.T; ++t) TRY(c->alloc(&sd.Dinv[t], mat));
    TRY(c->alloc(&sd.SigA, mat));
    TRY(c->alloc(&sd.SigB, mat));
    TRY(c->alloc(&sd.Y, mat));
    TRY(c->alloc(&sd.W, mat));
    TRY(c->alloc(&sd.V, mat));
    TRY(c->alloc(&sd.P, 64 * 64));
    TRY(c->alloc(&sd.U, (size_t)n_pad * 64));
    TRY(c->alloc(&sd.Vs, (size_t)n_pad * 64));
    TRY(c->alloc(&sd.wbuf, (size_t)sd.T * svec));
    TRY(c->alloc(&sd.ybuf, svec));
    TRY(c->alloc(&sd.tmp, svec));
    TRY(c->alloc(&sd.bright, svec));
    // trace bookkeeping: sums slots 2 per (sd, local slab) for Sigma and for Y
    const int base_sd = n_sums;
    n_sums += 2 * sd.T;
    for (int tl = sd.lo; tl <= sd.hi; ++tl) {
      TraceSlab ts;
      ts.t = sd.e0 + tl;
      ts.sd = base_sd + tl;                              // Sigma_tl
      ts.sy = (tl + 1 < sd.T) ? base_sd + sd.T + tl : -1;  // Y_tl
      ts.sym = (tl > 0) ? base_sd + sd.T + tl - 1 : -1;     // Y_{tl-1}
      tslabs.push_back(ts);
    }
    c->parts.push_back(std::move(sd));
  }
  TRY(c->alloc(&c->d_partials, (size_t)np * corr_grid() * 3));
  QSEL_CUDA_TRY(cudaMemset(c->d_partials, 0, (size_t)np * corr_grid() * 3 * sizeof(double)));
  for (int p = 0; p < np; ++p) c->parts[p].partial = c->d_partials + (size_t)p * corr_grid() * 3;
  TRY(c->alloc(&c->d_sums, (size_t)2 * std::max(n_sums, 1)));
  QSEL_CUDA_TRY(cudaMemset(c->d_sums, 0, (size_t)2 * std::max(n_sums, 1) * sizeof(double)));
  c->n_trace_slabs = (int)tslabs.size();
  TRY(upload(c, &c->d_slabs, tslabs));
  TRY(c->alloc(&c->d_diag, (size_t)n));
  TRY(c->alloc(&c->d_selinv, (size_t)n));
  TRY(c->alloc(&c->d_traces, 4));
  TRY(c->alloc(&c->d_err, 4));
  QSEL_CUDA_TRY(cudaHostAlloc(&c->h_counters, 64, cudaHostAllocDefault));
  QSEL_CUDA_TRY(cudaHostAlloc(&c->h_small, 64 * sizeof(double), cudaHostAllocDefault));
  for (auto &e : c->ev) QSEL_CUDA_TRY(cudaEventCreate(&e));
  return ok();
}

// ---------------------------------------------------------------------------
// Pipeline
// ---------------------------------------------------------------------------
static Err run_model(qsel_ctx *c) {
  launch_time_coeffs(c->stream, c->theta.log_kappa, c->theta.log_tau, c->theta.logit_rho, c->n_t, c->tc);
  launch_qs_values(c->stream, c->n_ent, c->d_c_pat, c->d_g_pat, c->d_h_pat, c->d_isqc_pat,
                   c->tc.scalars, c->d_qs, c->d_dqs, c->d_kc);
  QSEL_CUDA_TRY(cudaGetLastError());
  return ok();
}

static PcgVec pcg_vec(qsel_ctx *c) {
  PcgVec v;
  v.n = c->n;
  v.ld = c->ld;
  v.n_blocks_dot = bt_spmm_grid(c->n);
  v.n_tiles = (c->n + 63) / 64;
  v.x = c->d_X;
  v.r = c->d_r;
  v.z = c->d_zv;
  v.p = c->d_p;
  v.q = c->d_q;
  v.b = c->d_R;
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

static Err run_sampler(qsel_ctx *c) {
  cudaStream_t s = c->stream;
  const size_t vec = (size_t)c->n * c->ld * sizeof(double);
  launch_philox_normals(s, c->opt.seed, 0u, c->n, c->k, c->ld, c->d_z1);
  launch_philox_normals(s, c->opt.seed, 1u, c->n_obs, c->k, c->ld, c->d_z2);
  launch_perturbation_rhs(s, c->pat, c->d_kc, c->n_s, c->n_t, c->ld, c->tc.bdiag, c->tc.scalars,
                          c->d_z1, c->d_z2, c->d_obs_index, 1.0 / c->sigma, c->d_R);
  c->have_rhs = true;
  QSEL_CUDA_TRY(cudaEventRecord(c->ev[1], s));
  // preconditioner
  launch_jacobi_setup(s, c->pat, c->d_qs, c->tc.a0, c->tc.a1, c->d_obs, c->obs_w, c->n_s, c->n_t,
                      c->bsize, c->d_pblk, c->d_err);
  // PCG init: x = 0, r = b, p = 0, z = M^-1 r
  PcgVec v = pcg_vec(c);
  QSEL_CUDA_TRY(cudaMemsetAsync(c->d_X, 0, vec, s));
  QSEL_CUDA_TRY(cudaMemsetAsync(c->d_p, 0, vec, s));
  QSEL_CUDA_TRY(cudaMemsetAsync(c->d_scal, 0, (size_t)c->ld * sizeof(double), s));  // alpha = 0
  QSEL_CUDA_TRY(cudaMemcpyAsync(c->d_r, c->d_R, vec, cudaMemcpyDeviceToDevice, s));
  launch_pcg_update(s, v, c->d_pblk, c->bsize);
  launch_pcg_reduce_beta(s, v, c->opt.pcg_tol, 1);
  launch_pcg_p_update(s, v);
  BtSpmmArgs a{};
  a.pat = c->pat;
  a.val = c->d_qs;
  a.c0 = c->tc.a0;
  a.c1 = c->tc.a1;
  a.obs = c->d_obs;
  a.obs_w = c->obs_w;
  a.n_s = c->n_s;
  a.n_t = c->n_t;
  a.ld = c->ld;
  a.x = c->d_p;
  a.y = c->d_q;
  a.dot_partial = c->d_pa;
  const int check_every = 8;
  int it = 0;
  bool done = false;
  // iteration 0 check: all-zero right-hand sides converge immediately
  QSEL_CUDA_TRY(cudaMemcpyAsync(c->h_counters, c->d_counters, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  QSEL_CUDA_TRY(cudaStreamSynchronize(s));
  if (c->h_counters[0] == 0) done = true;
  while (!done && it < c->opt.pcg_max_iter) {
    const int batch = std::min(check_every, c->opt.pcg_max_iter - it);
    for (int b = 0; b < batch; ++b) {
      launch_bt_spmm(s, a);
      launch_pcg_reduce_alpha(s, v);
      launch_pcg_update(s, v, c->d_pblk, c->bsize);
      launch_pcg_reduce_beta(s, v, c->opt.pcg_tol, 0);
      launch_pcg_p_update(s, v);
    }
    it += batch;
    QSEL_CUDA_TRY(cudaGetLastError());
    QSEL_CUDA_TRY(cudaMemcpyAsync(c->h_counters, c->d_counters, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    QSEL_CUDA_TRY(cudaStreamSynchronize(s));
    if (c->h_counters[0] == 0) done = true;
  }
  QSEL_CUDA_TRY(cudaMemcpyAsync(c->h_small, v.max_rel, sizeof(double), cudaMemcpyDeviceToHost, s));
  QSEL_CUDA_TRY(cudaStreamSynchronize(s));
  c->stats.pcg_iterations = it;
  c->stats.pcg_max_rel_residual = c->h_small[0];
  if (!done)
    return fail(QSEL_ENOCONV, "PCG did not reach pcg_tol within pcg_max_iter iterations (max relative residual " +
                                  std::to_string(c->h_small[0]) + ")");
  return ok();
}

// Forward block factorisation (pivot-block inverses) and backward Takahashi
// recursion for every subdomain, batched in lockstep.
static Err run_selinv(qsel_ctx *c) {
  cudaStream_t s = c->stream;
  const int n_pad = c->n_pad, n_s = c->n_s;
  const int np = (int)c->parts.size();
  int maxT = 0;
  for (auto &sd : c->parts) maxT = std::max(maxT, sd.T);
  for (int g0 = 0; g0 < np; g0 += kMaxBatch) {
    const int g1 = std::min(np, g0 + kMaxBatch);
    // forward
    for (int t = 0; t < maxT; ++t) {
      SchurBatch sb{};
      SweepBatch wb{};
      SpBatch gb{};
      for (int p = g0; p < g1; ++p) {
        Subdomain &sd = c->parts[p];
        if (t >= sd.T) continue;
        const int tg = sd.e0 + t;
        SchurEntry &se = sb.e[sb.count++];
        se.W = (t > 0) ? sd.W : nullptr;
        se.D = sd.Dinv[t];
        se.a0 = c->tc.a0 + tg;
        se.c = (t > 0) ? c->tc.a1 + tg - 1 : c->tc.a1;
        se.obs = c->d_obs + (size_t)tg * n_s;
        SweepEntry &we = wb.e[wb.count++];
        we.A = sd.Dinv[t];
        we.P = sd.P;
        we.U = sd.U;
        we.V = sd.Vs;
        if (t + 1 < sd.T) {
          SpEntry &ge = gb.e[gb.count++];
          ge.B = sd.Dinv[t];
          ge.C = nullptr;
          ge.Out = sd.W;
          ge.alpha_ptr = c->tc.a1 + tg;
          ge.alpha = 1.0;
          ge.beta = 0.0;
        }
      }
      launch_schur_assemble(s, sb, c->pat, c->d_qs, c->obs_w, n_s, n_pad);
      spd_inverse(s, wb, n_pad, c->d_err);
      launch_sp_rowgather(s, gb, c->pat, c->d_qs, n_s, n_pad, n_pad, n_pad);
    }
    QSEL_CUDA_TRY(cudaGetLastError());
  }
  QSEL_CUDA_TRY(cudaEventRecord(c->ev[3], s));
  for (int g0 = 0; g0 < np; g0 += kMaxBatch) {
    const int g1 = std::min(np, g0 + kMaxBatch);
    std::vector<int> slot_base(np, 0);
    {
      int acc = 0;
      for (int p = 0; p < np; ++p) {
        slot_base[p] = acc;
        acc += 2 * c->parts[p].T;
      }
    }
    // Sigma_{T-1} = Dinv_{T-1}
    {
      ExtractBatch xb{};
      for (int p = g0; p < g1; ++p) {
        Subdomain &sd = c->parts[p];
        const int tl = sd.T - 1;
        if (tl < sd.lo || tl > sd.hi) continue;
        ExtractEntry &xe = xb.e[xb.count++];
        xe.S = sd.Dinv[tl];
        xe.diag_out = c->d_selinv + (size_t)(sd.e0 + tl) * n_s;
        xe.sums = c->d_sums + 2 * (size_t)(slot_base[p] + tl);
      }
      launch_extract(s, xb, c->pat, c->d_qs, c->d_dqs, n_s, n_pad);
    }
    std::vector<double *> sig_next(np, nullptr);
    std::vector<int> flip(np, 0);
    for (int p = g0; p < g1; ++p) sig_next[p] = c->parts[p].Dinv[c->parts[p].T - 1];
    for (int b = 0; b < maxT; ++b) {
      SpBatch wb{}, vb{};
      GemmBatch yb{}, sgb{};
      SweepBatch mb{};
      ExtractBatch xy{}, xs{};
      std::vector<int> active;
      for (int p = g0; p < g1; ++p) {
        Subdomain &sd = c->parts[p];
        const int tl = sd.T - 2 - b;
        if (tl < std::max(sd.lo - 1, 0)) continue;
        active.push_back(p);
        const int tg = sd.e0 + tl;
        SpEntry &we = wb.e[wb.count++];
        we.B = sd.Dinv[tl];
        we.C = nullptr;
        we.Out = sd.W;
        we.alpha_ptr = c->tc.a1 + tg;
        we.alpha = 1.0;
        we.beta = 0.0;
        GemmEntry &ye = yb.e[yb.count++];
        ye.A = sig_next[p];
        ye.B = sd.W;
        ye.C0 = nullptr;
        ye.C = sd.Y;
        ye.alpha = 1.0;
        ye.beta = 0.0;
        const bool y_needed = (tl >= sd.lo && tl <= sd.hi) || (tl + 1 >= sd.lo && tl + 1 <= sd.hi);
        if (y_needed) {
          ExtractEntry &xe = xy.e[xy.count++];
          xe.S = sd.Y;
          xe.diag_out = nullptr;
          xe.sums = c->d_sums + 2 * (size_t)(slot_base[p] + sd.T + tl);
        }
        if (tl >= sd.lo) {
          double *sig_cur = flip[p] ? sd.SigB : sd.SigA;
          SpEntry &ve = vb.e[vb.count++];
          ve.B = sd.Y;
          ve.C = nullptr;
          ve.Out = sd.V;
          ve.alpha_ptr = c->tc.a1 + tg;
          ve.alpha = 1.0;
          ve.beta = 0.0;
          GemmEntry &ge = sgb.e[sgb.count++];
          ge.A = sd.Dinv[tl];
          ge.B = sd.V;
          ge.C0 = sd.Dinv[tl];
          ge.C = sig_cur;
          ge.alpha = 1.0;
          ge.beta = 1.0;
          SweepEntry &me = mb.e[mb.count++];
          me.A = sig_cur;
          if (tl <= sd.hi) {
            ExtractEntry &xe = xs.e[xs.count++];
            xe.S = sig_cur;
            xe.diag_out = c->d_selinv + (size_t)tg * n_s;
            xe.sums = c->d_sums + 2 * (size_t)(slot_base[p] + tl);
          }
        }
      }
      if (active.empty()) break;
      launch_sp_rowgather(s, wb, c->pat, c->d_qs, n_s, n_pad, n_pad, n_pad);
      launch_gemm(s, yb, n_pad, n_pad, n_pad, n_pad, n_pad, n_pad, false);
      launch_extract(s, xy, c->pat, c->d_qs, c->d_dqs, n_s, n_pad);
      launch_sp_rowgather(s, vb, c->pat, c->d_qs, n_s, n_pad, n_pad, n_pad);
      launch_gemm(s, sgb, n_pad, n_pad, n_pad, n_pad, n_pad, n_pad, true);
      launch_mirror(s, mb, n_pad);
      launch_extract(s, xs, c->pat, c->d_qs, c->d_dqs, n_s, n_pad);
      for (int p : active) {
        Subdomain &sd = c->parts[p];
        const int tl = sd.T - 2 - b;
        if (tl >= sd.lo) {
          sig_next[p] = flip[p] ? sd.SigB : sd.SigA;
          flip[p] ^= 1;
        }
      }
      QSEL_CUDA_TRY(cudaGetLastError());
    }
  }
  return ok();
}

// RB correction: w = Q_{**}^-1 Q_{*S} x_S by the block LDL^T sweeps
//   forward  y_0 = b_0, u_t = D_t^-1 y_t, y_{t+1} = b_{t+1} - c_t Q_s u_t
//   backward w_{T-1} = u_{T-1}, w_t = u_t - D_t^-1 (c_t Q_s w_{t+1})
// then the squares and trace forms on the own rows.
static Err run_correction(qsel_ctx *c) {
  cudaStream_t s = c->stream;
  const int n_pad = c->n_pad, n_s = c->n_s, ld = c->ld;
  const int np = (int)c->parts.size();
  const size_t svec = (size_t)n_pad * ld;
  int maxT = 0;
  for (auto &sd : c->parts) maxT = std::max(maxT, sd.T);
  for (int g0 = 0; g0 < np; g0 += kMaxBatch) {
    const int g1 = std::min(np, g0 + kMaxBatch);
    std::vector<int> grp;
    for (int p = g0; p < g1; ++p)
      if (c->parts[p].sep_left >= 0 || c->parts[p].sep_right >= 0) grp.push_back(p);
    if (grp.empty()) continue;
    // boundary terms
    {
      SpBatch bl{}, br{};
      for (int p : grp) {
        Subdomain &sd = c->parts[p];
        if (sd.sep_left >= 0) {
          SpEntry &e = bl.e[bl.count++];
          e.B = c->d_X + (size_t)sd.sep_left * n_s * ld;
          e.C = nullptr;
          e.Out = sd.ybuf;
          e.alpha_ptr = c->tc.a1 + sd.sep_left;
          e.alpha = 1.0;
          e.beta = 0.0;
        } else {
          QSEL_CUDA_TRY(cudaMemsetAsync(sd.ybuf, 0, svec * sizeof(double), s));
        }
        if (sd.sep_right >= 0) {
          SpEntry &e = br.e[br.count++];
          e.B = c->d_X + (size_t)sd.sep_right * n_s * ld;
          e.C = nullptr;
          e.Out = sd.bright;
          e.alpha_ptr = c->tc.a1 + sd.sep_right - 1;
          e.alpha = 1.0;
          e.beta = 0.0;
        }
      }
      launch_sp_rowgather(s, bl, c->pat, c->d_qs, n_s, n_pad, ld, ld);
      launch_sp_rowgather(s, br, c->pat, c->d_qs, n_s, n_pad, ld, ld);
      for (int p : grp) {
        Subdomain &sd = c->parts[p];
        if (sd.T == 1 && sd.sep_right >= 0) launch_add(s, sd.ybuf, sd.bright, (int)svec);
      }
    }
    // forward sweep
    for (int t = 0; t < maxT; ++t) {
      GemmBatch ub{};
      SpBatch yb{};
      for (int p : grp) {
        Subdomain &sd = c->parts[p];
        if (t >= sd.T) continue;
        GemmEntry &g = ub.e[ub.count++];
        g.A = sd.Dinv[t];
        g.B = sd.ybuf;
        g.C0 = nullptr;
        g.C = sd.wbuf + (size_t)t * svec;
        g.alpha = 1.0;
        g.beta = 0.0;
        if (t + 1 < sd.T) {
          SpEntry &e = yb.e[yb.count++];
          e.B = sd.wbuf + (size_t)t * svec;
          const bool add_right = (t + 1 == sd.T - 1) && sd.sep_right >= 0;
          e.C = add_right ? sd.bright : nullptr;
          e.Out = sd.ybuf;
          e.alpha_ptr = c->tc.a1 + sd.e0 + t;
          e.alpha = -1.0;
          e.beta = add_right ? 1.0 : 0.0;
        }
      }
      if (ub.count == 0) break;
      launch_gemm(s, ub, n_pad, ld, n_pad, n_pad, ld, ld, false);
      launch_sp_rowgather(s, yb, c->pat, c->d_qs, n_s, n_pad, ld, ld);
    }
    // backward sweep
    for (int b = 0; b < maxT; ++b) {
      SpBatch tb{};
      GemmBatch wb{};
      for (int p : grp) {
        Subdomain &sd = c->parts[p];
        const int t = sd.T - 2 - b;
        if (t < std::max(sd.lo - 1, 0)) continue;
        SpEntry &e = tb.e[tb.count++];
        e.B = sd.wbuf + (size_t)(t + 1) * svec;
        e.C = nullptr;
        e.Out = sd.tmp;
        e.alpha_ptr = c->tc.a1 + sd.e0 + t;
        e.alpha = 1.0;
        e.beta = 0.0;
        GemmEntry &g = wb.e[wb.count++];
        g.A = sd.Dinv[t];
        g.B = sd.tmp;
        g.C0 = sd.wbuf + (size_t)t * svec;
        g.C = sd.wbuf + (size_t)t * svec;
        g.alpha = -1.0;
        g.beta = 1.0;
      }
      if (tb.count == 0) break;
      launch_sp_rowgather(s, tb, c->pat, c->d_qs, n_s, n_pad, ld, ld);
      launch_gemm(s, wb, n_pad, ld, n_pad, n_pad, ld, ld, false);
    }
    QSEL_CUDA_TRY(cudaGetLastError());
  }
  // squares and trace forms on the own rows of every subdomain
  for (int g0 = 0; g0 < np; g0 += kMaxBatch) {
    const int g1 = std::min(np, g0 + kMaxBatch);
    CorrBatch cb{};
    for (int p = g0; p < g1; ++p) {
      Subdomain &sd = c->parts[p];
      if (sd.sep_left < 0 && sd.sep_right < 0) continue;
      CorrEntry &e = cb.e[cb.count++];
      e.w = sd.wbuf;
      e.T = sd.T;
      e.lo = sd.lo;
      e.hi = sd.hi;
      e.e0 = sd.e0;
      e.diag_out = c->d_diag;
      e.partial = sd.partial;
    }
    launch_correction_terms(s, cb, c->pat, c->d_qs, c->d_dqs, c->tc.a0, c->tc.a1, c->tc.r0, c->tc.r1,
                            n_s, n_pad, ld, c->k);
  }
  QSEL_CUDA_TRY(cudaGetLastError());
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
    double ms[PROF_KINDS] = {0, 0, 0}, work[PROF_KINDS] = {0, 0, 0};
    int64_t cnt[PROF_KINDS] = {0, 0, 0};
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
  }
  return e;
}

static Err run_pipeline_body(qsel_ctx *c) {
  cudaStream_t s = c->stream;
  const int64_t launches0 = g_launch_count;
  QSEL_CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int32_t), s));
  QSEL_CUDA_TRY(cudaEventRecord(c->ev[0], s));
  TRY(run_model(c));
  const bool need_samples = c->parts.size() > 1;
  if (!c->injected) {
    if (need_samples) {
      TRY(run_sampler(c));
    } else {
      QSEL_CUDA_TRY(cudaEventRecord(c->ev[1], s));
      c->stats.pcg_iterations = 0;
      c->stats.pcg_max_rel_residual = 0.0;
    }
  } else {
    QSEL_CUDA_TRY(cudaEventRecord(c->ev[1], s));
  }
  QSEL_CUDA_TRY(cudaEventRecord(c->ev[2], s));
  TRY(run_selinv(c));
  QSEL_CUDA_TRY(cudaEventRecord(c->ev[4], s));
  QSEL_CUDA_TRY(cudaMemcpyAsync(c->d_diag, c->d_selinv, (size_t)c->n * sizeof(double),
                                cudaMemcpyDeviceToDevice, s));
  TRY(run_correction(c));
  // traces: selected-inverse pattern sums plus every subdomain's correction partials
  launch_trace_combine(s, c->d_slabs, c->n_trace_slabs, c->d_sums, c->d_partials,
                       (int)c->parts.size() * corr_grid(), c->tc.a0, c->tc.a1, c->tc.r0, c->tc.r1,
                       c->d_traces);
  QSEL_CUDA_TRY(cudaEventRecord(c->ev[5], s));
  QSEL_CUDA_TRY(cudaStreamSynchronize(s));
  QSEL_CUDA_TRY(cudaGetLastError());
  int32_t err = 0;
  QSEL_CUDA_TRY(cudaMemcpy(&err, c->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (err & 1) return fail(QSEL_ENOTSPD, "a pivot of a dense block factorisation was not positive");
  float ms;
  auto el = [&](int a, int b) {
    cudaEventElapsedTime(&ms, c->ev[a], c->ev[b]);
    return (double)ms;
  };
  c->stats.ms_rhs = c->injected ? 0.0 : el(0, 1);
  c->stats.ms_pcg = el(1, 2);
  c->stats.ms_factor = el(2, 3);
  c->stats.ms_takahashi = el(3, 4);
  c->stats.ms_correction = el(4, 5);
  c->stats.ms_total = el(0, 5);
  c->stats.kernel_launches = g_launch_count - launches0;
  c->computed = true;
  return ok();
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

qsel_status qsel_create(qsel_ctx **out, const qsel_model *model, const qsel_theta *theta,
                        const qsel_partition *partition, int32_t overlap, const qsel_options *opt) {
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
  c->n_s = model->n_s;
  c->n_t = model->n_t;
  c->n = model->n_s * model->n_t;
  c->k = opt->n_samples;
  c->ld = round_up(opt->n_samples, kColPad);
  c->n_pad = round_up(model->n_s, kTile);
  c->sigma = model->sigma;
  c->obs_w = 1.0 / (model->sigma * model->sigma);
  c->theta = *theta;
  c->opt = *opt;
  c->bsize = opt->precond_block == 0 ? 64 : opt->precond_block;
  c->stream = reinterpret_cast<cudaStream_t>(opt->cuda_stream);
  e = build(c, model, partition, overlap);
  if (e.code) {
    g_create_error = e.msg;
    delete c;
    return (qsel_status)e.code;
  }
  *out = c;
  return QSEL_OK;
}

qsel_status qsel_set_theta(qsel_ctx *ctx, const qsel_theta *theta) {
  if (!ctx || !theta) return QSEL_EINVAL;
  if (!std::isfinite(theta->log_kappa) || !std::isfinite(theta->log_tau) ||
      !std::isfinite(theta->logit_rho) || std::fabs(theta->logit_rho) > 36.0)
    return finish(ctx, fail(QSEL_EINVAL, "theta must be finite with |logit rho| <= 36"));
  ctx->theta = *theta;
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

qsel_status qsel_trace_grads(qsel_ctx *ctx, double grads_out[3]) {
  if (!ctx) return QSEL_EINVAL;
  if (!grads_out) return finish(ctx, fail(QSEL_EINVAL, "grads_out must not be NULL"));
  if (ctx->n_l < 1 && ctx->parts.size() > 1)
    return finish(ctx, fail(QSEL_EINVAL, "trace gradients need overlap >= 1 when there are several parts"));
  Err e = ensure(ctx);
  if (e.code) return finish(ctx, e);
  cudaError_t ce = cudaMemcpyAsync(ctx->h_small, ctx->d_traces, 3 * sizeof(double),
                                   cudaMemcpyDeviceToHost, ctx->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
  if (ce != cudaSuccess) return finish(ctx, cuda_fail(ce, "copy of traces", __FILE__, __LINE__));
  for (int j = 0; j < 3; ++j) grads_out[j] = ctx->h_small[j];
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
