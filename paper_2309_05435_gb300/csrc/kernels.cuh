// Host-side launchers of the library's kernels (internal interface).
#pragma once

#include <string>
#include <vector>

#include "common.cuh"

namespace qsel {

// Every launcher increments this counter (reported in qsel_stats).
extern thread_local int64_t g_launch_count;

// Opt-in per-launch timing of the hot kernels: CUDA events recorded on the
// launching stream around each launch, with the algorithmic work of the launch
// (FLOPs or bytes).  Read back after the pipeline has synchronised.
enum ProfKind { PROF_GEMM = 0, PROF_SWEEP = 1, PROF_SPMM = 2, PROF_KINDS = 3 };
struct Profiler {
  struct Rec {
    int kind;
    cudaEvent_t a, b;
    double work;
  };
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<Rec> recs;
  cudaEvent_t take() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
  void begin(cudaStream_t s, Rec &r) {
    r.a = take();
    cudaEventRecord(r.a, s);
  }
  void end(cudaStream_t s, Rec &r) {
    r.b = take();
    cudaEventRecord(r.b, s);
    recs.push_back(r);
  }
  void reset() {
    used = 0;
    recs.clear();
  }
  ~Profiler() {
    for (auto e : pool) cudaEventDestroy(e);
  }
};
extern thread_local Profiler *g_prof;

// Message returned by qsel_last_error(NULL) for calls without a context.
void set_context_free_error(const std::string &msg);

// ---------------------------------------------------------------- model.cu
// Time-structure scalars from theta (one thread).
void launch_time_coeffs(cudaStream_t s, double log_kappa, double log_tau, double logit_rho,
                        int n_t, TimeCoeffs tc);
// Values of Q_s, dQ_s/dlog kappa and K C^-1/2 on the sliced pattern.
void launch_qs_values(cudaStream_t s, int n_ent, const double *c_pat, const double *g_pat,
                      const double *h_pat, const double *isqc_pat, const double *scalars,
                      double *qs, double *dqs, double *kc);

// ---------------------------------------------------------------- sampler.cu
// Standard normals (Philox4x32-10 + Box-Muller), n_rows x ld, zero in
// columns [k, ld).
void launch_philox_normals(cudaStream_t s, uint64_t seed, uint32_t stream_id, int n_rows, int k,
                           int ld, double *z);
// Perturbation RHS r = F^T z1 + A^T z2 / sigma.
void launch_perturbation_rhs(cudaStream_t s, const SellPattern &pat, const double *kc, int n_s,
                             int n_t, int ld, const double *bdiag, const double *scalars,
                             const double *z1, const double *z2, const int32_t *obs_index,
                             double inv_sigma, double *r);

struct BtSpmmArgs {
  SellPattern pat;
  const double *val;      // spatial values on the pattern
  const double *c0;       // diagonal-block time coefficient per slab
  const double *c1;       // off-diagonal time coefficient per slab pair (t, t+1)
  const uint8_t *obs;     // observation mask (may be null)
  double obs_w;           // weight of the observation diagonal
  int n_s, n_t, ld;
  const double *x;
  double *y;
  double *dot_partial;    // if non-null: per-CTA per-column partial sums of x*y
};
int bt_spmm_grid(int n_rows);
void launch_bt_spmm(cudaStream_t s, const BtSpmmArgs &a);

struct PcgVec {
  int n, ld, n_blocks_dot, n_tiles;
  double *x, *r, *z, *p, *q, *b;
  double *partial_a, *partial_b;      // reduction scratch
  double *alpha, *beta, *rho, *bb, *rr;
  int32_t *active;
  int32_t *counters;                  // [0] active columns
  double *max_rel;                    // [0] max relative residual
};
void launch_jacobi_setup(cudaStream_t s, const SellPattern &pat, const double *qs, const double *a0,
                         const double *a1, const uint8_t *obs, double obs_w, int n_s, int n_t,
                         int bsize, double *pblk, int32_t *err_flag);
void launch_pcg_update(cudaStream_t s, const PcgVec &v, const double *pblk, int bsize);
void launch_pcg_reduce_alpha(cudaStream_t s, const PcgVec &v);
void launch_pcg_reduce_beta(cudaStream_t s, const PcgVec &v, double tol, int init);
void launch_pcg_p_update(cudaStream_t s, const PcgVec &v);

// ---------------------------------------------------------------- dense.cu
constexpr int kMaxBatch = 16;

struct GemmEntry {
  const double *A, *B, *C0;
  double *C;
  double alpha, beta;
};
struct GemmBatch {
  GemmEntry e[kMaxBatch];
  int count;
};
// C = alpha A B + beta C0 for row-major M x K and K x N operands (multiples of
// 64); lower = only tiles on or below the diagonal.
void launch_gemm(cudaStream_t s, const GemmBatch &b, int M, int N, int K, int lda, int ldb, int ldc,
                 bool lower);

struct SweepEntry {
  double *A;          // n_pad x n_pad, row-major, lower tiles used
  double *P;          // 64 x 64 scratch
  double *U, *V;      // n_pad x 64 scratch each (tile-major)
};
struct SweepBatch {
  SweepEntry e[kMaxBatch];
  int count;
};
// In-place SPD inverse by the blocked symmetric sweep; A becomes A^-1 with
// both triangles filled.  err_flag gets bit 1 on a non-positive pivot.
void spd_inverse(cudaStream_t s, const SweepBatch &b, int n_pad, int32_t *err_flag);
// Copy the lower tiles of each e[].A into its upper triangle (symmetric fill).
void launch_mirror(cudaStream_t s, const SweepBatch &b, int n_pad);

struct SpEntry {
  const double *B;          // dense input, rows indexed by pattern columns
  const double *C;          // optional additive input (beta term)
  double *Out;
  const double *alpha_ptr;  // optional device scalar multiplying alpha
  double alpha, beta;
};
struct SpBatch {
  SpEntry e[kMaxBatch];
  int count;
};
// Out[i, :] = alpha (Q_s B)[i, :] + beta C[i, :] for i < n_s (rows n_s..n_pad-1
// of Out are set to beta C, or zero when C is null).
void launch_sp_rowgather(cudaStream_t s, const SpBatch &b, const SellPattern &pat, const double *val,
                         int n_s, int n_pad, int ncol, int ld);

struct SchurEntry {
  const double *W;          // W_{t-1} = c Q_s Dinv_{t-1} (null for the first slab)
  double *D;                // output diagonal block
  const double *a0;         // device pointer to tau Q_t[t,t]
  const double *c;          // device pointer to the coupling c_{t-1} (ignored if W null)
  const uint8_t *obs;       // mask of slab t (n_s entries)
};
struct SchurBatch {
  SchurEntry e[kMaxBatch];
  int count;
};
// D[r, l] = a0 Q_s[r, l] + w_obs obs[r] delta_rl - c (W Q_s)[r, l], identity on padding.
void launch_schur_assemble(cudaStream_t s, const SchurBatch &b, const SellPattern &pat,
                           const double *qs, double obs_w, int n_s, int n_pad);

struct ExtractEntry {
  const double *S;          // n_pad x n_pad dense
  double *diag_out;         // n_s outputs (null: skip)
  double *sums;             // 2 outputs: <dQs, S>_pattern, <Qs, S>_pattern (null: skip)
};
struct ExtractBatch {
  ExtractEntry e[kMaxBatch];
  int count;
};
void launch_extract(cudaStream_t s, const ExtractBatch &b, const SellPattern &pat, const double *qs,
                    const double *dqs, int n_s, int n_pad);

// ---------------------------------------------------------------- rbmc.cu
struct CorrEntry {
  const double *w;          // T x n_pad x ld samples of the subdomain correction
  int T, lo, hi, e0;        // local own range [lo, hi], global slab of local 0
  double *diag_out;         // global diag output (rows of own slabs added)
  double *partial;          // per-CTA trace partials (3 per CTA)
};
struct CorrBatch {
  CorrEntry e[kMaxBatch];
  int count;
};
int corr_grid();
void launch_correction_terms(cudaStream_t s, const CorrBatch &b, const SellPattern &pat,
                             const double *qs, const double *dqs, const double *a0, const double *a1,
                             const double *r0, const double *r1, int n_s, int n_pad, int ld, int k);
// Final traces: combines the selected-inverse pattern sums and the correction
// partials into 3 doubles.
struct TraceSlab {
  int t;            // global slab of the row block
  int sd, sy, sym;  // indices into sums: Sigma_tt, Y_t (pair t,t+1), Y_{t-1} (pair t-1,t); -1 = absent
};
void launch_trace_combine(cudaStream_t s, const TraceSlab *slabs_dev, int n_slabs, const double *sums,
                          const double *partials, int n_partials, const double *a0, const double *a1,
                          const double *r0, const double *r1, double *out3);
void launch_add(cudaStream_t s, double *y, const double *x, int n);
void launch_scale_copy(cudaStream_t s, double *dst, const double *src, int n, double scale);

}  // namespace qsel
