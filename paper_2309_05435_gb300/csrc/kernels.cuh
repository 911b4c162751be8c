// Host-side launchers of the library's kernels (internal interface).
//
// Kernels that move sample blocks or dense blocks are templated on the
// storage/arithmetic type T (double for the FP64 path, float for the mixed
// path); reductions, pivots and the spatial pattern values stay in double.
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
enum ProfKind {
  PROF_GEMM = 0,      // dense tile GEMMs (CUDA-core and tcgen05)
  PROF_SWEEP = 1,     // updates of the blocked sweep (rank 64, or rank 64 kSweepPanel per panel)
  PROF_SPMM = 2,      // block-tridiagonal SpMM
  PROF_PIVOT = 3,     // 64x64 pivot-tile inverses (FP64)
  PROF_PANEL = 4,     // sweep panels: gathers, panel steps and patches, scatters, mirror
  PROF_SCHUR = 5,     // Schur assembly of the pivot blocks
  PROF_GATHER = 6,    // sparse row / column gathers
  PROF_PRECOND = 7,   // preconditioner apply (block Jacobi, or the Kronecker passes) with the PCG dots
  PROF_PCGVEC = 8,    // PCG axpy, direction update, reductions, refinement
  PROF_CORR = 9,      // RB correction terms
  PROF_EXTRACT = 10,  // diagonal and pattern extraction of Sigma blocks
  PROF_KINDS = 11
};
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
// Times the launches issued during its lifetime as one record of `kind`.
struct ProfScope {
  Profiler::Rec rec;
  cudaStream_t s;
  Profiler *p;
  ProfScope(cudaStream_t s_, int kind, double work = 0.0) : rec{kind, nullptr, nullptr, work}, s(s_), p(g_prof) {
    if (p) p->begin(s, rec);
  }
  ~ProfScope() {
    if (p) p->end(s, rec);
  }
};

// Message returned by qsel_last_error(NULL) for calls without a context.
void set_context_free_error(const std::string &msg);

// ---------------------------------------------------------------- model.cu
// theta_dev: (log kappa, log tau, logit rho) in device memory, so that a
// captured graph reads the current theta at every replay
void launch_time_coeffs(cudaStream_t s, const double *theta_dev, int n_t, TimeCoeffs tc);
void launch_qs_values(cudaStream_t s, int n_ent, const double *c_pat, const double *g_pat,
                      const double *h_pat, const double *isqc_pat, const double *scalars,
                      double *qs, double *dqs, double *kc);

// Per-block values of the diffusion model for theta_dev = (log gamma_s, log
// gamma_t, log gamma_e); layout of blk and coef in model.cu.
void launch_diffusion_values(cudaStream_t s, const double *theta_dev, int n_t, int n_ent, const double *c_pat,
                             const double *g_pat, const double *h_pat, const double *h3_pat, double *blk,
                             double *coef);

// ---------------------------------------------------------------- sampler.cu
void launch_philox_normals(cudaStream_t s, uint64_t seed, uint32_t stream_id, int n_rows, int k,
                           int ld, double *z);
void launch_perturbation_rhs(cudaStream_t s, const SellPattern &pat, const double *kc, int n_s,
                             int n_t, int ld, const double *bdiag, const double *scalars,
                             const double *z1, const double *z2, const int32_t *obs_index,
                             double inv_sigma, double *r);

template <typename T>
struct BtSpmmArgs {
  SellPattern pat;
  BtModel m;              // the block-tridiagonal matrix
  int n_s, n_t, ld;
  const T *x;
  T *y;
  double *dot_partial;    // if non-null: per-CTA per-column partial sums of x*y
  T *tmp = nullptr;       // if non-null and the model is separable (one spatial
                          // array scaled per block): n x ld scratch for the
                          // time combination
};
// Number of dot-partial rows launch_bt_spmm writes.
int bt_spmm_grid(int n_rows);
template <typename T>
void launch_bt_spmm(cudaStream_t s, const BtSpmmArgs<T> &a);

template <typename T>
struct PcgVec {
  int n, ld, n_blocks_dot, n_tiles;
  T *x, *r, *z, *p, *q;
  double *partial_a, *partial_b;      // reduction scratch
  double *alpha, *beta, *rho, *bb, *rr;
  int32_t *active;
  int32_t *counters;                  // [0] active columns
  double *max_rel;                    // [0] max relative residual
  const double *tol2_dev = nullptr;   // squared stopping tolerance in device memory (overrides the argument)
};
// Device-driven loops of captured graphs: the condition of a while node is
// set by these kernels from the active-column count.
//   loop[0] iterations of the current solve, loop[1] completed refinement
//   steps, loop[2] total inner iterations, loop[3] status (0 or QSEL_ENOCONV)
void launch_loop_init(cudaStream_t s, cudaGraphConditionalHandle h, const int32_t *counters, int32_t *loop,
                      int max_iter);
void launch_loop_ctl(cudaStream_t s, cudaGraphConditionalHandle h, const int32_t *counters, int32_t *loop, int step,
                     int max_iter);
void launch_loop_status(cudaStream_t s, const int32_t *counters, int32_t *loop);
void launch_refine_ctl(cudaStream_t s, cudaGraphConditionalHandle h, const int32_t *counters,
                       const double *max_rel, int32_t *loop, int first, int max_outer, int max_iter, double tol,
                       double inner_floor, double *tol2_dev);
template <typename T>
void launch_jacobi_setup(cudaStream_t s, const SellPattern &pat, const BtModel &m, int n_s, int n_t, int bsize,
                         T *pblk, int32_t *err_flag);
// Grid of the PCG update (also the number of its partial rows, PcgVec::n_tiles).
int pcg_update_grid(int n);
struct KronOperator;
// x += alpha p, r -= alpha q, then z = P r (block Jacobi with pblk, bsize) or,
// with kron, z = M^-1 r (the Kronecker preconditioner, q as scratch); the
// per-column partial sums <r, z>, <r, r>.
template <typename T>
void launch_pcg_update(cudaStream_t s, const PcgVec<T> &v, const T *pblk, int bsize, const KronOperator *kron = nullptr);
template <typename T>
void launch_pcg_reduce_alpha(cudaStream_t s, const PcgVec<T> &v);
template <typename T>
void launch_pcg_reduce_beta(cudaStream_t s, const PcgVec<T> &v, double tol, int init);
template <typename T>
void launch_pcg_p_update(cudaStream_t s, const PcgVec<T> &v);

// Mixed-precision refinement: r = b - y (FP64) with per-CTA per-column
// partial sums of r^2 and b^2, and the FP32 copy of r.
int residual_grid(int n);
void launch_residual(cudaStream_t s, const double *b, const double *y, double *r, float *r32, int n,
                     int ld, double *partial_rr, double *partial_bb);
// Per-column totals of the partials and the number of columns with
// ||r_c|| > tol ||b_c|| (counters[0]); max relative residual in max_rel[0].
void launch_residual_check(cudaStream_t s, const double *partial_rr, const double *partial_bb, int n_parts,
                           int ld, double tol, int32_t *counters, double *max_rel);
// x += (double) d
void launch_accumulate(cudaStream_t s, double *x, const float *d, int64_t count);

// ---------------------------------------------------------------- dense.cu
constexpr int kMaxBatch = 16;

template <typename T>
struct GemmEntry {
  const T *A, *B, *C0;
  T *C;
  double alpha, beta;
};
template <typename T>
struct GemmBatch {
  GemmEntry<T> e[kMaxBatch];
  int count;
};
// C = alpha A B + beta C0 for row-major M x K and K x N operands (multiples of
// 64); lower = only tiles on or below the diagonal.
template <typename T>
void launch_gemm(cudaStream_t s, const GemmBatch<T> &b, int M, int N, int K, int lda, int ldb, int ldc,
                 bool lower);

// Pivot tiles per panel of the tensor-core sweep (the rank of its updates is
// 64 kSweepPanel).
constexpr int kSweepPanel = 4;

template <typename T>
struct SweepEntry {
  T *A;          // n_pad x n_pad, row-major, lower tiles used
  T *P;          // 64 x 64 scratch (tensor-core path: 2 kSweepPanel of them, one
                 // per panel parity and pivot)
  T *U, *V;      // n_pad x 64 scratch each (tile-major)
  // tensor-core path, one set per panel parity: the products U, the pivot
  // columns V and the column panel W, n_pad x 64 kSweepPanel each (row-major)
  T *Up[2], *Vp[2], *Wp[2];
  T *Vk;         // tensor-core path: 2 kSweepPanel blocks of 64 kSweepPanel x 64 (the
                 // panel rows of the pivot column, per panel parity and pivot)
  T *Sp[4];      // tensor-core path: the panel update's U and V split into TF32 hi / lo
                 // (U_hi, U_lo, V_hi, V_lo; n_pad x 64 kSweepPanel each), or null
};
// Streams and events of the tensor-core sweep's look-ahead: the pivot chain
// (pivots, the panel's and the next panel's rows) runs on hi (high priority);
// the other rows' panel steps and look-ahead, the rank-64 kSweepPanel updates
// and the scatters on lo.  panel: hi's part of a panel done; lookahead: lo's
// look-ahead rows written; scatter: the panel back in A.
struct SweepStreams {
  cudaStream_t hi = nullptr, lo = nullptr;
  cudaEvent_t fork = nullptr, panel = nullptr, lookahead = nullptr, scatter = nullptr;
};
template <typename T>
struct SweepBatch {
  SweepEntry<T> e[kMaxBatch];
  int count;
  int pivot_fp64;  // float tiles: pivot inverses in binary64 instead of double-float
};
// In-place SPD inverse by the blocked symmetric sweep; A becomes A^-1 with
// both triangles filled.  The 64 x 64 pivot tiles are inverted in double
// (double tiles) or double-float (float tiles).  err_flag gets bit 0 on a non-positive pivot.  For float with
// tc_passes > 0 the pivots are taken kSweepPanel at a time on a gathered column
// panel and the rest of the matrix gets one rank-64 kSweepPanel update per
// panel on the tcgen05 tensor cores (Up, Vp, Wp and Vk are needed).  With ss the
// next panel is pivoted on ss->hi while the update of the current one runs on
// ss->lo (both joined back into s); without it everything runs on s.
template <typename T>
void spd_inverse(cudaStream_t s, const SweepBatch<T> &b, int n_pad, int32_t *err_flag, int tc_passes = 0,
                 const SweepStreams *ss = nullptr);
// Copy the lower tiles of each e[].A into its upper triangle (symmetric fill).
template <typename T>
void launch_mirror(cudaStream_t s, const SweepBatch<T> &b, int n_pad);

template <typename TI, typename TO>
struct SpEntry {
  const TI *B;              // dense input, rows indexed by pattern columns
  const TO *C;              // optional additive input (beta term)
  TO *Out;
  const double *alpha_ptr;  // optional device scalar multiplying alpha
  double alpha, beta;
  const double *val;        // spatial values of this entry's block on the pattern
};
template <typename TI, typename TO>
struct SpBatch {
  SpEntry<TI, TO> e[kMaxBatch];
  int count;
};
// Out[i, :] = alpha (M B)[i, :] + beta C[i, :] for i < n_s with M the
// symmetric spatial block of each entry (e.val on the pattern); rows
// n_s..n_pad-1 of Out are set to beta C, or zero when C is null.  B has
// leading dimension ldb, Out and C have ldo.
template <typename TI, typename TO>
void launch_sp_rowgather(cudaStream_t s, const SpBatch<TI, TO> &b, const SellPattern &pat, int n_s, int n_pad,
                         int ncol, int ldb, int ldo);

// Out = alpha B M + beta C on n_pad x n_pad blocks (column gather).
template <typename T>
void launch_sp_colgather(cudaStream_t s, const SpBatch<T, T> &b, const SellPattern &pat, int n_s, int n_pad);

template <typename T>
struct DiagRowEntry {
  const T *D0, *P, *R;      // diag_out[i] = D0[i,i] + sum_l P[i,l] R[i,l] (double)
  double *diag_out;
};
template <typename T>
struct DiagRowBatch {
  DiagRowEntry<T> e[kMaxBatch];
  int count;
};
template <typename T>
void launch_diag64_rows(cudaStream_t s, const DiagRowBatch<T> &b, int n_s, int n_pad);

// ---------------------------------------------------------------- tc_gemm.cu
// tcgen05 tensor-core GEMM (FP32 data, TF32 MMAs): C = alpha A B^T + beta C0
// with A (M x K) and B (N x K) row-major; passes 3 = 3xTF32, 1 = TF32.
// err gets bit 1 when a bounded wait gives up.  compact: 128 x 32 tiles in
// two stages (81 KB of shared memory), so that a CTA fits on an SM beside one
// of the persistent sweep update's.
bool tc_gemm_available();
bool launch_tc_gemm(cudaStream_t s, const GemmBatch<float> &b, int M, int N, int K, int lda, int ldb, int ldc,
                    bool lower, int passes, int32_t *err, bool compact = false);
// Persistent tcgen05 update of the lower 128 x 128 tiles of n x n matrices:
// C = alpha U V^T + beta C with U, V (n x K, leading dimension ldp) given as
// TF32 hi / lo parts (3xTF32), K a multiple of 32 (tc_update.cu).  False when
// a tensor map cannot be encoded (nothing is launched then).
struct UpdateEntry {
  const float *Uh, *Ul, *Vh, *Vl;
  float *C;
};
struct UpdateBatch {
  UpdateEntry e[kMaxBatch];
  int count;
};
bool launch_tc_update(cudaStream_t s, const UpdateBatch &b, int n, int K, int ldp, float alpha, float beta,
                      int32_t *err, int max_ctas = 0);
// C = alpha A B^T + beta C0 on operands given as TF32 hi / lo parts (A: M x K,
// B: N x K, row-major; K a multiple of 32, leading dimensions multiples of 4):
// the persistent 128 x 256-tile kernel of tc_gemm2.cu.  lower = only the tiles
// on or below the diagonal.  False when a tensor map cannot be encoded
// (nothing is launched then).
struct SplitGemmEntry {
  const float *Ah, *Al, *Bh, *Bl;
  const float *C0;
  float *C;
  float alpha, beta;
  int rows = 0, cols = 0;   // this entry's M and N (0: the launch's M and N); full tiles only
};
struct SplitGemmBatch {
  SplitGemmEntry e[kMaxBatch];
  int count;
};
bool launch_tc_gemm_split(cudaStream_t s, const SplitGemmBatch &b, int M, int N, int K, int lda, int ldb, int ldc,
                          bool lower, int32_t *err, int max_ctas = 0);
// hi = rn_tf32(x), lo = rn_tf32(x - hi) elementwise (16-byte aligned arrays).
void launch_split_tf32(cudaStream_t s, const float *src, float *hi, float *lo, int64_t count);
// the same for up to 2 kMaxBatch arrays of `count` floats each (count a
// multiple of 4, 16-byte aligned arrays), in one launch
struct SplitJob {
  const float *src;
  float *hi, *lo;
  int64_t count;   // floats, a multiple of 4 (0: the launch's count)
};
struct SplitJobs {
  SplitJob j[2 * kMaxBatch];
  int count;
};
void launch_split_tf32_jobs(cudaStream_t s, const SplitJobs &jobs, int64_t count);
// out[r, c] = alpha in[c, r] + beta c0[r, c] for each entry (see dense.cu).
struct TransEntry {
  const float *in, *c0;
  float *out;
  float alpha, beta;
};
struct TransBatch {
  TransEntry e[kMaxBatch];
  int count;
};
void launch_transpose_axpby(cudaStream_t s, const TransBatch &b, int rows, int cols, int ld_in, int ld_out);
// C = alpha A B + beta C0 on the tensor cores for an n_pad x n_pad A
// (b.e[].A) and row-major n_pad x ld blocks B, C0, C: Bt = B^T, then the
// K-major product Pt = Bt A^T (= (A B)^T, A row-major serves as the N x K
// operand), C = alpha Pt^T + beta C0; bt[q], pt[q] are ld x n_pad scratch.
// False when a tensor map cannot be encoded.
bool launch_symm_block_tc(cudaStream_t s, const GemmBatch<float> &b, float *const *bt, float *const *pt, int n_pad,
                          int ld, int passes, int32_t *err);

template <typename T>
struct SchurEntry {
  const T *W;               // W_{t-1} = B_{t-1} Dinv_{t-1} (null for the first slab)
  T *D;                     // output diagonal block
  const double *dval;       // spatial values of A_t on the pattern
  const double *a0;         // device scale of A_t, or null (1)
  const double *cval;       // spatial values of B_{t-1} on the pattern (ignored if W null)
  const double *c;          // device scale of B_{t-1}, or null (1)
  const uint8_t *obs;       // mask of slab t (n_s entries), or null
  int accumulate;           // 1: D -= c W B^T on the n_s x n_s block only (a second
                            // neighbour's term; dval, a0, obs ignored)
};
template <typename T>
struct SchurBatch {
  SchurEntry<T> e[kMaxBatch];
  int count;
};
template <typename T>
void launch_schur_assemble(cudaStream_t s, const SchurBatch<T> &b, const SellPattern &pat, double obs_w, int n_s,
                           int n_pad);
// The row / column gathers and the Schur assembly stage each row's or
// column's pattern in shared memory; widest pattern they accept, and the
// opt-in of those kernels to the shared memory pat.max_width needs.
constexpr int kMaxPatternWidth = 64;
// scheduling hook of the panel-blocked sweep (qsel_debug_sweep_schedule)
int sweep_serial();
int update_cta_cap();
int update_stages();
int pivot_exclusive();
bool configure_pattern_kernels(const SellPattern &pat);

template <typename T>
struct ExtractEntry {
  const T *S;               // n_pad x n_pad dense
  double *diag_out;         // n_s outputs (null: skip)
  double *sums;             // n_sums outputs <sv[j], S>_pattern (null: skip)
  const double *sv[kMaxTheta];  // spatial values of the derivative blocks
  // optional FP64 diagonal: when D0 is set, diag_out gets
  // D0[i,i] + sum_l D0[i,l] V[l,i] accumulated in double instead of S[i,i]
  const T *D0, *V;
};
template <typename T>
struct ExtractBatch {
  ExtractEntry<T> e[kMaxBatch];
  int count;
};
// diag_scratch: extract_scratch_bytes(n_pad) bytes of device memory (used when
// an entry sets D0).
size_t extract_scratch_bytes(int n_pad);
template <typename T>
void launch_extract(cudaStream_t s, const ExtractBatch<T> &b, const SellPattern &pat, int n_sums, int n_s,
                    int n_pad, double *diag_scratch);

// ---------------------------------------------------------------- rbmc.cu
template <typename T>
struct CorrEntry {
  const T *w;               // T_ x n_pad x ld samples of the subdomain correction
  int T_, lo, hi, e0;       // slabs, local own range [lo, hi], global slab of local 0
  double *corr_out;         // global correction output (own rows written)
  double *corr4_out;        // (1/k) sum w^4 of the own rows, or nullptr
  double *partial;          // per-CTA trace partials (kMaxTheta per CTA)
};
template <typename T>
struct CorrBatch {
  CorrEntry<T> e[kMaxBatch];
  int count;
};
int corr_grid();
template <typename T>
void launch_correction_terms(cudaStream_t s, const CorrBatch<T> &b, const SellPattern &pat, const DerivModels &dm,
                             int n_s, int n_pad, int ld, int k);
struct TraceSlab {
  int t;            // global slab of the row block
  int sd, sy, sym;  // indices into sums: Sigma_tt, Y_t (pair t,t+1), Y_{t-1} (pair t-1,t); -1 = absent
};
// sums: kMaxTheta per index; partials: kMaxTheta per CTA; out: dm.n traces
void launch_trace_combine(cudaStream_t s, const TraceSlab *slabs_dev, int n_slabs, const double *sums,
                          const double *partials, int n_partials, const DerivModels &dm, double *out);
template <typename T>
void launch_add(cudaStream_t s, T *y, const T *x, int64_t n);
// out = a + b (n doubles)
void launch_sum(cudaStream_t s, double *out, const double *a, const double *b, int n);
// per part: sum over own rows of ((m4 - m2^2) / (k - 1)) / v^2
void launch_part_error_sums(cudaStream_t s, const double *m2, const double *m4, const double *v,
                            const int32_t *slab_start_dev, int n_parts, int n_s, int k, double *out);

// ---------------------------------------------------------------- kron.cu
enum KronMode { KRON_NONE = 0, KRON_IN_DH = 1, KRON_OUT_DH = 2, KRON_OUT_SPEC = 3 };
// One pass y_g = op(B) x_g over the groups g of rows base(g) + k kstride.
struct KronPass {
  const void *Bt;           // op(B)^T, dim x dim row-major, in the pass's element type
  int dim, mode, m;
  int64_t kstride;          // rows between consecutive k
  int n_outer, n_inner;
  int64_t outer_stride, inner_stride;   // base(g) = (g / n_inner) outer + (g % n_inner) inner
  int ld;
  const void *scale;        // KRON_IN_DH / KRON_OUT_DH: dh_k dh_g (m x m);
                            // KRON_OUT_SPEC: the spectral scaling (n_t x m^2)
};
// The preconditioner's factors (device arrays) and scalars for one theta.
struct KronOperator {
  int m, n_t, ld;
  const double *V, *U, *dh, *lam, *mu;
  double kappa2, tau, omega;
  // tables in the sampler's element type, rebuilt by launch_kron_tables:
  // V, V^T, U, U^T, dh_i dh_j (m x m), spec[t m^2 + s] = 1 / (tau mu_t
  // (kappa^2 + lambda_a + lambda_b)^2 + omega) with s = a m + b
  void *tV, *tVT, *tU, *tUT, *dhdh, *spec;
  // tensor-core passes (float tables only): V, V^T, U, U^T split into TF32
  // hi / lo parts, [table][hi, lo]; use_tc selects them; err gets bit 1 when
  // a bounded wait of the tensor-core pass gives up
  float *split[4][2];
  int use_tc;
  int32_t *err;
};
// The whole apply z = M^-1 r on the tcgen05 tensor cores (kron_tc.cu), q as
// scratch; false when the shape is not supported or a tensor map cannot be
// encoded (nothing is launched then).
bool kron_tc_supported(int dim, int ld);
bool launch_kron_apply_tc(cudaStream_t s, const KronOperator &op, const float *r, float *q, float *z);
template <typename T>
void launch_kron_tables(cudaStream_t s, const KronOperator &op);
template <typename T>
void launch_kron_pass(cudaStream_t s, const KronPass &p, const T *x, T *y);
template <typename T>
void launch_kron_apply(cudaStream_t s, const KronOperator &op, const T *r, T *q, T *z);
template <typename T>
void launch_pcg_dots(cudaStream_t s, const PcgVec<T> &v);

// ---------------------------------------------------------------- hyper.cu
// Posterior mean and hyperparameter gradient (see hyper.cu).
void launch_data_rhs(cudaStream_t s, double *R, int ld, const uint8_t *obs, const int32_t *obs_index,
                     const double *y, int n, double inv_s2);
void launch_column_sum(cudaStream_t s, const double *partial, int rows, int ld, int col, double *out);
void launch_dense_K(cudaStream_t s, double *K, int n_pad, const SellPattern &pat, const double *c_pat,
                    const double *g_pat, const double *theta, int n_s);
void launch_loglik_combine(cudaStream_t s, const double *Kinv, int n_pad, const double *c_diag, int n_s, int n_t,
                           const double *theta, const double *traces, const double *extra, const double *quad,
                           double *grad, double *terms);
// fixed effects (see hyper.cu)
void launch_fe_rhs(cudaStream_t s, double *R, int ld, const int32_t *obs_nodes, const double *Z, int n_obs,
                   int n_beta, double inv_s2);
void launch_fe_schur(cudaStream_t s, const double *X, int ld, const int32_t *obs_nodes, const double *Z,
                     const double *y, int n_obs, int n_beta, double inv_s2, double beta_prec, double *S, double *m);
void launch_fe_solve(cudaStream_t s, const double *S, const double *m, int n_beta, double *Sinv, double *mu_beta,
                     int32_t *err_flag);
void launch_fe_mean(cudaStream_t s, double *X, int ld, int n, int n_beta, const double *mu_beta, const double *Sinv,
                    double *mu, double *corr);
void launch_fe_schur_trace(cudaStream_t s, const double *X, const double *Y, int ld, int n, int n_beta,
                           const double *Sinv, double *C, double *out);

// ---------------------------------------------------------------- lanczos.cu
struct LanczosArgs {
  int n, ld, k, m;
};
int lz_grid(int n);
void launch_bj_cholinv(cudaStream_t s, const SellPattern &pat, const BtModel &m, int n_s, int n_t, int b,
                       double *linv, int32_t *err_flag);
void launch_block_apply(cudaStream_t s, const double *linv, int b, int n, int ld, const double *x, double *y,
                        bool trans);
void launch_lz_vec(cudaStream_t s, int mode, const LanczosArgs &a, const double *vprev, const double *v, double *w,
                   double *xt, const double *coef, const double *scal, double *partial);
void launch_lz_reduce(cudaStream_t s, const LanczosArgs &a, const double *partial, bool sqrt_out, double *out,
                      double *store);
void launch_lz_scale(cudaStream_t s, const LanczosArgs &a, double *w, const double *scal);
void launch_lz_quadrature(cudaStream_t s, const LanczosArgs &a, const double *alpha, const double *beta,
                          const double *eta, double *dwork, double *U, double *coef, int32_t *err_flag);

// ---------------------------------------------------------------- mlp.cu
void launch_cv_features(cudaStream_t s, const SellPattern &pat, const BtModel &m, int n_s, int n_t,
                        const float *sep_dist, const float *bnd_dist, const double th[3], float *F);
void launch_cv_part_m2(cudaStream_t s, const float *y, const int32_t *slab_start_dev, int n_parts, int n_s,
                       double *out);
constexpr int kCvMaxTargets = 8;
struct CvTargetArgs {
  const double *corr[kCvMaxTargets];
  int count;
};
void launch_cv_targets(cudaStream_t s, const CvTargetArgs &a, const double *sel, int n, float *y);

}  // namespace qsel
