// Preconditioned Krylov sampler (Section 3.3, Eqs. sampling:2 and
// sampling:6-8, Algorithm 5.1): every column of the sample block is
//   x = L^-T V f(T) (eta e1),  f(t) = t^-1/2,
// with the block-Jacobi split preconditioner L = blockdiag(chol(Q_bb)), the
// Lanczos basis V and tridiagonal T of K_m(L^-1 Q L^-T, z), z the column of
// the Philox noise and eta = ||z||.  All columns advance together: one
// multi-right-hand-side SpMM per Lanczos step, per-column dot products
// reduced in double.  The basis is not stored: a first pass computes T, one
// warp per column diagonalises it (implicit QL with Wilkinson shifts, FP64)
// into the quadrature weights c = eta U f(Lambda) U^T e1, and a second pass
// regenerates the same vectors from the stored coefficients and accumulates
// x~ = sum_j c_j v_j.  FP64 throughout.
#include <cmath>

#include "qsel.h"
#include "kernels.cuh"
#include "bjblock.cuh"

namespace qsel {

// ---------------------------------------------------------------------------
// Block factor: Linv_b = chol(Q_bb)^-1 (lower triangular), b <= 64, FP64.
// A non-positive pivot sets bit 0 of *err_flag.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_bj_cholinv(SellPattern pat, BtModel m, int n_s, int n_t, int b,
                                                    double *__restrict__ linv, int32_t *err_flag) {
  extern __shared__ __align__(16) double smem_chol[];
  double *S = smem_chol;              // [64][65]
  double *X = smem_chol + 64 * 65;    // [64][65]
  assemble_diag_block(S, 65, pat, m, n_s, n_t, blockIdx.x * b, b);
  // right-looking Cholesky, lower triangle of S
  for (int k = 0; k < b; ++k) {
    if (threadIdx.x == 0) {
      const double d = S[k * 65 + k];
      if (!(d > 0.0) && err_flag) atomicOr(err_flag, 1);
      S[k * 65 + k] = sqrt(d > 0.0 ? d : 1.0);
    }
    __syncthreads();
    const double lkk = S[k * 65 + k];
    for (int i = k + 1 + threadIdx.x; i < b; i += blockDim.x) S[i * 65 + k] /= lkk;
    __syncthreads();
    const int r = b - k - 1;
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      const int i = k + 1 + e / r, j = k + 1 + e % r;
      if (j <= i) S[i * 65 + j] = fma(-S[i * 65 + k], S[j * 65 + k], S[i * 65 + j]);
    }
    __syncthreads();
  }
  // X = L^-1 by forward substitution, one column per thread
  if (threadIdx.x < b) {
    const int c = threadIdx.x;
    for (int i = 0; i < c; ++i) X[i * 65 + c] = 0.0;
    X[c * 65 + c] = 1.0 / S[c * 65 + c];
    for (int i = c + 1; i < b; ++i) {
      double acc = 0.0;
      for (int j = c; j < i; ++j) acc = fma(S[i * 65 + j], X[j * 65 + c], acc);
      X[i * 65 + c] = -acc / S[i * 65 + i];
    }
  }
  __syncthreads();
  double *L = linv + (int64_t)blockIdx.x * b * b;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e - (e / b) * b;
    L[e] = X[i * 65 + j];
  }
}

// ---------------------------------------------------------------------------
// y = B x per 64-row tile with B = blockdiag(Linv) (TRANS = false) or its
// transpose (TRANS = true); b in {16, 32, 64}.  The block is staged so that
// Bs[j][row] = B[row][j]; each thread accumulates an 8-row x 2-column tile.
// ---------------------------------------------------------------------------
template <bool TRANS>
__global__ void __launch_bounds__(256) k_block_apply(const double *__restrict__ linv, int b, int n, int ld,
                                                     const double *__restrict__ x, double *__restrict__ y) {
  constexpr int PS = 66, RS = 66, CW = 64;
  extern __shared__ __align__(16) double smem_apply[];
  double *Bs = smem_apply;            // [64][PS]
  double *xs = smem_apply + 64 * PS;  // [64][RS]
  const int tid = threadIdx.x, rg = tid >> 5, cg = tid & 31;
  const int n_blocks = (n + b - 1) / b;
  const int n_tiles = (n + 63) / 64;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int r0 = tile * 64;
    const int rows = min(64, n - r0);
    __syncthreads();
    {
      const int64_t base = (int64_t)(r0 / b) * b * b;
      const int64_t lim = (int64_t)n_blocks * b * b;
      for (int e = tid; e < 64 * b; e += blockDim.x) {
        const int blk = e / (b * b), rem = e - blk * b * b;
        const int r = rem / b, j = rem - r * b;
        const double v = (base + e < lim) ? linv[base + e] : 0.0;
        if (TRANS)
          Bs[(blk * b + r) * PS + blk * b + j] = v;     // B = Linv^T: B[j][r] = Linv[r][j]
        else
          Bs[(blk * b + j) * PS + blk * b + r] = v;     // B = Linv
      }
    }
    for (int c0 = 0; c0 < ld; c0 += CW) {
      __syncthreads();
      for (int e = tid; e < 64 * CW / 2; e += blockDim.x) {
        const int rr = e / (CW / 2), q = e - rr * (CW / 2);
        double2 val = make_double2(0.0, 0.0);
        if (rr < rows) val = *reinterpret_cast<const double2 *>(x + (int64_t)(r0 + rr) * ld + c0 + 2 * q);
        *reinterpret_cast<double2 *>(xs + rr * RS + 2 * q) = val;
      }
      __syncthreads();
      const int row0 = rg * 8;
      const int jb = (row0 / b) * b;
      double z[8][2];
#pragma unroll
      for (int a = 0; a < 8; ++a) z[a][0] = z[a][1] = 0.0;
      // B is triangular within its block: Linv is lower (j <= row), its
      // transpose upper (j >= row); the zero half is skipped
      const int j_lo = TRANS ? row0 - jb : 0;
      const int j_hi = TRANS ? b : row0 + 8 - jb;
      for (int jj = j_lo; jj < j_hi; ++jj) {
        const int jl = jb + jj;
        const double2 *pp = reinterpret_cast<const double2 *>(Bs + jl * PS + row0);
        double pv[8];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const double2 t2 = pp[u];
          pv[2 * u] = t2.x;
          pv[2 * u + 1] = t2.y;
        }
        const double2 rv = *reinterpret_cast<const double2 *>(xs + jl * RS + 2 * cg);
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          z[a][0] = fma(pv[a], rv.x, z[a][0]);
          z[a][1] = fma(pv[a], rv.y, z[a][1]);
        }
      }
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int rl = row0 + a;
        if (rl < rows)
          *reinterpret_cast<double2 *>(y + (int64_t)(r0 + rl) * ld + c0 + 2 * cg) = make_double2(z[a][0], z[a][1]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Lanczos vector kernels.  Rows are split across CTAs; within a CTA, 64
// consecutive columns x 4 row groups; per-CTA partial column sums in double
// are reduced in a fixed order by k_lz_reduce.  Columns >= k are held at 0.
// ---------------------------------------------------------------------------
constexpr int kLzGrid = 152 * 4;

int lz_grid(int n) {
  const int g = (n + 63) / 64;
  return g < kLzGrid ? g : kLzGrid;
}

// MODE 0: w -= beta_prev vprev; [xt += coef v]; partial = v . w
// MODE 1: w -= alpha v; partial = w . w
// MODE 2: partial = w . w (norm of the start vector)
template <int MODE>
__global__ void __launch_bounds__(256) k_lz_vec(const LanczosArgs a, const double *__restrict__ vprev,
                                                const double *__restrict__ v, double *__restrict__ w,
                                                double *__restrict__ xt, const double *__restrict__ coef,
                                                const double *__restrict__ scal, double *__restrict__ partial) {
  __shared__ double red[4][64];
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int64_t rows_per = (a.n + gridDim.x - 1) / gridDim.x;
  const int64_t r_begin = blockIdx.x * rows_per;
  const int64_t r_end = min((int64_t)a.n, r_begin + rows_per);
  for (int c0 = 0; c0 < a.ld; c0 += 64) {
    const int c = c0 + tx;
    const bool live = c < a.k;
    const double sc = live ? scal[c] : 0.0;
    const double cf = (coef != nullptr && live) ? coef[c] : 0.0;
    double acc = 0.0;
    for (int64_t r = r_begin + ty; r < r_end; r += 4) {
      const int64_t e = r * a.ld + c;
      if (MODE == 0) {
        const double vv = live ? v[e] : 0.0;
        double ww = live ? fma(-sc, vprev[e], w[e]) : 0.0;
        w[e] = ww;
        if (xt != nullptr) xt[e] = live ? fma(cf, vv, xt[e]) : 0.0;
        acc = fma(vv, ww, acc);
      } else if (MODE == 1) {
        const double ww = live ? fma(-sc, v[e], w[e]) : 0.0;
        w[e] = ww;
        acc = fma(ww, ww, acc);
      } else {
        const double ww = live ? w[e] : 0.0;
        acc = fma(ww, ww, acc);
      }
    }
    red[ty][tx] = acc;
    __syncthreads();
    if (ty == 0) partial[(int64_t)blockIdx.x * a.ld + c] = red[0][tx] + red[1][tx] + red[2][tx] + red[3][tx];
    __syncthreads();
  }
}

// out[c] = sum_g partial[g][c] (SQRT: its square root); store[c] = out[c]
// when store is given.  One thread per column, fixed order.
template <bool SQRT>
__global__ void k_lz_reduce(const LanczosArgs a, const double *__restrict__ partial, int n_part,
                            double *__restrict__ out, double *__restrict__ store) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.ld) return;
  double s = 0.0;
  for (int g = 0; g < n_part; ++g) s += partial[(int64_t)g * a.ld + c];
  if (c >= a.k) s = 0.0;
  const double r = SQRT ? sqrt(s) : s;
  out[c] = r;
  if (store) store[c] = r;
}

// w *= 1 / scal (0 where scal vanishes: breakdown or an empty column)
__global__ void k_lz_scale(const LanczosArgs a, double *__restrict__ w, const double *__restrict__ scal) {
  const int64_t total = (int64_t)a.n * a.ld;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % a.ld);
    const double s = scal[c];
    w[e] = (c < a.k && s > 1e-300) ? w[e] / s : 0.0;
  }
}

// ---------------------------------------------------------------------------
// Quadrature weights: for each column (one warp), T = tridiag(beta, alpha,
// beta) of size m_c (the steps before a breakdown), T = U Lambda U^T by the
// implicit QL algorithm with Wilkinson shifts (rotations applied to U by all
// lanes), then coef[j] = eta sum_i lambda_i^-1/2 U[0][i] U[j][i].
// Failures (an iteration limit, a non-positive eigenvalue) set bit 3 of
// *err_flag and zero the column's weights.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32) k_lz_quadrature(const LanczosArgs a, const double *__restrict__ alpha,
                                                      const double *__restrict__ beta, const double *__restrict__ eta,
                                                      double *__restrict__ dwork, double *__restrict__ U,
                                                      double *__restrict__ coef, int32_t *err_flag) {
  const int c = blockIdx.x;
  const int lane = threadIdx.x;
  const int m = a.m;
  double *d = dwork + (int64_t)c * 2 * m;
  double *e = d + m;
  double *Z = U + (int64_t)c * m * m;          // Z[r * m + j]
  if (c >= a.k || !(eta[c] > 0.0)) {
    for (int j = lane; j < m; j += 32) coef[(int64_t)j * a.ld + c] = 0.0;
    return;
  }
  // effective size: stop after the first vanishing beta
  int mc = m;
  for (int j = 0; j < m - 1; ++j)
    if (!(beta[(int64_t)j * a.ld + c] > 1e-300)) {
      mc = j + 1;
      break;
    }
  for (int j = 0; j < mc; ++j) {
    d[j] = alpha[(int64_t)j * a.ld + c];
    e[j] = (j + 1 < mc) ? beta[(int64_t)j * a.ld + c] : 0.0;
  }
  for (int r = lane; r < mc; r += 32)
    for (int j = 0; j < mc; ++j) Z[(int64_t)r * m + j] = (r == j) ? 1.0 : 0.0;
  __syncwarp();
  // every lane runs the same scalar recurrence on d and e (and writes the
  // same values), so no lane reads another lane's write there; the rows of Z
  // are split across the lanes
  bool failed = false;
  for (int l = 0; l < mc && !failed; ++l) {
    int iter = 0;
    for (;;) {
      int mm = l;
      for (; mm < mc - 1; ++mm) {
        const double dd = fabs(d[mm]) + fabs(d[mm + 1]);
        if (fabs(e[mm]) <= 2.3e-16 * dd) break;
      }
      if (mm == l) break;
      if (++iter > 60) {
        failed = true;
        break;
      }
      // Wilkinson shift from the leading 2 x 2 block
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = hypot(g, 1.0);
      g = d[mm] - d[l] + e[l] / (g + copysign(r, g));
      double s = 1.0, cs = 1.0, p = 0.0;
      bool early = false;
      for (int i = mm - 1; i >= l; --i) {
        const double f = s * e[i], bb = cs * e[i];
        r = hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {
          d[i + 1] -= p;
          e[mm] = 0.0;
          early = true;
          break;
        }
        s = f / r;
        cs = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * cs * bb;
        p = s * r;
        d[i + 1] = g + p;
        g = cs * r - bb;
        // rotate columns i, i + 1 of Z (each lane its own rows)
        for (int row = lane; row < mc; row += 32) {
          const double z1 = Z[(int64_t)row * m + i + 1];
          const double z0 = Z[(int64_t)row * m + i];
          Z[(int64_t)row * m + i + 1] = s * z0 + cs * z1;
          Z[(int64_t)row * m + i] = cs * z0 - s * z1;
        }
      }
      if (early) continue;
      d[l] -= p;
      e[l] = g;
      e[mm] = 0.0;
    }
  }
  __syncwarp();
  for (int i = 0; i < mc && !failed; ++i)
    if (!(d[i] > 0.0)) failed = true;
  if (failed) {
    if (lane == 0 && err_flag) atomicOr(err_flag, 8);
    for (int j = lane; j < m; j += 32) coef[(int64_t)j * a.ld + c] = 0.0;
    return;
  }
  const double et = eta[c];
  for (int j = lane; j < m; j += 32) {
    double acc = 0.0;
    if (j < mc)
      for (int i = 0; i < mc; ++i) acc += Z[i] / sqrt(d[i]) * Z[(int64_t)j * m + i];
    coef[(int64_t)j * a.ld + c] = et * acc;
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
void launch_bj_cholinv(cudaStream_t s, const SellPattern &pat, const BtModel &m, int n_s, int n_t, int b,
                       double *linv, int32_t *err_flag) {
  constexpr int smem = 2 * 64 * 65 * (int)sizeof(double);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_bj_cholinv, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  ++g_launch_count;
  const int nblk = (n_s * n_t + b - 1) / b;
  k_bj_cholinv<<<nblk, 256, smem, s>>>(pat, m, n_s, n_t, b, linv, err_flag);
}

void launch_block_apply(cudaStream_t s, const double *linv, int b, int n, int ld, const double *x, double *y,
                        bool trans) {
  constexpr int smem = 2 * 64 * 66 * (int)sizeof(double);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_block_apply<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_block_apply<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  ++g_launch_count;
  const int tiles = (n + 63) / 64;
  const int grid = tiles < 152 * 4 ? tiles : 152 * 4;
  if (trans)
    k_block_apply<true><<<grid, 256, smem, s>>>(linv, b, n, ld, x, y);
  else
    k_block_apply<false><<<grid, 256, smem, s>>>(linv, b, n, ld, x, y);
}

void launch_lz_vec(cudaStream_t s, int mode, const LanczosArgs &a, const double *vprev, const double *v, double *w,
                   double *xt, const double *coef, const double *scal, double *partial) {
  ++g_launch_count;
  const int grid = lz_grid(a.n);
  if (mode == 0)
    k_lz_vec<0><<<grid, 256, 0, s>>>(a, vprev, v, w, xt, coef, scal, partial);
  else if (mode == 1)
    k_lz_vec<1><<<grid, 256, 0, s>>>(a, vprev, v, w, xt, coef, scal, partial);
  else
    k_lz_vec<2><<<grid, 256, 0, s>>>(a, vprev, v, w, xt, coef, scal, partial);
}

void launch_lz_reduce(cudaStream_t s, const LanczosArgs &a, const double *partial, bool sqrt_out, double *out,
                      double *store) {
  ++g_launch_count;
  const int grid = (a.ld + 127) / 128;
  if (sqrt_out)
    k_lz_reduce<true><<<grid, 128, 0, s>>>(a, partial, lz_grid(a.n), out, store);
  else
    k_lz_reduce<false><<<grid, 128, 0, s>>>(a, partial, lz_grid(a.n), out, store);
}

void launch_lz_scale(cudaStream_t s, const LanczosArgs &a, double *w, const double *scal) {
  ++g_launch_count;
  const int64_t total = (int64_t)a.n * a.ld;
  const int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
  k_lz_scale<<<grid, 256, 0, s>>>(a, w, scal);
}

void launch_lz_quadrature(cudaStream_t s, const LanczosArgs &a, const double *alpha, const double *beta,
                          const double *eta, double *dwork, double *U, double *coef, int32_t *err_flag) {
  ++g_launch_count;
  k_lz_quadrature<<<a.ld, 32, 0, s>>>(a, alpha, beta, eta, dwork, U, coef, err_flag);
}

}  // namespace qsel
