// Global samples (Section 3.3): perturbation right-hand sides from
// counter-based Gaussian noise and one multi-right-hand-side preconditioned
// conjugate-gradient solve Q X = R.
//
// Layout: every n x k block of vectors is row-major with leading dimension
// ld (a multiple of 64): row t * n_s + i holds the k samples of node i of
// slab t contiguously, so one warp reads a whole row with 16-byte loads.
#include "kernels.cuh"
#include "sweep.cuh"

namespace qsel {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplications with the Philox constants, a cross-lane xor with the key,
// and a Weyl bump of the key between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Pair (2q, 2q+1) of row i: counter (i, q, stream, 0), key = seed words.
// u1 in (0, 1] from words 0-1, u2 in [0, 1) from words 2-3 (53 bits each),
// Box-Muller: sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2).
__global__ void k_philox_normals(uint2 key, uint32_t stream_id, int n_rows, int k, int ld,
                                 double *__restrict__ z) {
  const int half = ld >> 1;
  const int64_t total = (int64_t)n_rows * half;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int row = (int)(idx / half);
    const int q = (int)(idx - (int64_t)row * half);
    double z0 = 0.0, z1 = 0.0;
    if (2 * q < k) {
      const uint4 o = philox4x32_10(make_uint4((uint32_t)row, (uint32_t)q, stream_id, 0u), key);
      const uint64_t a = ((((uint64_t)o.x) << 32) | o.y) >> 11;
      const uint64_t b = ((((uint64_t)o.z) << 32) | o.w) >> 11;
      const double u1 = ((double)a + 1.0) * 0x1.0p-53;
      const double u2 = (double)b * 0x1.0p-53;
      const double rad = sqrt(-2.0 * log(u1));
      double sn, cs;
      sincospi(2.0 * u2, &sn, &cs);
      z0 = rad * cs;
      z1 = (2 * q + 1 < k) ? rad * sn : 0.0;
    }
    double2 out = make_double2(z0, z1);
    *reinterpret_cast<double2 *>(z + (int64_t)row * ld + 2 * q) = out;
  }
}

void launch_philox_normals(cudaStream_t s, uint64_t seed, uint32_t stream_id, int n_rows, int k,
                           int ld, double *z) {
  if (n_rows <= 0) return;
  ++g_launch_count;
  const uint2 key = make_uint2((uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32));
  int64_t total = (int64_t)n_rows * (ld / 2);
  int grid = (int)((total + 255) / 256);
  if (grid > 152 * 16) grid = 152 * 16;
  k_philox_normals<<<grid, 256, 0, s>>>(key, stream_id, n_rows, k, ld, z);
}

// ---------------------------------------------------------------------------
// r = F^T z1 + A^T z2 / sigma with F = sqrt(tau / (1 - rho^2)) (B (x) M^T),
// M = K C^-1/2: block t of (B^T (x) M) z1 is B_tt M z1_t + B_{t+1,t} M z1_{t+1}.
// One warp per output row, lanes over sample columns.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_perturbation_rhs(SellPattern pat, const double *__restrict__ kc,
                                                          int n_s, int n_t, int ld,
                                                          const double *__restrict__ bdiag,
                                                          const double *__restrict__ scalars,
                                                          const double *__restrict__ z1,
                                                          const double *__restrict__ z2,
                                                          const int32_t *__restrict__ obs_index,
                                                          double inv_sigma, double *__restrict__ r) {
  const int lane = threadIdx.x & 31;
  const int n_rows = n_s * n_t;
  const double fscale = scalars[3], boff = scalars[4];
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n_rows;
       row += (gridDim.x * blockDim.x) >> 5) {
    const int t = row / n_s, i = row - t * n_s;
    const int sl = i >> 5, li = i & 31;
    const int w = pat.slice_width[sl];
    const int base = pat.slice_ptr[sl] + li;
    const double cd = fscale * bdiag[t];
    const double co = (t + 1 < n_t) ? fscale * boff : 0.0;
    const int oi = obs_index[row];
    for (int c = lane; c < ld; c += 32) {
      double acc = 0.0;
      for (int s = 0; s < w; ++s) {
        const int j = pat.col[base + s * kSlice];
        const double v = kc[base + s * kSlice];
        acc += cd * v * z1[((int64_t)t * n_s + j) * ld + c];
        if (t + 1 < n_t) acc += co * v * z1[((int64_t)(t + 1) * n_s + j) * ld + c];
      }
      if (oi >= 0) acc += z2[(int64_t)oi * ld + c] * inv_sigma;
      r[(int64_t)row * ld + c] = acc;
    }
  }
}

void launch_perturbation_rhs(cudaStream_t s, const SellPattern &pat, const double *kc, int n_s,
                             int n_t, int ld, const double *bdiag, const double *scalars,
                             const double *z1, const double *z2, const int32_t *obs_index,
                             double inv_sigma, double *r) {
  ++g_launch_count;
  int64_t rows = (int64_t)n_s * n_t;
  int grid = (int)((rows * 32 + 255) / 256);
  if (grid > 152 * 16) grid = 152 * 16;
  k_perturbation_rhs<<<grid, 256, 0, s>>>(pat, kc, n_s, n_t, ld, bdiag, scalars, z1, z2, obs_index,
                                          inv_sigma, r);
}

// ---------------------------------------------------------------------------
// Block-tridiagonal sliced-ELL SpMM over many right-hand sides:
//   y_t = sum_{d=-1,0,1} c_{t,t+d} (V x_{t+d}) + w_obs diag(obs_t) x_t
// where V is the spatial matrix on the SELL-32 pattern (Q_s here) and the
// c's are the per-slab time coefficients.  One warp per (row, 64*V2-column
// chunk); column index and value are warp-uniform broadcasts, the three
// neighbour rows are read as coalesced double2 vectors.  Optional epilogue:
// per-CTA, per-column partial sums of x .* y (the PCG curvature <p, Q p>).
// ---------------------------------------------------------------------------
constexpr int kSpmmGridMax = 152 * 8;

int bt_spmm_grid(int n_rows) {
  int g = (n_rows + 7) / 8;
  return g < kSpmmGridMax ? (g < 1 ? 1 : g) : kSpmmGridMax;
}

template <int V2>
__global__ void __launch_bounds__(256) k_bt_spmm(BtSpmmArgs a) {
  __shared__ double red[8][512];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_rows = a.n_s * a.n_t;
  const int ld = a.ld;
  const int chunk_cols = 64 * V2;
  const int nchunk = ld / chunk_cols;
  const bool dot = a.dot_partial != nullptr;
  if (dot) {
    for (int c = lane; c < ld; c += 32) red[warp][c] = 0.0;
  }
  const int64_t slab = (int64_t)a.n_s * ld;
  const int64_t items = (int64_t)n_rows * nchunk;
  for (int64_t it = (int64_t)blockIdx.x * 8 + warp; it < items; it += (int64_t)gridDim.x * 8) {
    const int row = (int)(it / nchunk);
    const int ch = (int)(it - (int64_t)row * nchunk);
    const int t = row / a.n_s, i = row - t * a.n_s;
    const int sl = i >> 5, li = i & 31;
    const int w = a.pat.slice_width[sl];
    const int base = a.pat.slice_ptr[sl] + li;
    const double c0 = a.c0[t];
    const double cm = (t > 0) ? a.c1[t - 1] : 0.0;
    const double cp = (t + 1 < a.n_t) ? a.c1[t] : 0.0;
    const int coff = ch * chunk_cols + 2 * lane;
    double2 acc[V2];
#pragma unroll
    for (int v = 0; v < V2; ++v) acc[v] = make_double2(0.0, 0.0);
    for (int s = 0; s < w; ++s) {
      const int j = a.pat.col[base + s * kSlice];
      const double val = a.val[base + s * kSlice];
      const double *xc = a.x + ((int64_t)t * a.n_s + j) * ld + coff;
      const double f0 = c0 * val;
#pragma unroll
      for (int v = 0; v < V2; ++v) {
        const double2 xv = *reinterpret_cast<const double2 *>(xc + 64 * v);
        acc[v].x = fma(f0, xv.x, acc[v].x);
        acc[v].y = fma(f0, xv.y, acc[v].y);
      }
      if (t > 0) {
        const double fm = cm * val;
#pragma unroll
        for (int v = 0; v < V2; ++v) {
          const double2 xv = *reinterpret_cast<const double2 *>(xc - slab + 64 * v);
          acc[v].x = fma(fm, xv.x, acc[v].x);
          acc[v].y = fma(fm, xv.y, acc[v].y);
        }
      }
      if (t + 1 < a.n_t) {
        const double fp = cp * val;
#pragma unroll
        for (int v = 0; v < V2; ++v) {
          const double2 xv = *reinterpret_cast<const double2 *>(xc + slab + 64 * v);
          acc[v].x = fma(fp, xv.x, acc[v].x);
          acc[v].y = fma(fp, xv.y, acc[v].y);
        }
      }
    }
    const double *xr = a.x + (int64_t)row * ld + coff;
    const double ow = (a.obs != nullptr && a.obs[row]) ? a.obs_w : 0.0;
    double *yr = a.y + (int64_t)row * ld + coff;
#pragma unroll
    for (int v = 0; v < V2; ++v) {
      double2 xv = make_double2(0.0, 0.0);
      if (ow != 0.0 || dot) xv = *reinterpret_cast<const double2 *>(xr + 64 * v);
      acc[v].x = fma(ow, xv.x, acc[v].x);
      acc[v].y = fma(ow, xv.y, acc[v].y);
      *reinterpret_cast<double2 *>(yr + 64 * v) = acc[v];
      if (dot) {
        red[warp][coff + 64 * v] += xv.x * acc[v].x;
        red[warp][coff + 64 * v + 1] += xv.y * acc[v].y;
      }
    }
  }
  if (dot) {
    __syncthreads();
    for (int c = threadIdx.x; c < ld; c += blockDim.x) {
      double sum = 0.0;
#pragma unroll
      for (int ww = 0; ww < 8; ++ww) sum += red[ww][c];
      a.dot_partial[(int64_t)blockIdx.x * ld + c] = sum;
    }
  }
}

void launch_bt_spmm(cudaStream_t s, const BtSpmmArgs &a) {
  ++g_launch_count;
  const int grid = bt_spmm_grid(a.n_s * a.n_t);
  Profiler::Rec rec{PROF_SPMM, nullptr, nullptr, 0.0};
  if (g_prof) {
    // algorithmic bytes: read x once, write y once (the spatial pattern and the
    // neighbouring rows are re-read from cache)
    rec.work = 2.0 * (double)a.n_s * a.n_t * a.ld * sizeof(double);
    g_prof->begin(s, rec);
  }
  if (a.ld % 256 == 0)
    k_bt_spmm<4><<<grid, 256, 0, s>>>(a);
  else if (a.ld % 128 == 0)
    k_bt_spmm<2><<<grid, 256, 0, s>>>(a);
  else
    k_bt_spmm<1><<<grid, 256, 0, s>>>(a);
  if (g_prof) g_prof->end(s, rec);
}

// ---------------------------------------------------------------------------
// Block-Jacobi preconditioner (Section 3.3 names block-Jacobi / IC(0)):
// contiguous blocks of b global rows; P_blk = (Q_blk)^-1 by the symmetric
// sweep in shared memory.  Rows past n are padded with the identity.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_jacobi_setup(SellPattern pat, const double *__restrict__ qs,
                                                      const double *__restrict__ a0,
                                                      const double *__restrict__ a1,
                                                      const uint8_t *__restrict__ obs, double obs_w,
                                                      int n_s, int n_t, int b,
                                                      double *__restrict__ pblk, int32_t *err_flag) {
  __shared__ double S[64 * 65];
  const int n = n_s * n_t;
  const int r0 = blockIdx.x * b;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e - (e / b) * b;
    S[i * 65 + j] = (i == j && r0 + i >= n) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int rr = threadIdx.x; rr < b; rr += blockDim.x) {
    const int row = r0 + rr;
    if (row >= n) continue;
    const int t = row / n_s, i = row - t * n_s;
    const int sl = i >> 5, li = i & 31;
    const int w = pat.slice_width[sl];
    const int base = pat.slice_ptr[sl] + li;
    for (int s = 0; s < w; ++s) {
      const int j = pat.col[base + s * kSlice];
      const double v = qs[base + s * kSlice];
      for (int d = -1; d <= 1; ++d) {
        const int u = t + d;
        if (u < 0 || u >= n_t) continue;
        const int colg = u * n_s + j;
        if (colg < r0 || colg >= r0 + b) continue;
        const double c = (d == 0) ? a0[t] : (d < 0 ? a1[t - 1] : a1[t]);
        S[rr * 65 + (colg - r0)] += c * v;
      }
    }
    if (obs != nullptr && obs[row]) S[rr * 65 + rr] += obs_w;
  }
  __syncthreads();
  sym_sweep_inverse_smem(S, 65, b, err_flag);
  double *P = pblk + (int64_t)blockIdx.x * b * b;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e - (e / b) * b;
    P[e] = -S[i * 65 + j];
  }
}

void launch_jacobi_setup(cudaStream_t s, const SellPattern &pat, const double *qs, const double *a0,
                         const double *a1, const uint8_t *obs, double obs_w, int n_s, int n_t,
                         int bsize, double *pblk, int32_t *err_flag) {
  ++g_launch_count;
  const int n = n_s * n_t;
  const int nblk = (n + bsize - 1) / bsize;
  k_jacobi_setup<<<nblk, bsize >= 16 ? 256 : 32, 0, s>>>(pat, qs, a0, a1, obs, obs_w, n_s, n_t,
                                                         bsize, pblk, err_flag);
}

// ---------------------------------------------------------------------------
// PCG update for a 64-row tile: x += alpha p, r -= alpha q, z = P r (block
// Jacobi), and per-column partial sums <r, z>, <r, r>.
// ---------------------------------------------------------------------------
constexpr int kPcgUpdateSmem = (64 * 65 + 64 * 64 + 2 * 4 * 64) * (int)sizeof(double);

__global__ void __launch_bounds__(256) k_pcg_update(PcgVec v, const double *__restrict__ pblk, int b) {
  extern __shared__ double smem_upd[];
  double (*rs)[65] = reinterpret_cast<double (*)[65]>(smem_upd);
  double *Ps = smem_upd + 64 * 65;
  double (*red_a)[64] = reinterpret_cast<double (*)[64]>(Ps + 64 * 64);
  double (*red_b)[64] = reinterpret_cast<double (*)[64]>(Ps + 64 * 64 + 4 * 64);
  const int r0 = blockIdx.x * 64;
  const int rows = min(64, v.n - r0);
  const int n_blocks = (v.n + b - 1) / b;
  {
    const int64_t base = (int64_t)(r0 / b) * b * b;
    const int64_t lim = (int64_t)n_blocks * b * b;
    for (int e = threadIdx.x; e < 64 * b; e += blockDim.x)
      Ps[e] = (base + e < lim) ? pblk[base + e] : 0.0;
  }
  const int lc = threadIdx.x & 63, rg = threadIdx.x >> 6;
  for (int c0 = 0; c0 < v.ld; c0 += 64) {
    const int col = c0 + lc;
    const double al = v.alpha[col];
    for (int rr = rg; rr < 64; rr += 4) {
      double rv = 0.0;
      if (rr < rows) {
        const int64_t idx = (int64_t)(r0 + rr) * v.ld + col;
        rv = v.r[idx];
        if (al != 0.0) {
          v.x[idx] = fma(al, v.p[idx], v.x[idx]);
          rv = fma(-al, v.q[idx], rv);
          v.r[idx] = rv;
        }
      }
      rs[rr][lc] = rv;
    }
    __syncthreads();
    double sa = 0.0, sb = 0.0;
    for (int rr = rg; rr < rows; rr += 4) {
      const int blk = rr / b, bo = rr - blk * b;
      const double *Pr = Ps + blk * b * b + bo * b;
      const int rb = blk * b;
      double z = 0.0;
      for (int jj = 0; jj < b; ++jj) z = fma(Pr[jj], rs[rb + jj][lc], z);
      v.z[(int64_t)(r0 + rr) * v.ld + col] = z;
      sa = fma(rs[rr][lc], z, sa);
      sb = fma(rs[rr][lc], rs[rr][lc], sb);
    }
    red_a[rg][lc] = sa;
    red_b[rg][lc] = sb;
    __syncthreads();
    if (rg == 0) {
      v.partial_a[(int64_t)blockIdx.x * v.ld + col] = red_a[0][lc] + red_a[1][lc] + red_a[2][lc] + red_a[3][lc];
      v.partial_b[(int64_t)blockIdx.x * v.ld + col] = red_b[0][lc] + red_b[1][lc] + red_b[2][lc] + red_b[3][lc];
    }
    __syncthreads();
  }
}

void launch_pcg_update(cudaStream_t s, const PcgVec &v, const double *pblk, int bsize) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_pcg_update, cudaFuncAttributeMaxDynamicSharedMemorySize, kPcgUpdateSmem);
    attr_set = true;
  }
  ++g_launch_count;
  k_pcg_update<<<v.n_tiles, 256, kPcgUpdateSmem, s>>>(v, pblk, bsize);
}

// alpha_c = rho_c / <p_c, q_c> for active columns, 0 otherwise.
__global__ void k_pcg_reduce_alpha(PcgVec v) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= v.ld) return;
  double pq = 0.0;
  for (int g = 0; g < v.n_blocks_dot; ++g) pq += v.partial_a[(int64_t)g * v.ld + c];
  v.alpha[c] = (v.active[c] && pq != 0.0) ? v.rho[c] / pq : 0.0;
}

void launch_pcg_reduce_alpha(cudaStream_t s, const PcgVec &v) {
  ++g_launch_count;
  k_pcg_reduce_alpha<<<(v.ld + 127) / 128, 128, 0, s>>>(v);
}

// <r, z>, <r, r> -> beta, rho, convergence flags, active count and the
// maximum relative residual (single block, ld <= 1024 threads).
__global__ void k_pcg_reduce_beta(PcgVec v, double tol2, int init) {
  __shared__ int cnt[32];
  __shared__ double mx[32];
  const int c = threadIdx.x;
  int act = 0;
  double rel = 0.0;
  if (c < v.ld) {
    double rz = 0.0, rr = 0.0;
    for (int g = 0; g < v.n_tiles; ++g) {
      rz += v.partial_a[(int64_t)g * v.ld + c];
      rr += v.partial_b[(int64_t)g * v.ld + c];
    }
    if (init) {
      v.bb[c] = rr;
      v.rho[c] = rz;
      v.beta[c] = 0.0;
      v.active[c] = rr > 0.0 ? 1 : 0;
    } else if (v.active[c]) {
      v.beta[c] = v.rho[c] != 0.0 ? rz / v.rho[c] : 0.0;
      v.rho[c] = rz;
      if (rr <= tol2 * v.bb[c]) v.active[c] = 0;
    } else {
      v.beta[c] = 0.0;
    }
    v.rr[c] = rr;
    act = v.active[c];
    rel = v.bb[c] > 0.0 ? sqrt(rr / v.bb[c]) : 0.0;
  }
  for (int o = 16; o > 0; o >>= 1) {
    act += __shfl_down_sync(0xffffffffu, act, o);
    rel = fmax(rel, __shfl_down_sync(0xffffffffu, rel, o));
  }
  if ((threadIdx.x & 31) == 0) {
    cnt[threadIdx.x >> 5] = act;
    mx[threadIdx.x >> 5] = rel;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0;
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += cnt[w];
      m = fmax(m, mx[w]);
    }
    v.counters[0] = a;
    v.max_rel[0] = m;
  }
}

void launch_pcg_reduce_beta(cudaStream_t s, const PcgVec &v, double tol, int init) {
  ++g_launch_count;
  int threads = (v.ld + 31) / 32 * 32;
  k_pcg_reduce_beta<<<1, threads, 0, s>>>(v, tol * tol, init);
}

// p = z + beta p  (p = z where beta is zero, so stale values never leak in).
__global__ void k_pcg_p_update(PcgVec v) {
  const int64_t total = (int64_t)v.n * v.ld;
  for (int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * 2; e < total;
       e += (int64_t)gridDim.x * blockDim.x * 2) {
    const int c = (int)(e % v.ld);
    const double2 z = *reinterpret_cast<const double2 *>(v.z + e);
    double2 p = *reinterpret_cast<const double2 *>(v.p + e);
    const double b0 = v.beta[c], b1 = v.beta[c + 1];
    p.x = (b0 != 0.0) ? fma(b0, p.x, z.x) : z.x;
    p.y = (b1 != 0.0) ? fma(b1, p.y, z.y) : z.y;
    *reinterpret_cast<double2 *>(v.p + e) = p;
  }
}

void launch_pcg_p_update(cudaStream_t s, const PcgVec &v) {
  ++g_launch_count;
  int64_t total = (int64_t)v.n * v.ld / 2;
  int grid = (int)((total + 255) / 256);
  if (grid > 152 * 16) grid = 152 * 16;
  k_pcg_p_update<<<grid, 256, 0, s>>>(v);
}

}  // namespace qsel
