// Global samples (Section 3.3): perturbation right-hand sides from
// counter-based Gaussian noise and one multi-right-hand-side preconditioned
// conjugate-gradient solve Q X = R.
//
// Layout: every n x k block of vectors is row-major with leading dimension
// ld (a multiple of 64): row t * n_s + i holds the k samples of node i of
// slab t contiguously, so one warp reads a whole row with 16-byte loads.
#include "qsel.h"
#include "kernels.cuh"
#include "sweep.cuh"
#include "bjblock.cuh"

#include <algorithm>
#include <type_traits>

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

// Two adjacent elements of T (16 bytes for double, 8 for float).
template <typename T>
struct Pair;
template <>
struct Pair<double> {
  using V = double2;
};
template <>
struct Pair<float> {
  using V = float2;
};

template <typename T>
__device__ __forceinline__ typename Pair<T>::V load2(const T *p) {
  return *reinterpret_cast<const typename Pair<T>::V *>(p);
}
template <typename T>
__device__ __forceinline__ void store2(T *p, T a, T b) {
  typename Pair<T>::V v;
  v.x = a;
  v.y = b;
  *reinterpret_cast<typename Pair<T>::V *>(p) = v;
}

// ---------------------------------------------------------------------------
// Block-tridiagonal sliced-ELL SpMM over many right-hand sides:
//   y_t = sum_{d=-1,0,1} c_{t,t+d} (V x_{t+d}) + w_obs diag(obs_t) x_t
// where V is the spatial matrix on the SELL-32 pattern (Q_s here) and the
// c's are the per-slab time coefficients.  One warp per (row, 64*NV-column
// chunk); column index and value are warp-uniform broadcasts, the three
// neighbour rows are read as coalesced 2-element vectors.  Optional epilogue:
// per-CTA, per-column partial sums of x .* y in double (the PCG curvature).
// ---------------------------------------------------------------------------
constexpr int kSpmmGridMax = 152 * 8;

int bt_spmm_grid(int n_rows) {
  int g = (n_rows + 7) / 8;
  return g < kSpmmGridMax ? (g < 1 ? 1 : g) : kSpmmGridMax;
}



// Time combination of the block-tridiagonal product of a separable model
// (every block the same spatial array V, scaled per block):
//   zc_t = c0_t x_t + c1_{t-1} x_{t-1} + c1_t x_{t+1}   (16-byte vectors)
// so that y_t = V zc_t + w_obs diag(obs_t) x_t needs one spatial pass that
// reads w neighbour rows per output row instead of 3w.
template <typename T>
__global__ void __launch_bounds__(256) k_time_combine(BtSpmmArgs<T> a) {
  using V4 = typename std::conditional<std::is_same<T, float>::value, float4, double2>::type;
  constexpr int E = (int)(sizeof(V4) / sizeof(T));
  const int64_t slab = (int64_t)a.n_s * a.ld / E;
  const int64_t total = slab * a.n_t;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(e / slab);
    const T c0 = (T)a.m.diag.scale(t);
    const T cm = (t > 0) ? (T)a.m.off.scale(t - 1) : T(0);
    const T cp = (t + 1 < a.n_t) ? (T)a.m.off.scale(t) : T(0);
    const V4 x0 = reinterpret_cast<const V4 *>(a.x)[e];
    V4 z;
    const T *xs = reinterpret_cast<const T *>(&x0);
    T *zs = reinterpret_cast<T *>(&z);
#pragma unroll
    for (int q = 0; q < E; ++q) zs[q] = c0 * xs[q];
    if (t > 0) {
      const V4 xm = reinterpret_cast<const V4 *>(a.x)[e - slab];
      const T *ms = reinterpret_cast<const T *>(&xm);
#pragma unroll
      for (int q = 0; q < E; ++q) zs[q] = fma(cm, ms[q], zs[q]);
    }
    if (t + 1 < a.n_t) {
      const V4 xp = reinterpret_cast<const V4 *>(a.x)[e + slab];
      const T *ps = reinterpret_cast<const T *>(&xp);
#pragma unroll
      for (int q = 0; q < E; ++q) zs[q] = fma(cp, ps[q], zs[q]);
    }
    reinterpret_cast<V4 *>(a.tmp)[e] = z;
  }
}

// COMB: the neighbour rows are read from the time combination a.tmp (one
// term per pattern entry) instead of three slabs of a.x.
template <typename T, int NV, bool COMB>
__global__ void __launch_bounds__(256) k_bt_spmm(BtSpmmArgs<T> a) {
  __shared__ T red[8][512];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_rows = a.n_s * a.n_t;
  const int ld = a.ld;
  const int chunk_cols = 64 * NV;
  const int nchunk = ld / chunk_cols;
  const bool dot = a.dot_partial != nullptr;
  if (dot) {
    for (int c = lane; c < ld; c += 32) red[warp][c] = T(0);
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
    // per-row scalars in T: the FP32 path issues no double arithmetic per element
    const T c0 = (T)a.m.diag.scale(t);
    const T cm = (t > 0) ? (T)a.m.off.scale(t - 1) : T(0);
    const T cp = (t + 1 < a.n_t) ? (T)a.m.off.scale(t) : T(0);
    const double *v0p = a.m.diag.at(t);
    const double *vmp = a.m.off.at(t > 0 ? t - 1 : 0);
    const double *vpp = a.m.off.at(t + 1 < a.n_t ? t : 0);
    const int coff = ch * chunk_cols + 2 * lane;
    T ax[NV], ay[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) ax[v] = ay[v] = T(0);
    const bool has_m = t > 0, has_p = t + 1 < a.n_t;
    for (int s0 = 0; s0 < w; s0 += 32) {
      // the row's pattern entries, one per lane, then broadcast: no dependent
      // loads inside the neighbour loop
      int my_col = i;
      T my_val = T(0), my_f0 = T(0), my_fm = T(0), my_fp = T(0);
      if (s0 + lane < w) {
        const int idx = base + (s0 + lane) * kSlice;
        my_col = a.pat.col[idx];
        if (COMB) {
          my_val = (T)v0p[idx];
        } else {
          my_f0 = c0 * (T)v0p[idx];
          my_fm = has_m ? cm * (T)vmp[idx] : T(0);
          my_fp = has_p ? cp * (T)vpp[idx] : T(0);
        }
      }
      const int cnt = min(32, w - s0);
#pragma unroll 4
      for (int s = 0; s < cnt; ++s) {
        const int j = __shfl_sync(0xffffffffu, my_col, s);
        if (COMB) {
          const T val = __shfl_sync(0xffffffffu, my_val, s);
          const T *zc = a.tmp + ((int64_t)t * a.n_s + j) * ld + coff;
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const auto z0 = load2(zc + 64 * v);
            ax[v] = fma(val, z0.x, ax[v]);
            ay[v] = fma(val, z0.y, ay[v]);
          }
          continue;
        }
        const T *xc = a.x + ((int64_t)t * a.n_s + j) * ld + coff;
        const T f0 = __shfl_sync(0xffffffffu, my_f0, s);
        const T fm = __shfl_sync(0xffffffffu, my_fm, s);
        const T fp = __shfl_sync(0xffffffffu, my_fp, s);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const auto x0 = load2(xc + 64 * v);
          ax[v] = fma(f0, x0.x, ax[v]);
          ay[v] = fma(f0, x0.y, ay[v]);
          if (has_m) {
            const auto xm = load2(xc - slab + 64 * v);
            ax[v] = fma(fm, xm.x, ax[v]);
            ay[v] = fma(fm, xm.y, ay[v]);
          }
          if (has_p) {
            const auto xp = load2(xc + slab + 64 * v);
            ax[v] = fma(fp, xp.x, ax[v]);
            ay[v] = fma(fp, xp.y, ay[v]);
          }
        }
      }
    }
    const T *xr = a.x + (int64_t)row * ld + coff;
    const T ow = (a.m.obs != nullptr && a.m.obs[row]) ? (T)a.m.obs_w : T(0);
    T *yr = a.y + (int64_t)row * ld + coff;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T x0 = T(0), x1 = T(0);
      if (ow != T(0) || dot) {
        const auto xv = load2(xr + 64 * v);
        x0 = xv.x;
        x1 = xv.y;
      }
      ax[v] = fma(ow, x0, ax[v]);
      ay[v] = fma(ow, x1, ay[v]);
      store2(yr + 64 * v, ax[v], ay[v]);
      if (dot) {
        red[warp][coff + 64 * v] = fma(x0, ax[v], red[warp][coff + 64 * v]);
        red[warp][coff + 64 * v + 1] = fma(x1, ay[v], red[warp][coff + 64 * v + 1]);
      }
    }
  }
  if (dot) {
    __syncthreads();
    for (int c = threadIdx.x; c < ld; c += blockDim.x) {
      double sum = 0.0;
#pragma unroll
      for (int ww = 0; ww < 8; ++ww) sum += (double)red[ww][c];
      a.dot_partial[(int64_t)blockIdx.x * ld + c] = sum;
    }
  }
}

template <typename T>
void launch_bt_spmm(cudaStream_t s, const BtSpmmArgs<T> &a) {
  ++g_launch_count;
  const int grid = bt_spmm_grid(a.n_s * a.n_t);
  Profiler::Rec rec{PROF_SPMM, nullptr, nullptr, 0.0};
  if (g_prof) {
    // algorithmic bytes: read x once, write y once (the spatial pattern and the
    // neighbouring rows are re-read from cache)
    rec.work = 2.0 * (double)a.n_s * a.n_t * a.ld * sizeof(T);
    g_prof->begin(s, rec);
  }
  // the time combination needs every block to be the same spatial array
  const bool separable = a.m.diag.stride == 0 && a.m.off.stride == 0 && a.m.diag.v == a.m.off.v &&
                         a.m.diag.coef != nullptr && a.m.off.coef != nullptr;
  if (a.tmp && separable) {
    ++g_launch_count;
    const int64_t vec = (int64_t)a.n_s * a.n_t * a.ld / (16 / (int)sizeof(T));
    k_time_combine<T><<<(int)std::min<int64_t>((vec + 255) / 256, 152 * 8), 256, 0, s>>>(a);
    if (a.ld % 256 == 0)
      k_bt_spmm<T, 4, true><<<grid, 256, 0, s>>>(a);
    else if (a.ld % 128 == 0)
      k_bt_spmm<T, 2, true><<<grid, 256, 0, s>>>(a);
    else
      k_bt_spmm<T, 1, true><<<grid, 256, 0, s>>>(a);
  } else if (a.ld % 256 == 0) {
    k_bt_spmm<T, 4, false><<<grid, 256, 0, s>>>(a);
  } else if (a.ld % 128 == 0) {
    k_bt_spmm<T, 2, false><<<grid, 256, 0, s>>>(a);
  } else {
    k_bt_spmm<T, 1, false><<<grid, 256, 0, s>>>(a);
  }
  if (g_prof) g_prof->end(s, rec);
}
template void launch_bt_spmm<double>(cudaStream_t, const BtSpmmArgs<double> &);
template void launch_bt_spmm<float>(cudaStream_t, const BtSpmmArgs<float> &);

// ---------------------------------------------------------------------------
// Block-Jacobi preconditioner (Section 3.3 names block-Jacobi / IC(0)):
// contiguous blocks of b global rows; P_blk = (Q_blk)^-1 by the symmetric
// sweep in shared memory (double).  Rows past n are padded with the identity.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_jacobi_setup(SellPattern pat, BtModel m, int n_s, int n_t, int b,
                                                      T *__restrict__ pblk, int32_t *err_flag) {
  __shared__ double S[64 * 65];
  assemble_diag_block(S, 65, pat, m, n_s, n_t, blockIdx.x * b, b);
  sym_sweep_inverse_smem(S, 65, b, err_flag);
  T *P = pblk + (int64_t)blockIdx.x * b * b;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e - (e / b) * b;
    P[e] = (T)(-S[i * 65 + j]);
  }
}

template <typename T>
void launch_jacobi_setup(cudaStream_t s, const SellPattern &pat, const BtModel &m, int n_s, int n_t, int bsize,
                         T *pblk, int32_t *err_flag) {
  ++g_launch_count;
  const int n = n_s * n_t;
  const int nblk = (n + bsize - 1) / bsize;
  k_jacobi_setup<T><<<nblk, bsize >= 16 ? 256 : 32, 0, s>>>(pat, m, n_s, n_t, bsize, pblk, err_flag);
}
template void launch_jacobi_setup<double>(cudaStream_t, const SellPattern &, const BtModel &, int, int, int, double *,
                                          int32_t *);
template void launch_jacobi_setup<float>(cudaStream_t, const SellPattern &, const BtModel &, int, int, int, float *,
                                         int32_t *);

// ---------------------------------------------------------------------------
// PCG update for a 64-row tile: x += alpha p, r -= alpha q, z = P r (block
// Jacobi), and per-column partial sums <r, z>, <r, r> in double.
// ---------------------------------------------------------------------------
constexpr int kUpdGrid = 152 * 4;

int pcg_update_grid(int n) {
  const int tiles = (n + 63) / 64;
  return tiles < kUpdGrid ? tiles : kUpdGrid;
}

// x += alpha p, r -= alpha q: streaming, 16-byte vectors, grid-stride.
template <typename T>
__global__ void __launch_bounds__(256) k_pcg_axpy(PcgVec<T> v) {
  using V4 = typename std::conditional<std::is_same<T, float>::value, float4, double2>::type;
  constexpr int E = (int)(sizeof(V4) / sizeof(T));
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // the reduction that follows accumulates into these
    v.counters[0] = 0;
    v.max_rel[0] = 0.0;
  }
  const int64_t total = (int64_t)v.n * v.ld / E;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)((e * E) % v.ld);
    T al[E];
    bool any = false;
#pragma unroll
    for (int q = 0; q < E; ++q) {
      al[q] = (T)v.alpha[c + q];
      any |= al[q] != T(0);
    }
    if (!any) continue;
    V4 x = reinterpret_cast<const V4 *>(v.x)[e];
    V4 r = reinterpret_cast<const V4 *>(v.r)[e];
    const V4 p = reinterpret_cast<const V4 *>(v.p)[e];
    const V4 qq = reinterpret_cast<const V4 *>(v.q)[e];
    T *xs = reinterpret_cast<T *>(&x);
    T *rs = reinterpret_cast<T *>(&r);
    const T *ps = reinterpret_cast<const T *>(&p);
    const T *qs = reinterpret_cast<const T *>(&qq);
#pragma unroll
    for (int q = 0; q < E; ++q) {
      xs[q] = fma(al[q], ps[q], xs[q]);
      rs[q] = fma(-al[q], qs[q], rs[q]);
    }
    reinterpret_cast<V4 *>(v.x)[e] = x;
    reinterpret_cast<V4 *>(v.r)[e] = r;
  }
}

// z = P r for 64-row tiles (block Jacobi) and per-column partial sums
// <r, z>, <r, r>.  Per tile the P blocks are staged once in shared memory,
// transposed (Pt[j][row]); then for every chunk of CW columns the r tile is
// staged and each thread accumulates an 8-row x (CW/32)-column register tile:
// per j two 16-byte loads of P (warp broadcast) and one of r feed
// 8 x (CW/32) FMAs.  Rows of one 8-row group lie in one block (b >= 8).
template <typename T, int CW>
struct PrecondSmem {
  static constexpr int PS = 64 + 16 / (int)sizeof(T);        // Pt row stride (elements)
  static constexpr int RS = CW + 16 / (int)sizeof(T);        // r tile row stride
  static constexpr int bytes = (64 * PS + 64 * RS) * (int)sizeof(T) + 2 * 8 * CW * 8 + 2 * 512 * 8;
};

template <typename T, int CW>
__global__ void __launch_bounds__(256) k_pcg_precond(PcgVec<T> v, const T *__restrict__ pblk, int b) {
  using SM = PrecondSmem<T, CW>;
  constexpr int NC = CW / 32;                                  // columns per thread
  using VC = typename std::conditional<NC * sizeof(T) == 16, typename std::conditional<std::is_same<T, float>::value, float4, double2>::type,
                                       typename std::conditional<std::is_same<T, float>::value, float2, double>::type>::type;
  using V16 = typename std::conditional<std::is_same<T, float>::value, float4, double2>::type;
  constexpr int E16 = 16 / (int)sizeof(T);
  extern __shared__ __align__(16) unsigned char smem_pc_raw[];
  T *Pt = reinterpret_cast<T *>(smem_pc_raw);                  // [64][PS]
  T *rsm = Pt + 64 * SM::PS;                                   // [64][RS]
  double *red = reinterpret_cast<double *>(rsm + 64 * SM::RS); // [2][8][CW]
  double *acc = red + 2 * 8 * CW;                              // [2][512]
  const int tid = threadIdx.x, rg = tid >> 5, cg = tid & 31;
  const int n_blocks = (v.n + b - 1) / b;
  const int n_tiles = (v.n + 63) / 64;
  for (int c = tid; c < v.ld; c += blockDim.x) {
    acc[c] = 0.0;
    acc[512 + c] = 0.0;
  }
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int r0 = tile * 64;
    const int rows = min(64, v.n - r0);
    __syncthreads();
    {
      const int64_t base = (int64_t)(r0 / b) * b * b;
      const int64_t lim = (int64_t)n_blocks * b * b;
      for (int e = tid; e < 64 * b; e += blockDim.x) {
        const int blk = e / (b * b), rem = e - blk * b * b;
        const int r = rem / b, j = rem - r * b;
        Pt[(blk * b + j) * SM::PS + blk * b + r] = (base + e < lim) ? pblk[base + e] : T(0);
      }
    }
    for (int c0 = 0; c0 < v.ld; c0 += CW) {
      __syncthreads();
      // stage r[r0 .. r0+63][c0 .. c0+CW) with 16-byte loads
      for (int e = tid; e < 64 * CW / E16; e += blockDim.x) {
        const int rr = e / (CW / E16), q = e - rr * (CW / E16);
        V16 val;
        if (rr < rows) {
          val = *reinterpret_cast<const V16 *>(v.r + (int64_t)(r0 + rr) * v.ld + c0 + q * E16);
        } else {
          T *z = reinterpret_cast<T *>(&val);
#pragma unroll
          for (int u = 0; u < E16; ++u) z[u] = T(0);
        }
        *reinterpret_cast<V16 *>(rsm + rr * SM::RS + q * E16) = val;
      }
      __syncthreads();
      const int row0 = rg * 8;
      T z[8][NC];
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int q = 0; q < NC; ++q) z[a][q] = T(0);
      if (b >= 8) {
        const int jb = (row0 / b) * b;
        for (int jj = 0; jj < b; ++jj) {
          const int jl = jb + jj;
          T pv[8];
          const V16 *pp = reinterpret_cast<const V16 *>(Pt + jl * SM::PS + row0);
#pragma unroll
          for (int u = 0; u < 8 / E16; ++u) {
            const V16 t4 = pp[u];
            const T *ts = reinterpret_cast<const T *>(&t4);
#pragma unroll
            for (int w = 0; w < E16; ++w) pv[u * E16 + w] = ts[w];
          }
          const VC rv = *reinterpret_cast<const VC *>(rsm + jl * SM::RS + cg * NC);
          const T *rs = reinterpret_cast<const T *>(&rv);
#pragma unroll
          for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int q = 0; q < NC; ++q) z[a][q] = fma(pv[a], rs[q], z[a][q]);
        }
      } else {
        // b == 1: Jacobi, P holds the inverse diagonal
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const int rl = row0 + a;
          const T d = Pt[rl * SM::PS + rl];
#pragma unroll
          for (int q = 0; q < NC; ++q) z[a][q] = d * rsm[rl * SM::RS + cg * NC + q];
        }
      }
      T sa[NC], sb[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) sa[q] = sb[q] = T(0);
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int rl = row0 + a;
        if (rl < rows) {
          VC out;
          T *os = reinterpret_cast<T *>(&out);
#pragma unroll
          for (int q = 0; q < NC; ++q) {
            os[q] = z[a][q];
            const T rd = rsm[rl * SM::RS + cg * NC + q];
            sa[q] = fma(rd, z[a][q], sa[q]);
            sb[q] = fma(rd, rd, sb[q]);
          }
          *reinterpret_cast<VC *>(v.z + (int64_t)(r0 + rl) * v.ld + c0 + cg * NC) = out;
        }
      }
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        red[rg * CW + cg * NC + q] = (double)sa[q];
        red[8 * CW + rg * CW + cg * NC + q] = (double)sb[q];
      }
      __syncthreads();
      for (int c = tid; c < 2 * CW; c += blockDim.x) {
        const int which = c / CW, cc = c - which * CW;
        double s2 = 0.0;
#pragma unroll
        for (int g = 0; g < 8; ++g) s2 += red[which * 8 * CW + g * CW + cc];
        acc[which * 512 + c0 + cc] += s2;
      }
    }
  }
  __syncthreads();
  for (int c = tid; c < v.ld; c += blockDim.x) {
    v.partial_a[(int64_t)blockIdx.x * v.ld + c] = acc[c];
    v.partial_b[(int64_t)blockIdx.x * v.ld + c] = acc[512 + c];
  }
}

template <typename T>
void launch_pcg_update(cudaStream_t s, const PcgVec<T> &v, const T *pblk, int bsize, const KronOperator *kron) {
  // 128-column chunks for FP32 when they divide ld, else 64
  constexpr int CWF = std::is_same<T, float>::value ? 128 : 64;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_pcg_precond<T, CWF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         PrecondSmem<T, CWF>::bytes);
    cudaFuncSetAttribute(k_pcg_precond<T, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         PrecondSmem<T, 64>::bytes);
    attr_set = true;
  }
  g_launch_count += 2;
  const int64_t vec = (int64_t)v.n * v.ld / (16 / (int)sizeof(T));
  const int grid = (int)std::min<int64_t>((vec + 255) / 256, 152 * 8);
  {
    ProfScope ps_(s, PROF_PCGVEC);
    k_pcg_axpy<T><<<grid, 256, 0, s>>>(v);
  }
  if (kron) {
    --g_launch_count;   // counted by the launchers below
    launch_kron_apply<T>(s, *kron, v.r, v.q, v.z);
    launch_pcg_dots<T>(s, v);
    return;
  }
  // algorithmic work: 2 b FLOPs per element of z (b = 1: one multiply)
  ProfScope ps_(s, PROF_PRECOND, (bsize > 1 ? 2.0 * bsize : 1.0) * (double)v.n * v.ld);
  if (v.ld % CWF == 0)
    k_pcg_precond<T, CWF><<<v.n_tiles, 256, PrecondSmem<T, CWF>::bytes, s>>>(v, pblk, bsize);  // n_tiles = grid
  else
    k_pcg_precond<T, 64><<<v.n_tiles, 256, PrecondSmem<T, 64>::bytes, s>>>(v, pblk, bsize);
}
template void launch_pcg_update<double>(cudaStream_t, const PcgVec<double> &, const double *, int,
                                        const KronOperator *);
template void launch_pcg_update<float>(cudaStream_t, const PcgVec<float> &, const float *, int,
                                       const KronOperator *);

// Column sums of per-CTA partial rows: 8 row groups x 32 columns per block,
// fixed order within each group and across groups.
__device__ __forceinline__ double column_sum(const double *__restrict__ part, int n_rows, int ld, int c, int rg,
                                             double (*sh)[33]) {
  double acc = 0.0;
  for (int g = rg; g < n_rows; g += 8) acc += part[(int64_t)g * ld + c];
  sh[rg][threadIdx.x & 31] = acc;
  __syncthreads();
  double tot = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) tot += sh[q][threadIdx.x & 31];
  return tot;
}

// alpha_c = rho_c / <p_c, q_c> for active columns, 0 otherwise.
template <typename T>
__global__ void __launch_bounds__(256) k_pcg_reduce_alpha(PcgVec<T> v) {
  __shared__ double sh[8][33];
  const int c = blockIdx.x * 32 + (threadIdx.x & 31), rg = threadIdx.x >> 5;
  const double pq = column_sum(v.partial_a, v.n_blocks_dot, v.ld, c, rg, sh);
  if (rg == 0) v.alpha[c] = (v.active[c] && pq != 0.0) ? v.rho[c] / pq : 0.0;
}

template <typename T>
void launch_pcg_reduce_alpha(cudaStream_t s, const PcgVec<T> &v) {
  ++g_launch_count;
  {
    ProfScope ps_(s, PROF_PCGVEC);
    k_pcg_reduce_alpha<T><<<v.ld / 32, 256, 0, s>>>(v);
  }
}
template void launch_pcg_reduce_alpha<double>(cudaStream_t, const PcgVec<double> &);
template void launch_pcg_reduce_alpha<float>(cudaStream_t, const PcgVec<float> &);

// <r, z>, <r, r> -> beta, rho, convergence flags; active count and maximum
// relative residual by integer atomics (the update kernel zeroed them).
template <typename T>
__global__ void __launch_bounds__(256) k_pcg_reduce_beta(PcgVec<T> v, double tol2, int init) {
  __shared__ double sh[8][33];
  const int c = blockIdx.x * 32 + (threadIdx.x & 31), rg = threadIdx.x >> 5;
  const double rz = column_sum(v.partial_a, v.n_tiles, v.ld, c, rg, sh);
  __syncthreads();
  const double rr = column_sum(v.partial_b, v.n_tiles, v.ld, c, rg, sh);
  if (rg != 0) return;
  if (init) {
    v.bb[c] = rr;
    v.rho[c] = rz;
    v.beta[c] = 0.0;
    v.active[c] = rr > 0.0 ? 1 : 0;
  } else if (v.active[c]) {
    v.beta[c] = v.rho[c] != 0.0 ? rz / v.rho[c] : 0.0;
    v.rho[c] = rz;
    if (rr <= (v.tol2_dev ? *v.tol2_dev : tol2) * v.bb[c]) v.active[c] = 0;
  } else {
    v.beta[c] = 0.0;
  }
  v.rr[c] = rr;
  int act = v.active[c];
  double rel = v.bb[c] > 0.0 ? sqrt(rr / v.bb[c]) : 0.0;
  for (int o = 16; o > 0; o >>= 1) {
    act += __shfl_down_sync(0xffffffffu, act, o);
    rel = fmax(rel, __shfl_down_sync(0xffffffffu, rel, o));
  }
  if (threadIdx.x == 0) {
    if (act) atomicAdd(v.counters, act);
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long *>(v.max_rel), (unsigned long long)__double_as_longlong(rel));
  }
}

template <typename T>
void launch_pcg_reduce_beta(cudaStream_t s, const PcgVec<T> &v, double tol, int init) {
  ++g_launch_count;
  {
    ProfScope ps_(s, PROF_PCGVEC);
    k_pcg_reduce_beta<T><<<v.ld / 32, 256, 0, s>>>(v, tol * tol, init);
  }
}
template void launch_pcg_reduce_beta<double>(cudaStream_t, const PcgVec<double> &, double, int);
template void launch_pcg_reduce_beta<float>(cudaStream_t, const PcgVec<float> &, double, int);

// p = z + beta p  (p = z where beta is zero, so stale values never leak in).
template <typename T>
__global__ void k_pcg_p_update(PcgVec<T> v) {
  using V4 = typename std::conditional<std::is_same<T, float>::value, float4, double2>::type;
  constexpr int E = (int)(sizeof(V4) / sizeof(T));
  const int64_t total = (int64_t)v.n * v.ld / E;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)((e * E) % v.ld);
    const V4 z = reinterpret_cast<const V4 *>(v.z)[e];
    V4 p = reinterpret_cast<const V4 *>(v.p)[e];
    const T *zs = reinterpret_cast<const T *>(&z);
    T *ps = reinterpret_cast<T *>(&p);
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const T bq = (T)v.beta[c + q];
      ps[q] = (bq != T(0)) ? fma(bq, ps[q], zs[q]) : zs[q];
    }
    reinterpret_cast<V4 *>(v.p)[e] = p;
  }
}

template <typename T>
void launch_pcg_p_update(cudaStream_t s, const PcgVec<T> &v) {
  ++g_launch_count;
  int64_t total = (int64_t)v.n * v.ld / (16 / (int)sizeof(T));
  int grid = (int)((total + 255) / 256);
  if (grid > 152 * 8) grid = 152 * 8;
  {
    ProfScope ps_(s, PROF_PCGVEC);
    k_pcg_p_update<T><<<grid, 256, 0, s>>>(v);
  }
}
template void launch_pcg_p_update<double>(cudaStream_t, const PcgVec<double> &);
template void launch_pcg_p_update<float>(cudaStream_t, const PcgVec<float> &);

// ---------------------------------------------------------------------------
// Iterative refinement of the FP32 solves (mixed precision): the true
// residual r = b - Q x is formed in double, its FP32 copy is the right-hand
// side of the next inner solve, and the FP32 correction is added in double.
// ---------------------------------------------------------------------------
constexpr int kResGrid = 152 * 4;

int residual_grid(int n) {
  int g = (n + 63) / 64;
  return g < kResGrid ? g : kResGrid;
}

__global__ void __launch_bounds__(256) k_residual(const double *__restrict__ b, const double *__restrict__ y,
                                                  double *__restrict__ r, float *__restrict__ r32, int n,
                                                  int ld, double *__restrict__ prr, double *__restrict__ pbb) {
  __shared__ double sr[4][64], sbb[4][64];
  const int lc = threadIdx.x & 63, rg = threadIdx.x >> 6;
  for (int c0 = 0; c0 < ld; c0 += 64) {
    const int col = c0 + lc;
    double a = 0.0, bsum = 0.0;
    for (int row = blockIdx.x * 4 + rg; row < n; row += gridDim.x * 4) {
      const int64_t idx = (int64_t)row * ld + col;
      const double bv = b[idx];
      const double rv = bv - y[idx];
      r[idx] = rv;
      r32[idx] = (float)rv;
      a = fma(rv, rv, a);
      bsum = fma(bv, bv, bsum);
    }
    sr[rg][lc] = a;
    sbb[rg][lc] = bsum;
    __syncthreads();
    if (rg == 0) {
      prr[(int64_t)blockIdx.x * ld + col] = sr[0][lc] + sr[1][lc] + sr[2][lc] + sr[3][lc];
      pbb[(int64_t)blockIdx.x * ld + col] = sbb[0][lc] + sbb[1][lc] + sbb[2][lc] + sbb[3][lc];
    }
    __syncthreads();
  }
}

void launch_residual(cudaStream_t s, const double *b, const double *y, double *r, float *r32, int n,
                     int ld, double *partial_rr, double *partial_bb) {
  ++g_launch_count;
  {
    ProfScope ps_(s, PROF_PCGVEC);
    k_residual<<<residual_grid(n), 256, 0, s>>>(b, y, r, r32, n, ld, partial_rr, partial_bb);
  }
}

__global__ void k_residual_check(const double *__restrict__ prr, const double *__restrict__ pbb,
                                 int n_parts, int ld, double tol2, int32_t *counters, double *max_rel) {
  __shared__ int cnt[32];
  __shared__ double mx[32];
  const int c = threadIdx.x;
  int bad = 0;
  double rel = 0.0;
  if (c < ld) {
    double rr = 0.0, bb = 0.0;
    for (int g = 0; g < n_parts; ++g) {
      rr += prr[(int64_t)g * ld + c];
      bb += pbb[(int64_t)g * ld + c];
    }
    bad = (rr > tol2 * bb) ? 1 : 0;
    rel = bb > 0.0 ? sqrt(rr / bb) : 0.0;
  }
  for (int o = 16; o > 0; o >>= 1) {
    bad += __shfl_down_sync(0xffffffffu, bad, o);
    rel = fmax(rel, __shfl_down_sync(0xffffffffu, rel, o));
  }
  if ((threadIdx.x & 31) == 0) {
    cnt[threadIdx.x >> 5] = bad;
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
    counters[0] = a;
    max_rel[0] = m;
  }
}

void launch_residual_check(cudaStream_t s, const double *partial_rr, const double *partial_bb, int n_parts,
                           int ld, double tol, int32_t *counters, double *max_rel) {
  ++g_launch_count;
  k_residual_check<<<1, (ld + 31) / 32 * 32, 0, s>>>(partial_rr, partial_bb, n_parts, ld, tol * tol, counters,
                                                     max_rel);
}

// ---------------------------------------------------------------------------
// Loop control for captured graphs (conditional while nodes).  Every loop
// body ends with a control kernel that counts iterations, so a loop ends
// after at most max_iter iterations whatever the data.
// ---------------------------------------------------------------------------
__global__ void k_loop_init(cudaGraphConditionalHandle h, const int32_t *counters, int32_t *loop, int max_iter) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  loop[0] = 0;
  const int limit = max_iter - loop[2];
  cudaGraphSetConditional(h, (counters[0] > 0 && limit > 0) ? 1u : 0u);
}

__global__ void k_loop_ctl(cudaGraphConditionalHandle h, const int32_t *counters, int32_t *loop, int step,
                           int max_iter) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int it = loop[0] + step;
  loop[0] = it;
  const int limit = max_iter - loop[2];
  cudaGraphSetConditional(h, (counters[0] > 0 && it < limit) ? 1u : 0u);
}

__global__ void k_loop_status(const int32_t *counters, int32_t *loop) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  loop[2] = loop[0];
  if (counters[0] > 0) loop[3] = QSEL_ENOCONV;
}

// Refinement loop of the mixed sampler: after a residual check, decide
// whether another inner solve runs and with which inner tolerance
// max(floor, 0.5 tol / rel).
__global__ void k_refine_ctl(cudaGraphConditionalHandle h, const int32_t *counters, const double *max_rel,
                             int32_t *loop, int first, int max_outer, int max_iter, double tol, double inner_floor,
                             double *tol2_dev) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (first) {
    loop[0] = 0;
    loop[1] = 0;
    loop[2] = 0;
    loop[3] = 0;
  } else {
    loop[1] += 1;
    loop[2] += loop[0];
  }
  bool go = counters[0] > 0;
  if (go && (loop[1] >= max_outer || loop[2] >= max_iter)) {
    loop[3] = QSEL_ENOCONV;
    go = false;
  }
  if (go) {
    const double it = fmax(inner_floor, 0.5 * tol / fmax(*max_rel, 1e-300));
    *tol2_dev = it * it;
  }
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

void launch_loop_init(cudaStream_t s, cudaGraphConditionalHandle h, const int32_t *counters, int32_t *loop,
                      int max_iter) {
  ++g_launch_count;
  k_loop_init<<<1, 32, 0, s>>>(h, counters, loop, max_iter);
}
void launch_loop_ctl(cudaStream_t s, cudaGraphConditionalHandle h, const int32_t *counters, int32_t *loop, int step,
                     int max_iter) {
  ++g_launch_count;
  k_loop_ctl<<<1, 32, 0, s>>>(h, counters, loop, step, max_iter);
}
void launch_loop_status(cudaStream_t s, const int32_t *counters, int32_t *loop) {
  ++g_launch_count;
  k_loop_status<<<1, 32, 0, s>>>(counters, loop);
}
void launch_refine_ctl(cudaStream_t s, cudaGraphConditionalHandle h, const int32_t *counters,
                       const double *max_rel, int32_t *loop, int first, int max_outer, int max_iter, double tol,
                       double inner_floor, double *tol2_dev) {
  ++g_launch_count;
  k_refine_ctl<<<1, 32, 0, s>>>(h, counters, max_rel, loop, first, max_outer, max_iter, tol, inner_floor, tol2_dev);
}

__global__ void k_accumulate(double *__restrict__ x, const float *__restrict__ d, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += (double)d[i];
}

void launch_accumulate(cudaStream_t s, double *x, const float *d, int64_t count) {
  ++g_launch_count;
  int64_t grid = (count + 255) / 256;
  if (grid > 152 * 16) grid = 152 * 16;
  {
    ProfScope ps_(s, PROF_PCGVEC);
    k_accumulate<<<(int)grid, 256, 0, s>>>(x, d, count);
  }
}

}  // namespace qsel
