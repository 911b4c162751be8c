// Dense FP64 kernels of the exact subdomain selected inversion.
//
// Per overlapping subdomain Omega_p^* (T slabs), Q_{**} is block tridiagonal
// with diagonal blocks A_tt = a0_t Q_s + diag(obs_t)/sigma^2 and couplings
// A_{t+1,t} = c_t Q_s (c_t = tau Q_t[t,t+1]).  The block factorisation keeps
// the pivot blocks D_t (block LDL^T; D_t = L_tt L_tt^T of the block Cholesky):
//   D_0 = A_00,  D_{t+1} = A_{t+1,t+1} - c_t^2 Q_s D_t^-1 Q_s,
// and the Takahashi recursion runs backwards with W_t = c_t Q_s D_t^-1
// (= L_{t+1,t} L_tt^-1):
//   Sigma_{T-1} = D_{T-1}^-1,
//   Y_t = Sigma_{t+1} W_t,  Sigma_{t+1,t} = -Y_t,
//   Sigma_t = D_t^-1 + W_t^T Y_t = D_t^-1 + D_t^-1 (c_t Q_s Y_t).
// Because the couplings are sparse (the Q_s pattern), only the D_t^-1, the
// Sigma_{t+1} W_t and the D_t^-1 V products are dense n_s^3 work; they run
// here as 64 x 64 FP64 tiles.  Every dense matrix is n_pad x n_pad row-major
// (n_pad = n_s rounded up to 64, identity on the padded diagonal).
#include <atomic>
#include <mutex>
#include "qsel.h"
#include "kernels.cuh"
#include "sweep.cuh"

#include <type_traits>

namespace qsel {

// ---------------------------------------------------------------------------
// 64 x 64 FP64 tile product: acc += op(A) op(B) over K (multiple of 16).
// 256 threads, thread (ty, tx) owns rows ty + 16 i and columns tx + 16 j.
// op(A)(r, kk) = TA ? A[kk * lda + r] : A[r * lda + kk]
// op(B)(kk, c) = TB ? B[c * ldb + kk] : B[kk * ldb + c]
// ---------------------------------------------------------------------------
template <typename T>
struct TileSmem {
  T As[2][16][64];
  T Bs[2][16][64];
};

template <bool TA, bool TB, typename T>
__device__ __forceinline__ void tile_load(const T *__restrict__ A, int lda, const T *__restrict__ B, int ldb,
                                          int k0, T ra[4], T rb[4]) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int idx = tid + 256 * u;
    if (TA) {
      const int kk = idx >> 6, r = idx & 63;
      ra[u] = A[(int64_t)(k0 + kk) * lda + r];
    } else {
      const int r = idx >> 4, kk = idx & 15;
      ra[u] = A[(int64_t)r * lda + k0 + kk];
    }
    if (TB) {
      const int c = idx >> 4, kk = idx & 15;
      rb[u] = B[(int64_t)c * ldb + k0 + kk];
    } else {
      const int kk = idx >> 6, c = idx & 63;
      rb[u] = B[(int64_t)(k0 + kk) * ldb + c];
    }
  }
}

template <bool TA, bool TB, typename T>
__device__ __forceinline__ void tile_store(TileSmem<T> &sm, int buf, const T ra[4], const T rb[4]) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int idx = tid + 256 * u;
    if (TA)
      sm.As[buf][idx >> 6][idx & 63] = ra[u];
    else
      sm.As[buf][idx & 15][idx >> 4] = ra[u];
    if (TB)
      sm.Bs[buf][idx & 15][idx >> 4] = rb[u];
    else
      sm.Bs[buf][idx >> 6][idx & 63] = rb[u];
  }
}

template <bool TA, bool TB, typename T>
__device__ __forceinline__ void tile_mma(TileSmem<T> &sm, const T *__restrict__ A, int lda,
                                         const T *__restrict__ B, int ldb, int K, T acc[4][4]) {
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  T ra[4], rb[4];
  tile_load<TA, TB>(A, lda, B, ldb, 0, ra, rb);
  tile_store<TA, TB>(sm, 0, ra, rb);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += 16) {
    const bool more = k0 + 16 < K;
    if (more) tile_load<TA, TB>(A, lda, B, ldb, k0 + 16, ra, rb);
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sm.As[buf][kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sm.Bs[buf][kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (more) {
      tile_store<TA, TB>(sm, buf ^ 1, ra, rb);
      __syncthreads();
      buf ^= 1;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Batched GEMM: C = alpha A B + beta C0 (C0 may alias C).
// ---------------------------------------------------------------------------
template <typename T, bool LOWER>
__global__ void __launch_bounds__(256) k_gemm64(GemmBatch<T> bt, int K, int lda, int ldb, int ldc) {
  __shared__ TileSmem<T> sm;
  const GemmEntry<T> e = bt.e[blockIdx.z];
  const int bm = blockIdx.y, bn = blockIdx.x;
  if (LOWER && bn > bm) return;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  tile_mma<false, false>(sm, e.A + (int64_t)bm * 64 * lda, lda, e.B + (int64_t)bn * 64, ldb, K, acc);
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t row = (int64_t)bm * 64 + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t idx = row * ldc + bn * 64 + tx + 16 * j;
      T v = (T)e.alpha * acc[i][j];
      if (e.beta != 0.0) v = fma((T)e.beta, e.C0[idx], v);
      e.C[idx] = v;
    }
  }
}

template <typename T>
void launch_gemm(cudaStream_t s, const GemmBatch<T> &b, int M, int N, int K, int lda, int ldb, int ldc,
                 bool lower) {
  if (b.count <= 0) return;
  ++g_launch_count;
  dim3 grid(N / 64, M / 64, b.count);
  Profiler::Rec rec{PROF_GEMM, nullptr, nullptr, 0.0};
  if (g_prof) {
    const double mt = M / 64, nt = N / 64;
    const double tiles = lower ? (nt * (nt + 1) / 2) : mt * nt;
    rec.work = 2.0 * 64.0 * 64.0 * K * tiles * b.count;
    g_prof->begin(s, rec);
  }
  if (lower)
    k_gemm64<T, true><<<grid, 256, 0, s>>>(b, K, lda, ldb, ldc);
  else
    k_gemm64<T, false><<<grid, 256, 0, s>>>(b, K, lda, ldb, ldc);
  if (g_prof) g_prof->end(s, rec);
}
// ---------------------------------------------------------------------------
// out[r, c] = alpha in[c, r] + beta c0[r, c]   (out, c0: rows x cols with row
// stride ld_out; in: cols x rows with row stride ld_in), 32 x 32 tiles staged
// in shared memory so that both sides are read and written along rows.
// c0 may alias out (each entry is read and written by the same thread).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_transpose_axpby(TransBatch bt, int rows, int cols, int ld_in, int ld_out) {
  __shared__ float tile[32][33];
  const TransEntry e = bt.e[blockIdx.z];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    tile[i][threadIdx.x] = (c < cols && r < rows) ? e.in[(int64_t)c * ld_in + r] : 0.0f;
  }
  __syncthreads();
  const bool add_c0 = e.c0 != nullptr && e.beta != 0.0f;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) {
      float v = e.alpha * tile[threadIdx.x][i];
      if (add_c0) v = fmaf(e.beta, e.c0[(int64_t)r * ld_out + c], v);
      e.out[(int64_t)r * ld_out + c] = v;
    }
  }
}

void launch_transpose_axpby(cudaStream_t s, const TransBatch &b, int rows, int cols, int ld_in, int ld_out) {
  if (b.count <= 0) return;
  ++g_launch_count;
  ProfScope ps_(s, PROF_CORR);
  k_transpose_axpby<<<dim3((cols + 31) / 32, (rows + 31) / 32, b.count), dim3(32, 8), 0, s>>>(b, rows, cols, ld_in,
                                                                                              ld_out);
}

bool launch_symm_block_tc(cudaStream_t s, const GemmBatch<float> &b, float *const *bt, float *const *pt, int n_pad,
                          int ld, int passes, int32_t *err) {
  if (b.count <= 0) return true;
  TransBatch tin{}, tout{};
  GemmBatch<float> g{};
  tin.count = tout.count = g.count = b.count;
  for (int q = 0; q < b.count; ++q) {
    tin.e[q] = TransEntry{b.e[q].B, nullptr, bt[q], 1.0f, 0.0f};
    g.e[q].A = bt[q];
    g.e[q].B = b.e[q].A;
    g.e[q].C0 = nullptr;
    g.e[q].C = pt[q];
    g.e[q].alpha = 1.0;
    g.e[q].beta = 0.0;
    tout.e[q] = TransEntry{pt[q], b.e[q].C0, b.e[q].C, (float)b.e[q].alpha, (float)b.e[q].beta};
  }
  launch_transpose_axpby(s, tin, ld, n_pad, ld, n_pad);
  if (!launch_tc_gemm(s, g, ld, n_pad, n_pad, n_pad, n_pad, n_pad, false, passes, err)) return false;
  launch_transpose_axpby(s, tout, n_pad, ld, n_pad, ld);
  return true;
}

template void launch_gemm<double>(cudaStream_t, const GemmBatch<double> &, int, int, int, int, int, int, bool);
template void launch_gemm<float>(cudaStream_t, const GemmBatch<float> &, int, int, int, int, int, int, bool);

// ---------------------------------------------------------------------------
// Blocked symmetric sweep: in-place SPD inverse on the lower 64 x 64 tiles.
// Step k with pivot tile P = A_kk^-1:
//   panel  U_i = A_ik P,  V_i = A_ik            (i != k; A_ik = A_ki^T for i < k)
//   update A_ij -= U_i V_j^T                     (lower tiles, i, j != k)
//          A_ik <- U_i,  A_kk <- -P
// After every step the swept matrix holds -A^-1 (Goodnight's sweep operator);
// the final mirror negates it and fills the upper triangle.
// ---------------------------------------------------------------------------
// P = Tk^-1 for the 64 x 64 tile at Tk (row stride ld), from its lower half:
// in binary64 for double tiles; for float tiles in double-float (about 48
// bits, on the FP32 pipe) or, with fp64, in binary64.  NT threads.
template <int NT, typename T>
__device__ __forceinline__ void invert_pivot_tile(const T *Tk, int ld, T *P, int32_t *err_flag, bool fp64) {
  // one buffer for either arithmetic (dfloat and double are both 8 bytes)
  constexpr int kSweepBytes = (64 * 65 + 65 + 64) * 8;
  constexpr int kBytes = (int)sizeof(Inverse64Smem) > kSweepBytes ? (int)sizeof(Inverse64Smem) : kSweepBytes;
  __shared__ __align__(16) unsigned char pv_smem[kBytes];
  if constexpr (std::is_same<T, float>::value && NT >= 512) {
    if (!fp64) {
      // the diagonal tile is kept symmetric; the lower half is what is read
      sym_inverse64_df_2x2<NT>(Tk, ld, P, *reinterpret_cast<Inverse64Smem *>(pv_smem), err_flag);
      return;
    }
  }
  if constexpr (std::is_same<T, float>::value) {
    if (!fp64) {
      dfloat *Sf = reinterpret_cast<dfloat *>(pv_smem);
      dfloat *colf = Sf + 64 * 65, *wvf = colf + 65;
#pragma unroll 4
      for (int idx = threadIdx.x; idx < 64 * 16; idx += NT) {
        const int r = idx >> 4, c4 = (idx & 15) * 4;
        const float4 v = *reinterpret_cast<const float4 *>(Tk + (int64_t)r * ld + c4);
        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (r >= c4 + u) Sf[r * 65 + c4 + u] = dfloat{vv[u], 0.0f};
      }
      __syncthreads();
      sym_sweep_inverse64_lower_df<NT>(Sf, 65, colf, wvf, err_flag);
      for (int idx = threadIdx.x; idx < 64 * 64; idx += NT) {
        const int r = idx >> 6, c = idx & 63;
        const dfloat v = Sf[(r >= c) ? r * 65 + c : c * 65 + r];
        P[idx] = -__fadd_rn(v.hi, v.lo);
      }
      return;
    }
  }
  double *S = reinterpret_cast<double *>(pv_smem);
  double *col = S + 64 * 65, *wv = col + 65;
  for (int idx = threadIdx.x; idx < 64 * 64; idx += NT) {
    const int r = idx >> 6, c = idx & 63;
    if (r >= c) S[r * 65 + c] = (double)Tk[(int64_t)r * ld + c];
  }
  __syncthreads();
  sym_sweep_inverse64_lower<NT>(S, 65, col, wv, err_flag);
  for (int idx = threadIdx.x; idx < 64 * 64; idx += NT) {
    const int r = idx >> 6, c = idx & 63;
    P[idx] = (T)(-S[(r >= c) ? r * 65 + c : c * 65 + r]);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_sweep_pivot(SweepBatch<T> bt, int k, int ld, int32_t *err_flag) {
  const SweepEntry<T> e = bt.e[blockIdx.x];
  invert_pivot_tile<256>(e.A + (int64_t)k * 64 * ld + k * 64, ld, e.P, err_flag, bt.pivot_fp64 != 0);
}

template <typename T>
__global__ void __launch_bounds__(256) k_sweep_panel(SweepBatch<T> bt, int k, int ld) {
  __shared__ TileSmem<T> sm;
  const SweepEntry<T> e = bt.e[blockIdx.y];
  const int i = (int)blockIdx.x < k ? (int)blockIdx.x : (int)blockIdx.x + 1;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  T *U = e.U + (int64_t)i * 64 * 64;
  T *V = e.V + (int64_t)i * 64 * 64;
  if (i > k) {
    const T *C = e.A + (int64_t)i * 64 * ld + k * 64;
    tile_mma<false, false>(sm, C, ld, e.P, 64, 64, acc);
    for (int idx = threadIdx.x; idx < 4096; idx += 256) V[idx] = C[(int64_t)(idx >> 6) * ld + (idx & 63)];
  } else {
    // A_ik = (A_ki)^T, tile (k, i) is in the lower triangle
    const T *C = e.A + (int64_t)k * 64 * ld + i * 64;
    tile_mma<true, false>(sm, C, ld, e.P, 64, 64, acc);
    for (int idx = threadIdx.x; idx < 4096; idx += 256) V[idx] = C[(int64_t)(idx & 63) * ld + (idx >> 6)];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) U[(ty + 16 * a) * 64 + tx + 16 * b] = acc[a][b];
}

// ---------------------------------------------------------------------------
// Panel-blocked sweep (tensor-core path).  Pivoting the tiles of a panel
// K = {k0, ..., k0 + bw - 1} one after the other changes an entry A_ij with
// i, j outside K by - sum_k U^(k)_i V^(k)_j^T, V^(k) being column k as it
// stands when k is pivoted and U^(k) = V^(k) P_k.  Those columns depend on the
// earlier pivots of the panel only through the panel's own columns, so the
// column panel A[:, K] is gathered into W (n_pad x 64 bw, row stride
// 64 kSweepPanel), swept there pivot by pivot, and the rest of the matrix
// receives one rank-64 bw update C -= [U^(k)] [V^(k)]^T on the tensor cores
// (which also overwrites rows and columns K; the scatter restores them).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_bsweep_gather(SweepBatch<T> bt, int k0, int bw, int ld, int buf) {
  __shared__ T S[64 * 65];
  const SweepEntry<T> e = bt.e[blockIdx.y];
  constexpr int ldw = 64 * kSweepPanel;
  const int i = blockIdx.x;
  for (int q = 0; q < bw; ++q) {
    const int j = k0 + q;
    // A_ij lives in tile (max(i, j), min(i, j)) of the lower triangle
    const T *src = e.A + (int64_t)max(i, j) * 64 * ld + min(i, j) * 64;
    for (int idx = threadIdx.x; idx < 4096; idx += 256)
      S[(idx >> 6) * 65 + (idx & 63)] = src[(int64_t)(idx >> 6) * ld + (idx & 63)];
    __syncthreads();
    T *dst = (buf ? e.Wp[1] : e.Wp[0]) + (int64_t)i * 64 * ldw + q * 64;
    for (int idx = threadIdx.x; idx < 4096; idx += 256) {
      const int r = idx >> 6, c = idx & 63;
      const bool direct = i > j || (i == j && r >= c);
      dst[(int64_t)r * ldw + c] = direct ? S[r * 65 + c] : S[c * 65 + r];
    }
    __syncthreads();
  }
}

// Pivot k = k0 + q of the panel: P = W_kq^-1 (FP64), and Vk = rows K of
// column q as they stand before the pivot.
constexpr int kPivotThreads = 512;

// P and Vk of pivot q of a panel of parity buf, kept until the rows outside
// the panel have taken the panel's pivots: 2 kSweepPanel slots of each
template <typename T>
__device__ __forceinline__ T *pivot_P(const SweepEntry<T> &e, int buf, int q) {
  return e.P + (int64_t)(buf * kSweepPanel + q) * 4096;
}
template <typename T>
__device__ __forceinline__ T *pivot_Vk(const SweepEntry<T> &e, int buf, int q) {
  return e.Vk + (int64_t)(buf * kSweepPanel + q) * kSweepPanel * 4096;
}

template <typename T>
__global__ void __launch_bounds__(kPivotThreads) k_bsweep_pivot(SweepBatch<T> bt, int k0, int q, int bw, int buf,
                                                                int32_t *err_flag) {
  const SweepEntry<T> e = bt.e[blockIdx.x];
  constexpr int ldw = 64 * kSweepPanel;
  const T *W = (buf ? e.Wp[1] : e.Wp[0]);
  T *Vk = pivot_Vk(e, buf, q);
  // 16-byte rows: ldw, q * 64 and the Vk row length are multiples of 4 elements
  constexpr int V = 16 / sizeof(T);
  using Vec = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
#pragma unroll 4
  for (int idx = threadIdx.x; idx < bw * 64 * (64 / V); idx += kPivotThreads) {
    const int r = idx / (64 / V), c = (idx % (64 / V)) * V;
    *reinterpret_cast<Vec *>(Vk + r * 64 + c) =
        *reinterpret_cast<const Vec *>(W + (int64_t)(k0 * 64 + r) * ldw + q * 64 + c);
  }
  invert_pivot_tile<kPivotThreads>(W + (int64_t)(k0 + q) * 64 * ldw + q * 64, ldw, pivot_P(e, buf, q), err_flag,
                                   bt.pivot_fp64 != 0);
}

// One pivot on the panel, CTA per row tile i:
//   U_i = W_iq P,  V_i = W_iq           (saved at column q of U, V)
//   W_ij -= U_i Vk_j^T                  (panel columns j != q)
//   W_iq <- U_i,  W_kj <- U_j^T (j in K),  W_kq <- -P.
// Row k belongs to no CTA's update, so the writes never overlap.  The 64 x 64
// products stage both operands whole in shared memory, the left one
// transposed (sA[kk][r]); each thread owns the 4 x 4 block at rows 4 ty,
// columns 4 tx and reads 4 + 4 operands per k with two 16-byte loads.
constexpr int kPanelLd = 68;   // padded shared row: 16-byte aligned, staggered banks

__device__ __forceinline__ void panel_mma64(const float *sA, const float *sB, float acc[4][4]) {
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll 8
  for (int kk = 0; kk < 64; ++kk) {
    const float4 a = *reinterpret_cast<const float4 *>(sA + kk * kPanelLd + 4 * ty);
    const float4 b = *reinterpret_cast<const float4 *>(sB + kk * kPanelLd + 4 * tx);
    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
  }
}

// dst[kk][r] = src[r][kk] for a 64 x 64 tile at src (row stride lds); lanes
// take consecutive rows so that the shared stores do not conflict
__device__ __forceinline__ void panel_load_transposed(float *dst, const float *src, int64_t lds) {
  for (int e = threadIdx.x; e < 64 * 16; e += 256) {
    const int r = e & 63, k4 = (e >> 6) * 4;
    const float4 v = *reinterpret_cast<const float4 *>(src + r * lds + k4);
    dst[(k4 + 0) * kPanelLd + r] = v.x;
    dst[(k4 + 1) * kPanelLd + r] = v.y;
    dst[(k4 + 2) * kPanelLd + r] = v.z;
    dst[(k4 + 3) * kPanelLd + r] = v.w;
  }
}

// A 64 x 64 tile (row stride lds) into registers, 4 float4 per thread: element
// group e = threadIdx.x + 256 m holds row e & 63, columns 4 (e >> 6) .. + 3.
__device__ __forceinline__ void tile_to_regs(const float *src, int64_t lds, float4 (&r)[4]) {
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int e = threadIdx.x + 256 * m;
    r[m] = *reinterpret_cast<const float4 *>(src + (int64_t)(e & 63) * lds + (e >> 6) * 4);
  }
}
// the same groups into shared memory transposed: dst[kk][r] = tile[r][kk]
__device__ __forceinline__ void regs_to_smem_transposed(float *dst, const float4 (&r)[4]) {
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int e = threadIdx.x + 256 * m;
    const int row = e & 63, k4 = (e >> 6) * 4;
    dst[(k4 + 0) * kPanelLd + row] = r[m].x;
    dst[(k4 + 1) * kPanelLd + row] = r[m].y;
    dst[(k4 + 2) * kPanelLd + row] = r[m].z;
    dst[(k4 + 3) * kPanelLd + row] = r[m].w;
  }
}

// Pivot q of the panel on row tile i != k of the panel W (CTA-wide; sA, sB
// staging of 64 x kPanelLd floats each).  Wk: row tile k's panel row, written
// with U_i^T when i lies in the panel (else null).  Every global operand is
// loaded into registers a step ahead of its use, so that the CTA waits on
// memory about once per product instead of once per load.
__device__ __forceinline__ void panel_row_step(float *Wi, float *Ui, float *Vi, const float *P, const float *Vk,
                                               float *Wk, int q, int bw, float *sA, float *sB) {
  constexpr int ldw = 64 * kSweepPanel;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  float4 w[4], pr[4], vk[4];
  tile_to_regs(Wi + q * 64, ldw, w);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int idx = threadIdx.x + 256 * m;
    pr[m] = *reinterpret_cast<const float4 *>(P + (idx >> 4) * 64 + (idx & 15) * 4);
  }
  int jj = (q == 0) ? 1 : 0;   // first panel column other than q
  if (jj < bw) tile_to_regs(Vk + jj * 4096, 64, vk);
  regs_to_smem_transposed(sA, w);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int idx = threadIdx.x + 256 * m;
    *reinterpret_cast<float4 *>(sB + (idx >> 4) * kPanelLd + (idx & 15) * 4) = pr[m];
    // V_i = A_ik before the pivot
    const int e = idx;
    *reinterpret_cast<float4 *>(Vi + (int64_t)(e & 63) * ldw + (e >> 6) * 4) = w[m];
  }
  __syncthreads();
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
  panel_mma64(sA, sB, acc);
  __syncthreads();  // sA is reused for U_i below; column q of W was read
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int r = 4 * ty + a;
    const float4 v = make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
    *reinterpret_cast<float4 *>(Ui + (int64_t)r * ldw + 4 * tx) = v;
    *reinterpret_cast<float4 *>(Wi + (int64_t)r * ldw + q * 64 + 4 * tx) = v;
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int c = 4 * tx + b;
    const float4 v = make_float4(acc[0][b], acc[1][b], acc[2][b], acc[3][b]);
    // U_i^T staged as the left operand of the updates: sA[kk][r] = U_i[r][kk]
    *reinterpret_cast<float4 *>(sA + c * kPanelLd + 4 * ty) = v;
    if (Wk) *reinterpret_cast<float4 *>(Wk + (int64_t)c * ldw + 4 * ty) = v;
  }
  while (jj < bw) {
    int nx = jj + 1;
    if (nx == q) ++nx;
    __syncthreads();  // sB free, sA complete
    // sB[kk][c] = Vk_jj[c][kk]
    regs_to_smem_transposed(sB, vk);
    if (nx < bw) tile_to_regs(Vk + nx * 4096, 64, vk);
    float4 wij[4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
      wij[a] = *reinterpret_cast<const float4 *>(Wi + (int64_t)(4 * ty + a) * ldw + jj * 64 + 4 * tx);
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
    panel_mma64(sA, sB, acc);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      float4 w2 = wij[a];
      w2.x -= acc[a][0];
      w2.y -= acc[a][1];
      w2.z -= acc[a][2];
      w2.w -= acc[a][3];
      *reinterpret_cast<float4 *>(Wi + (int64_t)(4 * ty + a) * ldw + jj * 64 + 4 * tx) = w2;
    }
    jj = nx;
  }
}

// Pivot q of the panel on the panel's own row tiles i = k0 + blockIdx.x (the
// rows the next pivot reads).  Row k takes -P; the other rows the step above.
template <typename T>
__global__ void __launch_bounds__(256) k_bsweep_panel(SweepBatch<T> bt, int k0, int q, int bw, int buf) {
  static_assert(std::is_same<T, float>::value, "the panel-blocked sweep runs on float tiles");
  __shared__ __align__(16) float sA[64 * kPanelLd];
  __shared__ __align__(16) float sB[64 * kPanelLd];
  const SweepEntry<T> e = bt.e[blockIdx.y];
  constexpr int ldw = 64 * kSweepPanel;
  const int i = k0 + blockIdx.x, k = k0 + q;
  float *Wi = (buf ? e.Wp[1] : e.Wp[0]) + (int64_t)i * 64 * ldw;
  float *Ui = (buf ? e.Up[1] : e.Up[0]) + (int64_t)i * 64 * ldw + q * 64;
  float *Vi = (buf ? e.Vp[1] : e.Vp[0]) + (int64_t)i * 64 * ldw + q * 64;
  const float *P = pivot_P(e, buf, q);
  if (i == k) {
    for (int idx = threadIdx.x; idx < 4096; idx += 256) {
      const int64_t o = (int64_t)(idx >> 6) * ldw + (idx & 63);
      Wi[o + q * 64] = -P[idx];
      Ui[o] = 0.0f;
      Vi[o] = 0.0f;
    }
    return;
  }
  float *Wk = (buf ? e.Wp[1] : e.Wp[0]) + (int64_t)k * 64 * ldw + (i - k0) * 64;
  panel_row_step(Wi, Ui, Vi, P, pivot_Vk(e, buf, q), Wk, q, bw, sA, sB);
}

// Column panel back into the lower tiles: A_ij for j in K from W row tile i
// (transposed into tile (j, i) when i < j; panel rows i < j come from row j).
template <typename T>
__global__ void __launch_bounds__(256) k_bsweep_scatter(SweepBatch<T> bt, int k0, int bw, int ld, int buf) {
  __shared__ T S[64 * 65];
  const SweepEntry<T> e = bt.e[blockIdx.y];
  constexpr int ldw = 64 * kSweepPanel;
  // CTA per (row tile i, panel column q)
  const int i = (int)blockIdx.x / bw, q = (int)blockIdx.x % bw;
  const bool in_panel = i >= k0 && i < k0 + bw;
  // the swept panel: rows K in W, the other rows in U (= W A_KK^-1)
  const T *src = (in_panel ? (buf ? e.Wp[1] : e.Wp[0]) : (buf ? e.Up[1] : e.Up[0])) + (int64_t)i * 64 * ldw + q * 64;
  const int j = k0 + q;
  if (i >= j) {
    T *dst = e.A + (int64_t)i * 64 * ld + j * 64;
    for (int idx = threadIdx.x; idx < 4096; idx += 256)
      dst[(int64_t)(idx >> 6) * ld + (idx & 63)] = src[(int64_t)(idx >> 6) * ldw + (idx & 63)];
  } else if (!in_panel) {
    for (int idx = threadIdx.x; idx < 4096; idx += 256)
      S[(idx >> 6) * 65 + (idx & 63)] = src[(int64_t)(idx >> 6) * ldw + (idx & 63)];
    __syncthreads();
    T *dst = e.A + (int64_t)j * 64 * ld + i * 64;
    for (int idx = threadIdx.x; idx < 4096; idx += 256) {
      const int r = idx >> 6, c = idx & 63;
      dst[(int64_t)r * ld + c] = S[c * 65 + r];
    }
  }
}

// Look-ahead: the next panel K' was gathered before the update of panel K
// reached it.  Its rows outside K get that update as a small tensor-core
// product; its rows K are final in panel K's U (rows K' of the swept panel,
// where A_{K', K} stands), and are copied transposed here:
// Wp[nxt](K, :) = Up[cur](K', 0 : 64 bw)^T.
// CTA per (a, c) tile pair, a < bw rows of K, c < bw1 columns of K'.
template <typename T>
__global__ void __launch_bounds__(256) k_bsweep_rows(SweepBatch<T> bt, int k0, int bw, int k1, int bw1, int cur) {
  __shared__ T S[64 * 65];
  const SweepEntry<T> e = bt.e[blockIdx.y];
  constexpr int ldw = 64 * kSweepPanel;
  const int a = (int)blockIdx.x / bw1, c = (int)blockIdx.x % bw1;
  const T *src = (cur ? e.Up[1] : e.Up[0]) + (int64_t)(k1 + c) * 64 * ldw + a * 64;
  T *dst = (cur ? e.Wp[0] : e.Wp[1]) + (int64_t)(k0 + a) * 64 * ldw + c * 64;
  for (int idx = threadIdx.x; idx < 4096; idx += 256)
    S[(idx >> 6) * 65 + (idx & 63)] = src[(int64_t)(idx >> 6) * ldw + (idx & 63)];
  __syncthreads();
  for (int idx = threadIdx.x; idx < 4096; idx += 256) {
    const int r = idx >> 6, cc = idx & 63;
    dst[(int64_t)r * ldw + cc] = S[cc * 65 + r];
  }
  (void)bw;
}

template <typename T>
__global__ void __launch_bounds__(256) k_sweep_update(SweepBatch<T> bt, int k, int nt, int ld) {
  __shared__ TileSmem<T> sm;
  const SweepEntry<T> e = bt.e[blockIdx.y];
  // linear index over lower tiles (i >= j): i = floor((sqrt(8 l + 1) - 1) / 2)
  const int l = blockIdx.x;
  int i = (int)((sqrt(8.0 * l + 1.0) - 1.0) * 0.5);
  while ((i + 1) * (i + 2) / 2 <= l) ++i;
  while (i * (i + 1) / 2 > l) --i;
  const int j = l - i * (i + 1) / 2;
  T *Tij = e.A + (int64_t)i * 64 * ld + j * 64;
  if (i == k && j == k) {
    for (int idx = threadIdx.x; idx < 4096; idx += 256) Tij[(int64_t)(idx >> 6) * ld + (idx & 63)] = -e.P[idx];
    return;
  }
  if (j == k) {  // i > k: A_ik <- U_i
    const T *U = e.U + (int64_t)i * 4096;
    for (int idx = threadIdx.x; idx < 4096; idx += 256) Tij[(int64_t)(idx >> 6) * ld + (idx & 63)] = U[idx];
    return;
  }
  if (i == k) {  // j < k: tile (k, j) holds A_kj = A_jk^T <- U_j^T
    const T *U = e.U + (int64_t)j * 4096;
    for (int idx = threadIdx.x; idx < 4096; idx += 256) {
      const int r = idx >> 6, c = idx & 63;
      Tij[(int64_t)r * ld + c] = U[c * 64 + r];
    }
    return;
  }
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  tile_mma<false, true>(sm, e.U + (int64_t)i * 4096, 64, e.V + (int64_t)j * 4096, 64, 64, acc);
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      T *p = Tij + (int64_t)(ty + 16 * a) * ld + tx + 16 * b;
      *p -= acc[a][b];
    }
  (void)nt;
}

// A <- sign * A from the lower tiles, mirrored into the upper triangle (after
// the sweep the lower tiles hold -A^-1, so the sweep mirrors with sign -1).
template <typename T>
__global__ void __launch_bounds__(256) k_sweep_mirror(SweepBatch<T> bt, int ld, double sign) {
  __shared__ T S[64 * 65];
  const SweepEntry<T> e = bt.e[blockIdx.y];
  const T sg = (T)sign;
  const int l = blockIdx.x;
  int i = (int)((sqrt(8.0 * l + 1.0) - 1.0) * 0.5);
  while ((i + 1) * (i + 2) / 2 <= l) ++i;
  while (i * (i + 1) / 2 > l) --i;
  const int j = l - i * (i + 1) / 2;
  T *Tij = e.A + (int64_t)i * 64 * ld + j * 64;
  for (int idx = threadIdx.x; idx < 4096; idx += 256) {
    const int r = idx >> 6, c = idx & 63;
    S[r * 65 + c] = Tij[(int64_t)r * ld + c];
  }
  __syncthreads();
  if (i == j) {
    for (int idx = threadIdx.x; idx < 4096; idx += 256) {
      const int r = idx >> 6, c = idx & 63;
      Tij[(int64_t)r * ld + c] = sg * ((r >= c) ? S[r * 65 + c] : S[c * 65 + r]);
    }
  } else {
    T *Tji = e.A + (int64_t)j * 64 * ld + i * 64;
    for (int idx = threadIdx.x; idx < 4096; idx += 256) {
      const int r = idx >> 6, c = idx & 63;
      Tij[(int64_t)r * ld + c] = sg * S[r * 65 + c];
      Tji[(int64_t)r * ld + c] = sg * S[c * 65 + r];
    }
  }
}

static std::atomic<int> g_sweep_serial{0}, g_update_ctas{0}, g_update_stages{2}, g_pivot_shared{0};
int sweep_serial() { return g_sweep_serial.load(); }
int update_cta_cap() { return g_update_ctas.load(); }
int update_stages() { return g_update_stages.load(); }
int pivot_exclusive() { return !g_pivot_shared.load(); }
// Unused dynamic shared memory that keeps a pivot CTA (42 KB static) off the
// SMs of the persistent rank-64 bw update (129 KB): 42 + 64 + 129 KB plus the
// per-CTA reserve exceed the SM's 228 KB, so the pivot runs on an SM that the
// update leaves free, beside panel CTAs only.
constexpr int kPivotPad = 64 * 1024;

template <typename T>
void spd_inverse(cudaStream_t s, const SweepBatch<T> &b, int n_pad, int32_t *err_flag, int tc_passes,
                 const SweepStreams *ss) {
  if (b.count <= 0) return;
  if (sweep_serial()) ss = nullptr;
  const int nt = n_pad / 64;
  const int n_lower = nt * (nt + 1) / 2;
  if constexpr (std::is_same<T, float>::value) {
    if (tc_passes > 0) {
      // Panels of kSweepPanel pivots K.  The pivots sweep the panel's own rows
      // K in turn (pivot tile inverse, then the panel step on rows K), which
      // leaves W_KK = -A_KK^-1; every other row takes the whole panel at once,
      // U_i = W_iK (-W_KK) = A_iK A_KK^-1 (the block form of the same sweep), and
      // the rest of the matrix the rank-64 bw update A -= U W^T.  On hi (the
      // critical path): the pivots, then the next panel's rows K' (their U),
      // its gather, its look-ahead product on rows K' and its rows K; the next
      // panel's pivots follow at once.  On lo: U on every other row, the
      // look-ahead on those rows, the update and the scatter.  Buffers (W, U,
      // V, P, Vk) alternate with the panel's parity; the events order the two
      // streams' shared rows.
      constexpr int ldw = 64 * kSweepPanel;
      cudaStream_t hi = s, lo = s;
      if (ss) {
        hi = ss->hi;
        lo = ss->lo;
        cudaEventRecord(ss->fork, s);
        cudaStreamWaitEvent(hi, ss->fork, 0);
        cudaStreamWaitEvent(lo, ss->fork, 0);
      }
      const bool split_ops = tc_passes == 3 && b.e[0].Sp[0] != nullptr;
      // C = alpha A B^T + beta C0 through the tensor cores, timed under class cls
      auto tc_update = [&](cudaStream_t st, const GemmBatch<float> &gb, int M, int N, int K, int ldc, bool lower,
                           int cls, double work, bool compact) {
        Profiler::Rec rec{cls, nullptr, nullptr, 0.0};
        const bool prof = g_prof != nullptr;
        if (prof) {
          rec.work = work;
          g_prof->begin(st, rec);
        }
        Profiler *saved = g_prof;
        g_prof = nullptr;  // timed under cls, not as a GEMM
        launch_tc_gemm(st, gb, M, N, K, ldw, ldw, ldc, lower, tc_passes, err_flag, compact);
        g_prof = saved;
        if (prof) g_prof->end(st, rec);
      };
      // the swept panel on row tiles [r0, r1) outside K: U = W (-W_KK); W_KK is
      // symmetric up to rounding, so it serves as the K-major right operand
      auto panel_apply = [&](cudaStream_t st, int cur, int k0, int bw, int r0, int r1, bool compact) {
        if (r1 <= r0) return;
        GemmBatch<float> gb{};
        gb.count = b.count;
        for (int e = 0; e < b.count; ++e) {
          gb.e[e].A = b.e[e].Wp[cur] + (int64_t)r0 * 64 * ldw;
          gb.e[e].B = b.e[e].Wp[cur] + (int64_t)k0 * 64 * ldw;
          gb.e[e].C0 = nullptr;
          gb.e[e].C = b.e[e].Up[cur] + (int64_t)r0 * 64 * ldw;
          gb.e[e].alpha = -1.0;
          gb.e[e].beta = 0.0;
        }
        tc_update(st, gb, 64 * (r1 - r0), 64 * bw, 64 * bw, ldw, false, PROF_PANEL,
                  2.0 * 64.0 * (r1 - r0) * 64.0 * bw * 64.0 * bw * b.count, compact);
      };
      // look-ahead rows [r0, r1) of panel K' = (k1, bw1): W'(r, :) -= U(r, :) W(K', :)^T
      auto lookahead = [&](cudaStream_t st, int cur, int k1, int bw, int bw1, int r0, int r1, bool compact) {
        if (r1 <= r0) return;
        GemmBatch<float> fb{};
        fb.count = b.count;
        for (int e = 0; e < b.count; ++e) {
          fb.e[e].A = b.e[e].Up[cur] + (int64_t)r0 * 64 * ldw;
          fb.e[e].B = b.e[e].Wp[cur] + (int64_t)k1 * 64 * ldw;
          fb.e[e].C0 = b.e[e].Wp[cur ^ 1] + (int64_t)r0 * 64 * ldw;
          fb.e[e].C = b.e[e].Wp[cur ^ 1] + (int64_t)r0 * 64 * ldw;
          fb.e[e].alpha = -1.0;
          fb.e[e].beta = 1.0;
        }
        tc_update(st, fb, 64 * (r1 - r0), 64 * bw1, 64 * bw, ldw, false, PROF_PANEL,
                  2.0 * 64.0 * (r1 - r0) * 64.0 * bw1 * 64.0 * bw * b.count, compact);
      };
      const int n_panels = (nt + kSweepPanel - 1) / kSweepPanel;
      // the update's CTA count, and the pivot CTAs' padding
      int upd_ctas = update_cta_cap();
      int pad = 0;
      if (pivot_exclusive()) {
        static std::once_flag once;
        static bool pad_ok = false;
        std::call_once(once, [] {
          pad_ok = cudaFuncSetAttribute(k_bsweep_pivot<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kPivotPad) == cudaSuccess;
          if (!pad_ok) cudaGetLastError();
        });
        if (pad_ok) {
          pad = kPivotPad;
          if (upd_ctas == 0) {
            int sms = 152, dev = 0;
            if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            upd_ctas = std::max(1, sms - b.count);
          }
        }
      }
      ++g_launch_count;
      {
        ProfScope ps_(hi, PROF_PANEL);
        k_bsweep_gather<T><<<dim3(nt, b.count), 256, 0, hi>>>(b, 0, std::min(kSweepPanel, nt), n_pad, 0);
      }
      for (int p = 0; p < n_panels; ++p) {
        const int k0 = p * kSweepPanel, bw = std::min(kSweepPanel, nt - k0), cur = p & 1;
        const bool has_next = p + 1 < n_panels;
        const int k1 = k0 + bw, bw1 = has_next ? std::min(kSweepPanel, nt - k1) : 0;
        g_launch_count += 2 * bw;
        for (int q = 0; q < bw; ++q) {
          {
            ProfScope ps_(hi, PROF_PIVOT, 2.0 * 64.0 * 64.0 * 64.0 * b.count);
            k_bsweep_pivot<T><<<b.count, kPivotThreads, pad, hi>>>(b, k0, q, bw, cur, err_flag);
          }
          {
            ProfScope ps_(hi, PROF_PANEL);
            k_bsweep_panel<T><<<dim3(bw, b.count), 256, 0, hi>>>(b, k0, q, bw, cur);
          }
        }
        if (has_next) {
          // rows K' of this panel: the previous panel's look-ahead on them ran on lo
          if (ss && p > 0) cudaStreamWaitEvent(hi, ss->lookahead, 0);
          g_launch_count += 2;
          panel_apply(hi, cur, k0, bw, k1, k1 + bw1, split_ops);
          // columns K' as the previous update and scatter left them
          if (ss && p > 0) cudaStreamWaitEvent(hi, ss->scatter, 0);
          {
            ProfScope ps_(hi, PROF_PANEL);
            k_bsweep_gather<T><<<dim3(nt, b.count), 256, 0, hi>>>(b, k1, bw1, n_pad, cur ^ 1);
          }
          // compact tiles: the product runs beside the previous panel's
          // persistent update instead of waiting for its SMs
          lookahead(hi, cur, k1, bw, bw1, k1, k1 + bw1, split_ops);
          {
            ProfScope ps_(hi, PROF_PANEL);
            k_bsweep_rows<T><<<dim3(bw * bw1, b.count), 256, 0, hi>>>(b, k0, bw, k1, bw1, cur);
          }
        }
        if (ss) {
          cudaEventRecord(ss->panel, hi);
          cudaStreamWaitEvent(lo, ss->panel, 0);
        }
        // the swept panel on the other rows (outside K and K'), their look-ahead
        // (rows K come from k_bsweep_rows above), the update of the rest
        const int r1s = has_next ? k1 + bw1 : k1;   // other rows: [0, k0) and [r1s, nt)
        bool fused = false;
        if (split_ops) {
          // W (the products' left operand and the update's right one) and U's
          // rows K' (the look-ahead's right operand) split once
          {
            ProfScope ps_(lo, PROF_PANEL);
            SplitJobs jobs{};
            for (int e = 0; e < b.count; ++e) {
              jobs.j[jobs.count++] = SplitJob{b.e[e].Wp[cur], b.e[e].Sp[2], b.e[e].Sp[3], 0};
              if (has_next) {
                const int64_t off = (int64_t)k1 * 64 * ldw;
                jobs.j[jobs.count++] = SplitJob{b.e[e].Up[cur] + off, b.e[e].Sp[0] + off, b.e[e].Sp[1] + off,
                                                (int64_t)64 * bw1 * ldw};
              }
            }
            launch_split_tf32_jobs(lo, jobs, (int64_t)n_pad * ldw);
          }
          // U = W (-W_KK)^T and W' -= W U_K'^T (= U W_K'^T: W_KK is symmetric)
          // on both row ranges of every matrix: one persistent launch per
          // kMaxBatch products
          Profiler::Rec rec{PROF_PANEL, nullptr, nullptr, 0.0};
          Profiler *saved = g_prof;
          if (saved) saved->begin(lo, rec);
          g_prof = nullptr;
          fused = true;
          SplitGemmBatch gb{};
          auto flush = [&]() {
            if (gb.count > 0 && !launch_tc_gemm_split(lo, gb, n_pad, 64 * kSweepPanel, 64 * bw, ldw, ldw, ldw, false,
                                                      err_flag))
              fused = false;
            gb.count = 0;
          };
          for (int e = 0; e < b.count && fused; ++e) {
            const int ranges[2][2] = {{0, k0}, {r1s, nt}};
            for (const auto &rg : ranges) {
              if (rg[1] <= rg[0]) continue;
              const int64_t ro = (int64_t)rg[0] * 64 * ldw;
              const int rows = 64 * (rg[1] - rg[0]);
              if (gb.count == kMaxBatch) flush();
              gb.e[gb.count++] = SplitGemmEntry{b.e[e].Sp[2] + ro, b.e[e].Sp[3] + ro,
                                                b.e[e].Sp[2] + (int64_t)k0 * 64 * ldw,
                                                b.e[e].Sp[3] + (int64_t)k0 * 64 * ldw, nullptr, b.e[e].Up[cur] + ro,
                                                -1.0f, 0.0f, rows, 64 * bw};
              if (has_next) {
                if (gb.count == kMaxBatch) flush();
                gb.e[gb.count++] = SplitGemmEntry{b.e[e].Sp[2] + ro, b.e[e].Sp[3] + ro,
                                                  b.e[e].Sp[0] + (int64_t)k1 * 64 * ldw,
                                                  b.e[e].Sp[1] + (int64_t)k1 * 64 * ldw, b.e[e].Wp[cur ^ 1] + ro,
                                                  b.e[e].Wp[cur ^ 1] + ro, -1.0f, 1.0f, rows, 64 * bw1};
              }
            }
          }
          flush();
          g_prof = saved;
          if (saved) saved->end(lo, rec);
        }
        if (!fused) {
          panel_apply(lo, cur, k0, bw, 0, k0, false);
          panel_apply(lo, cur, k0, bw, r1s, nt, false);
          if (has_next) {
            lookahead(lo, cur, k1, bw, bw1, 0, k0, false);
            lookahead(lo, cur, k1, bw, bw1, r1s, nt, false);
          }
        }
        if (ss && has_next) cudaEventRecord(ss->lookahead, lo);
        if (nt > bw) {
          // algorithmic work: the rank-64 bw update of the lower tiles off the
          // panel's rows and columns
          const double rest = (double)(nt - bw) * (nt - bw + 1) / 2.0;
          const double work = 2.0 * 64.0 * 64.0 * 64.0 * bw * rest * b.count;
          if (split_ops) {
            // U split (W was split above, or is split here), then the
            // persistent 3xTF32 update
            {
              ProfScope ps_(lo, PROF_PANEL);
              SplitJobs jobs{};
              for (int e = 0; e < b.count; ++e) {
                jobs.j[jobs.count++] = SplitJob{b.e[e].Up[cur], b.e[e].Sp[0], b.e[e].Sp[1], 0};
                if (!fused) jobs.j[jobs.count++] = SplitJob{b.e[e].Wp[cur], b.e[e].Sp[2], b.e[e].Sp[3], 0};
              }
              launch_split_tf32_jobs(lo, jobs, (int64_t)n_pad * ldw);
            }
            Profiler::Rec rec{PROF_SWEEP, nullptr, nullptr, work};
            Profiler *saved = g_prof;
            if (saved) saved->begin(lo, rec);
            bool done = false;
            if (update_stages() == 4) {
              // the persistent 128 x 256-tile kernel over the lower tiles (the
              // tiles' parts above the diagonal are written too; the sweep
              // reads lower tiles only)
              g_prof = nullptr;
              SplitGemmBatch ug{};
              for (int e = 0; e < b.count; ++e)
                ug.e[ug.count++] = SplitGemmEntry{b.e[e].Sp[0], b.e[e].Sp[1], b.e[e].Sp[2], b.e[e].Sp[3], b.e[e].A,
                                                  b.e[e].A, -1.0f, 1.0f};
              done = launch_tc_gemm_split(lo, ug, n_pad, n_pad, 64 * bw, ldw, ldw, n_pad, true, err_flag, upd_ctas);
              g_prof = saved;
            }
            if (!done) {
              UpdateBatch ub{};
              ub.count = b.count;
              for (int e = 0; e < b.count; ++e)
                ub.e[e] = UpdateEntry{b.e[e].Sp[0], b.e[e].Sp[1], b.e[e].Sp[2], b.e[e].Sp[3], b.e[e].A};
              launch_tc_update(lo, ub, n_pad, 64 * bw, ldw, -1.0f, 1.0f, err_flag, upd_ctas);
            }
            if (saved) saved->end(lo, rec);
          } else {
            GemmBatch<float> gb{};
            gb.count = b.count;
            for (int e = 0; e < b.count; ++e) {
              gb.e[e].A = b.e[e].Up[cur];
              gb.e[e].B = b.e[e].Wp[cur];
              gb.e[e].C0 = b.e[e].A;
              gb.e[e].C = b.e[e].A;
              gb.e[e].alpha = -1.0;
              gb.e[e].beta = 1.0;
            }
            tc_update(lo, gb, n_pad, n_pad, 64 * bw, n_pad, true, PROF_SWEEP, work, false);
          }
        }
        ++g_launch_count;
        {
          ProfScope ps_(lo, PROF_PANEL);
          k_bsweep_scatter<T><<<dim3(nt * bw, b.count), 256, 0, lo>>>(b, k0, bw, n_pad, cur);
        }
        if (ss) cudaEventRecord(ss->scatter, lo);
      }
      if (ss) cudaStreamWaitEvent(s, ss->scatter, 0);
      ++g_launch_count;
      {
        ProfScope ps_(s, PROF_PANEL);
        k_sweep_mirror<T><<<dim3(n_lower, b.count), 256, 0, s>>>(b, n_pad, -1.0);
      }
      return;
    }
  }
  for (int k = 0; k < nt; ++k) {
    g_launch_count += 3;
    {
      ProfScope ps_(s, PROF_PIVOT, 2.0 * 64.0 * 64.0 * 64.0 * b.count);
      k_sweep_pivot<T><<<b.count, 256, 0, s>>>(b, k, n_pad, err_flag);
    }
    {
      ProfScope ps_(s, PROF_PANEL);
      if (nt > 1) k_sweep_panel<T><<<dim3(nt - 1, b.count), 256, 0, s>>>(b, k, n_pad);
    }
    Profiler::Rec rec{PROF_SWEEP, nullptr, nullptr, 0.0};
    if (g_prof) {
      // rank-64 update of the lower tiles off row/column k: 2 * 64^3 FLOPs each
      const double upd = (double)n_lower - nt;
      rec.work = 2.0 * 64.0 * 64.0 * 64.0 * upd * b.count;
      g_prof->begin(s, rec);
    }
    k_sweep_update<T><<<dim3(n_lower, b.count), 256, 0, s>>>(b, k, nt, n_pad);
    if (g_prof) g_prof->end(s, rec);
  }
  ++g_launch_count;
  {
    ProfScope ps_(s, PROF_PANEL);
    k_sweep_mirror<T><<<dim3(n_lower, b.count), 256, 0, s>>>(b, n_pad, -1.0);
  }
}
template void spd_inverse<double>(cudaStream_t, const SweepBatch<double> &, int, int32_t *, int,
                                  const SweepStreams *);
template void spd_inverse<float>(cudaStream_t, const SweepBatch<float> &, int, int32_t *, int, const SweepStreams *);

template <typename T>
void launch_mirror(cudaStream_t s, const SweepBatch<T> &b, int n_pad) {
  if (b.count <= 0) return;
  const int nt = n_pad / 64;
  ++g_launch_count;
  {
    ProfScope ps_(s, PROF_PANEL);
    k_sweep_mirror<T><<<dim3(nt * (nt + 1) / 2, b.count), 256, 0, s>>>(b, n_pad, 1.0);
  }
}
template void launch_mirror<double>(cudaStream_t, const SweepBatch<double> &, int);
template void launch_mirror<float>(cudaStream_t, const SweepBatch<float> &, int);

// ---------------------------------------------------------------------------
// Out = alpha M B + beta C on the spatial pattern (row gather; M = the entry's
// symmetric spatial block, values e.val): one warp per
// row, the row's pattern entries staged once in the warp's shared slots, then
// four 64-column chunks at a time (2 elements per lane per chunk, eight
// independent loads per pattern entry).  Accumulation in the output type.
// ---------------------------------------------------------------------------
template <typename TI, typename TO>
__global__ void __launch_bounds__(256) k_sp_rowgather(SpBatch<TI, TO> bt, SellPattern pat, int n_s, int n_pad,
                                                      int ncol, int ldb, int ldo) {
  extern __shared__ __align__(16) unsigned char rg_smem[];
  const SpEntry<TI, TO> e = bt.e[blockIdx.y];
  const double *__restrict__ val = e.val;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int *w_col = reinterpret_cast<int *>(rg_smem) + warp * pat.max_width;
  TO *w_val = reinterpret_cast<TO *>(reinterpret_cast<int *>(rg_smem) + 8 * pat.max_width) + warp * pat.max_width;
  const int nch = ncol / 64;
  const TO alpha = (TO)(e.alpha * (e.alpha_ptr ? *e.alpha_ptr : 1.0));
  const bool add_c = e.C != nullptr && e.beta != 0.0;
  const TO beta = (TO)e.beta;
  for (int row = blockIdx.x * 8 + warp; row < n_pad; row += gridDim.x * 8) {
    int w = 0;
    if (row < n_s) {
      const int sl = row >> 5, li = row & 31;
      w = pat.slice_width[sl];
      const int base = pat.slice_ptr[sl] + li;
      for (int s = lane; s < w; s += 32) {
        w_col[s] = pat.col[base + s * kSlice];
        w_val[s] = (TO)val[base + s * kSlice];
      }
    }
    __syncwarp();
    TO *orow = e.Out + (int64_t)row * ldo;
    const TO *crow = add_c ? e.C + (int64_t)row * ldo : nullptr;
    for (int ch0 = 0; ch0 < nch; ch0 += 4) {
      TO acc[4][2];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u][0] = acc[u][1] = TO(0);
      for (int s = 0; s < w; ++s) {
        const TI *bp = e.B + (int64_t)w_col[s] * ldb + 2 * lane;
        const TO v = w_val[s];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (ch0 + u < nch) {
            const int col = (ch0 + u) * 64;
            acc[u][0] = fma(v, (TO)bp[col], acc[u][0]);
            acc[u][1] = fma(v, (TO)bp[col + 1], acc[u][1]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (ch0 + u < nch) {
          const int col = (ch0 + u) * 64 + 2 * lane;
          TO a0 = acc[u][0] * alpha, a1 = acc[u][1] * alpha;
          if (add_c) {
            a0 = fma(beta, crow[col], a0);
            a1 = fma(beta, crow[col + 1], a1);
          }
          orow[col] = a0;
          orow[col + 1] = a1;
        }
      }
    }
    __syncwarp();  // the slots are refilled for the next row
  }
}

template <typename TI, typename TO>
void launch_sp_rowgather(cudaStream_t s, const SpBatch<TI, TO> &b, const SellPattern &pat, int n_s, int n_pad,
                         int ncol, int ldb, int ldo) {
  if (b.count <= 0) return;
  ++g_launch_count;
  int grid = (n_pad + 7) / 8;
  if (grid > 152 * 8) grid = 152 * 8;
  const size_t smem = (size_t)8 * pat.max_width * (sizeof(int) + sizeof(TO));
  {
    ProfScope ps_(s, PROF_GATHER);
    k_sp_rowgather<TI, TO><<<dim3(grid, b.count), 256, smem, s>>>(b, pat, n_s, n_pad, ncol, ldb, ldo);
  }
}
template void launch_sp_rowgather<double, double>(cudaStream_t, const SpBatch<double, double> &,
                                                  const SellPattern &, int, int, int, int, int);
template void launch_sp_rowgather<float, float>(cudaStream_t, const SpBatch<float, float> &, const SellPattern &,
                                                int, int, int, int, int);
template void launch_sp_rowgather<double, float>(cudaStream_t, const SpBatch<double, float> &,
                                                 const SellPattern &, int, int, int, int, int);

// ---------------------------------------------------------------------------
// Column gathers over the symmetric pattern, (B Q_s)[r, l] =
// sum_{j in pat(l)} B[r, j] Q_s[l, j].  A block covers 256 columns and
// kGatherRows rows; each thread keeps its column's pattern (j, Q_s[l, j]) in
// its own shared slots [s * 256 + t] (no sharing, no block barrier) and reuses
// it for every row.  Shared memory: max_width * 256 * (4 + sizeof(T)) bytes.
// ---------------------------------------------------------------------------
constexpr int kGatherRows = 64;   // rows per block (a multiple of kGatherRowBlock)
constexpr int kGatherRowBlock = 4; // rows per thread at a time: one pattern read, four FMAs

template <typename T>
__device__ __forceinline__ int stage_col_pattern(const SellPattern &pat, const double *__restrict__ val, int l,
                                                 int n_s, int *s_col, T *s_val) {
  if (l >= n_s) return 0;
  const int sl = l >> 5, li = l & 31;
  const int w = pat.slice_width[sl];
  const int base = pat.slice_ptr[sl] + li;
  for (int s = 0; s < w; ++s) {
    s_col[s * 256 + threadIdx.x] = pat.col[base + s * kSlice];
    s_val[s * 256 + threadIdx.x] = (T)val[base + s * kSlice];
  }
  return w;
}

template <typename T>
size_t col_pattern_smem(const SellPattern &pat) {
  return (size_t)pat.max_width * 256 * (sizeof(int) + sizeof(T));
}

// Out = alpha B M + beta C (M = the entry's symmetric spatial block); rows and
// columns past n_s of Out are zero.  With B = D^-1 (symmetric) this is
// (M D^-1)^T.
template <typename T>
__global__ void __launch_bounds__(256) k_sp_colgather(SpBatch<T, T> bt, SellPattern pat, int n_s, int n_pad) {
  extern __shared__ __align__(16) unsigned char cg_smem[];
  int *s_col = reinterpret_cast<int *>(cg_smem);
  T *s_val = reinterpret_cast<T *>(s_col + pat.max_width * 256);
  const SpEntry<T, T> e = bt.e[blockIdx.z];
  const int l = blockIdx.x * 256 + threadIdx.x;
  if (l >= n_pad) return;
  const int w = stage_col_pattern(pat, e.val, l, n_s, s_col, s_val);
  const T alpha = (T)(e.alpha * (e.alpha_ptr ? *e.alpha_ptr : 1.0));
  const bool add_c = e.C != nullptr && e.beta != 0.0;
  const int r0 = blockIdx.y * kGatherRows, r1 = min(n_pad, r0 + kGatherRows);
  for (int r = r0; r < r1; r += kGatherRowBlock) {
    // kGatherRowBlock rows per pattern entry read (n_pad is a multiple of 64)
    T acc[kGatherRowBlock];
#pragma unroll
    for (int q = 0; q < kGatherRowBlock; ++q) acc[q] = T(0);
    if (l < n_s && r < n_s) {
      const T *Br = e.B + (int64_t)r * n_pad;
      for (int s = 0; s < w; ++s) {
        const int j = s_col[s * 256 + threadIdx.x];
        const T v = s_val[s * 256 + threadIdx.x];
#pragma unroll
        for (int q = 0; q < kGatherRowBlock; ++q) acc[q] = fma(Br[(int64_t)q * n_pad + j], v, acc[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < kGatherRowBlock; ++q) {
      const int rq = r + q;
      T out = T(0);
      if (rq < n_s && l < n_s) {
        out = alpha * acc[q];
        if (add_c) out = fma((T)e.beta, e.C[(int64_t)rq * n_pad + l], out);
      }
      e.Out[(int64_t)rq * n_pad + l] = out;
    }
  }
}

template <typename T>
void launch_sp_colgather(cudaStream_t s, const SpBatch<T, T> &b, const SellPattern &pat, int n_s, int n_pad) {
  if (b.count <= 0) return;
  ++g_launch_count;
  dim3 grid((n_pad + 255) / 256, (n_pad + kGatherRows - 1) / kGatherRows, b.count);
  {
    ProfScope ps_(s, PROF_GATHER);
    k_sp_colgather<T><<<grid, 256, col_pattern_smem<T>(pat), s>>>(b, pat, n_s, n_pad);
  }
}
template void launch_sp_colgather<double>(cudaStream_t, const SpBatch<double, double> &, const SellPattern &, int,
                                          int);
template void launch_sp_colgather<float>(cudaStream_t, const SpBatch<float, float> &, const SellPattern &, int, int);

// diag_out[i] = D0[i, i] + sum_l P[i, l] R[i, l] accumulated in double (one
// warp per row, coalesced along the row): the diagonal of
// Sigma_t = D_t^-1 + Y^T W with P = Y^T and R = W^T.
template <typename T>
__global__ void __launch_bounds__(256) k_diag64_rows(DiagRowBatch<T> bt, int n_s, int n_pad) {
  const DiagRowEntry<T> e = bt.e[blockIdx.y];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + warp;
  if (i >= n_s) return;
  const T *Pi = e.P + (int64_t)i * n_pad;
  const T *Ri = e.R + (int64_t)i * n_pad;
  double acc = 0.0;
  if constexpr (std::is_same<T, float>::value) {
    // 16-byte loads; four products summed in binary32 (about 4 units of
    // roundoff of that partial), the partials in double: a quarter of the
    // FP64 operations.  Entries past n_s are zero in both operands.
    for (int l = 4 * lane; l < n_pad; l += 128) {
      const float4 p = *reinterpret_cast<const float4 *>(Pi + l);
      const float4 r = *reinterpret_cast<const float4 *>(Ri + l);
      acc += (double)fmaf(p.w, r.w, fmaf(p.z, r.z, fmaf(p.y, r.y, p.x * r.x)));
    }
  } else {
    for (int l = lane; l < n_s; l += 32) acc = fma((double)Pi[l], (double)Ri[l], acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) e.diag_out[i] = (double)e.D0[(int64_t)i * n_pad + i] + acc;
}

template <typename T>
void launch_diag64_rows(cudaStream_t s, const DiagRowBatch<T> &b, int n_s, int n_pad) {
  if (b.count <= 0) return;
  ++g_launch_count;
  {
    ProfScope ps_(s, PROF_EXTRACT);
    k_diag64_rows<T><<<dim3((n_s + 7) / 8, b.count), 256, 0, s>>>(b, n_s, n_pad);
  }
}
template void launch_diag64_rows<double>(cudaStream_t, const DiagRowBatch<double> &, int, int);
template void launch_diag64_rows<float>(cudaStream_t, const DiagRowBatch<float> &, int, int);

// ---------------------------------------------------------------------------
// D = a0 A_t + w_obs diag(obs) - c W B (column gather over the symmetric
// pattern: (W B)[r, l] = sum_{j in pat(l)} W[r, j] B[l, j], B = the coupling
// B_{t-1} without its scale c), blocked and staged like k_sp_colgather.  The
// Schur term accumulates in T.  Entries off the pattern are -c times the
// Schur sum in T; afterwards each thread
// rewrites the entries of its column on the pattern (and the diagonal), at
// most max_width of them, combining the terms in double.  Keeping that path
// out of the row loop keeps the FP64 pipe out of the common case.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T schur_sum(const T *__restrict__ Wr, int w, const int *s_col, const T *s_val) {
  T acc = T(0);
  for (int s = 0; s < w; ++s) acc = fma(Wr[s_col[s * 256 + threadIdx.x]], s_val[s * 256 + threadIdx.x], acc);
  return acc;
}

template <typename T>
__global__ void __launch_bounds__(256) k_schur_assemble(SchurBatch<T> bt, SellPattern pat, double obs_w, int n_s,
                                                        int n_pad) {
  extern __shared__ __align__(16) unsigned char sa_smem[];
  int *s_col = reinterpret_cast<int *>(sa_smem);
  T *s_val = reinterpret_cast<T *>(s_col + pat.max_width * 256);
  const SchurEntry<T> e = bt.e[blockIdx.z];
  const int l = blockIdx.x * 256 + threadIdx.x;
  if (l >= n_pad) return;
  const int w = stage_col_pattern(pat, e.W ? e.cval : e.dval, l, n_s, s_col, s_val);
  const double *__restrict__ dval = e.dval;
  const T neg_c = e.W ? (T)(-(e.c ? *e.c : 1.0)) : T(0);
  const int r0 = blockIdx.y * kGatherRows, r1 = min(n_pad, r0 + kGatherRows);
  if (e.accumulate) {
    // a second Schur term on the spatial block (the middle slab of a
    // two-ended factorisation), combined in double like the pattern entries
    if (l >= n_s || !e.W) return;
    const double c = e.c ? *e.c : 1.0;
    for (int r = r0; r < min(r1, n_s); ++r) {
      T *d = e.D + (int64_t)r * n_pad + l;
      *d = (T)((double)*d - c * (double)schur_sum(e.W + (int64_t)r * n_pad, w, s_col, s_val));
    }
    return;
  }
  for (int r = r0; r < r1; r += kGatherRowBlock) {
    // kGatherRowBlock rows per pattern entry read (n_pad is a multiple of 64)
    T acc[kGatherRowBlock];
#pragma unroll
    for (int q = 0; q < kGatherRowBlock; ++q) acc[q] = T(0);
    if (e.W && l < n_s && r < n_s) {
      const T *Wr = e.W + (int64_t)r * n_pad;
      for (int s = 0; s < w; ++s) {
        const int j = s_col[s * 256 + threadIdx.x];
        const T v = s_val[s * 256 + threadIdx.x];
#pragma unroll
        for (int q = 0; q < kGatherRowBlock; ++q) acc[q] = fma(Wr[(int64_t)q * n_pad + j], v, acc[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < kGatherRowBlock; ++q) {
      const int rq = r + q;
      T out;
      if (rq < n_s && l < n_s)
        out = e.W ? neg_c * acc[q] : T(0);
      else
        out = (rq == l) ? T(1) : T(0);
      e.D[(int64_t)rq * n_pad + l] = out;
    }
  }
  if (l >= n_s) return;
  // entries on the pattern of column l within this block's rows, in double.
  // A row can fill several slots (padding slots repeat the diagonal with a
  // zero value): its first slot sums them all.
  const int base = pat.slice_ptr[l >> 5] + (l & 31);
  const double a0 = e.a0 ? *e.a0 : 1.0;
  const double c = e.W ? (e.c ? *e.c : 1.0) : 0.0;
  bool diag_seen = false;
  for (int s = 0; s <= w; ++s) {
    int r;
    double aq = 0.0;
    if (s < w) {
      r = s_col[s * 256 + threadIdx.x];
      diag_seen |= (r == l);
      if (r < r0 || r >= r1 || r >= n_s) continue;
      bool first = true;
      for (int q = 0; q < s; ++q) first &= (s_col[q * 256 + threadIdx.x] != r);
      if (!first) continue;
      for (int q = s; q < w; ++q)
        if (s_col[q * 256 + threadIdx.x] == r) aq += dval[base + q * kSlice];
    } else {
      if (diag_seen) break;
      r = l;  // a diagonal outside the pattern still gets its observation term
      if (r < r0 || r >= r1) continue;
    }
    double o = a0 * aq;
    if (r == l && e.obs && e.obs[r]) o += obs_w;
    if (e.W) o -= c * (double)schur_sum(e.W + (int64_t)r * n_pad, w, s_col, s_val);
    e.D[(int64_t)r * n_pad + l] = (T)o;
  }
}

template <typename T>
void launch_schur_assemble(cudaStream_t s, const SchurBatch<T> &b, const SellPattern &pat, double obs_w, int n_s,
                           int n_pad) {
  if (b.count <= 0) return;
  ++g_launch_count;
  dim3 grid((n_pad + 255) / 256, (n_pad + kGatherRows - 1) / kGatherRows, b.count);
  {
    ProfScope ps_(s, PROF_SCHUR);
    k_schur_assemble<T><<<grid, 256, col_pattern_smem<T>(pat), s>>>(b, pat, obs_w, n_s, n_pad);
  }
}
// Opt the pattern-staging kernels in to the shared memory that
// max_width needs (beyond the default 48 KB); false when it cannot be had.
bool configure_pattern_kernels(const SellPattern &pat) {
  const int cg_d = (int)col_pattern_smem<double>(pat), cg_f = (int)col_pattern_smem<float>(pat);
  const int rg_d = 8 * pat.max_width * (int)(sizeof(int) + sizeof(double));
  const int rg_f = 8 * pat.max_width * (int)(sizeof(int) + sizeof(float));
  bool ok = true;
  ok &= cudaFuncSetAttribute(k_sp_colgather<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, cg_d) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_sp_colgather<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, cg_f) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_schur_assemble<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, cg_d) ==
        cudaSuccess;
  ok &= cudaFuncSetAttribute(k_schur_assemble<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, cg_f) ==
        cudaSuccess;
  ok &= cudaFuncSetAttribute(k_sp_rowgather<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, rg_d) ==
        cudaSuccess;
  ok &= cudaFuncSetAttribute(k_sp_rowgather<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, rg_f) ==
        cudaSuccess;
  ok &= cudaFuncSetAttribute(k_sp_rowgather<double, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, rg_f) ==
        cudaSuccess;
  if (!ok) cudaGetLastError();
  return ok;
}

template void launch_schur_assemble<double>(cudaStream_t, const SchurBatch<double> &, const SellPattern &, double,
                                            int, int);
template void launch_schur_assemble<float>(cudaStream_t, const SchurBatch<float> &, const SellPattern &, double, int,
                                           int);

// ---------------------------------------------------------------------------
// diag(S) and the pattern inner products <M_j, S> with the entry's spatial
// derivative blocks M_j (j < n_sums) in double (one block per entry, fixed
// reduction order).  With D0 set, the diagonal is
// instead diag(D0) + diag(D0 V) accumulated in double over column chunks
// (k_diag64), D0 symmetric so that D0[i, l] = D0[l, i] reads coalesce.
// ---------------------------------------------------------------------------
constexpr int kDiagChunks = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_diag64(ExtractBatch<T> bt, int n_s, int n_pad, double *partial) {
  const ExtractEntry<T> e = bt.e[blockIdx.z];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_s || e.D0 == nullptr || e.diag_out == nullptr) return;
  const int chunk = (n_s + kDiagChunks - 1) / kDiagChunks;
  const int l0 = blockIdx.y * chunk, l1 = min(n_s, l0 + chunk);
  double acc = 0.0;
  for (int l = l0; l < l1; ++l) acc = fma((double)e.D0[(int64_t)l * n_pad + i], (double)e.V[(int64_t)l * n_pad + i], acc);
  partial[((int64_t)blockIdx.z * kDiagChunks + blockIdx.y) * n_pad + i] = acc;
}

template <typename T>
__global__ void __launch_bounds__(1024) k_extract(ExtractBatch<T> bt, SellPattern pat, int n_sums, int n_s, int n_pad,
                                                  const double *__restrict__ diag_partial) {
  __shared__ double red[kMaxTheta][32];
  const ExtractEntry<T> e = bt.e[blockIdx.x];
  double acc[kMaxTheta] = {0.0, 0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < n_s; i += blockDim.x) {
    const T *Si = e.S + (int64_t)i * n_pad;
    if (e.diag_out) {
      if (e.D0) {
        double d = (double)e.D0[(int64_t)i * n_pad + i];
        for (int c = 0; c < kDiagChunks; ++c) d += diag_partial[((int64_t)blockIdx.x * kDiagChunks + c) * n_pad + i];
        e.diag_out[i] = d;
      } else {
        e.diag_out[i] = (double)Si[i];
      }
    }
    if (e.sums) {
      const int sl = i >> 5, li = i & 31;
      const int w = pat.slice_width[sl];
      const int base = pat.slice_ptr[sl] + li;
      for (int s = 0; s < w; ++s) {
        const int idx = base + s * kSlice;
        const double sv = (double)Si[pat.col[idx]];
#pragma unroll
        for (int j = 0; j < kMaxTheta; ++j)
          if (j < n_sums) acc[j] = fma(e.sv[j][idx], sv, acc[j]);
      }
    }
  }
  if (!e.sums) return;
#pragma unroll
  for (int j = 0; j < kMaxTheta; ++j) {
    for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_down_sync(0xffffffffu, acc[j], o);
    if ((threadIdx.x & 31) == 0) red[j][threadIdx.x >> 5] = acc[j];
  }
  __syncthreads();
  if (threadIdx.x < n_sums) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[threadIdx.x][w];
    e.sums[threadIdx.x] = a;
  }
}

// Scratch for the FP64 diagonal partials (per device, grown on demand by the
// context through extract_scratch_bytes()).
size_t extract_scratch_bytes(int n_pad) { return (size_t)kMaxBatch * kDiagChunks * n_pad * sizeof(double); }

template <typename T>
void launch_extract(cudaStream_t s, const ExtractBatch<T> &b, const SellPattern &pat, int n_sums, int n_s,
                    int n_pad, double *diag_scratch) {
  if (b.count <= 0) return;
  bool any_d0 = false;
  for (int q = 0; q < b.count; ++q) any_d0 |= (b.e[q].D0 != nullptr);
  if (any_d0) {
    ++g_launch_count;
    {
      ProfScope ps_(s, PROF_EXTRACT);
      k_diag64<T><<<dim3((n_s + 255) / 256, kDiagChunks, b.count), 256, 0, s>>>(b, n_s, n_pad, diag_scratch);
    }
  }
  ++g_launch_count;
  {
    ProfScope ps_(s, PROF_EXTRACT);
    k_extract<T><<<b.count, 1024, 0, s>>>(b, pat, n_sums, n_s, n_pad, diag_scratch);
  }
}
template void launch_extract<double>(cudaStream_t, const ExtractBatch<double> &, const SellPattern &, int, int, int,
                                     double *);
template void launch_extract<float>(cudaStream_t, const ExtractBatch<float> &, const SellPattern &, int, int, int,
                                    double *);

}  // namespace qsel

extern "C" qsel_status qsel_debug_sweep_schedule(int32_t serial, int32_t update_ctas, int32_t update_stages,
                                                 int32_t shared_pivot) {
  if (update_ctas < 0 || (update_stages != 0 && update_stages != 2 && update_stages != 3 && update_stages != 4))
    return QSEL_EINVAL;
  qsel::g_sweep_serial.store(serial ? 1 : 0);
  qsel::g_update_ctas.store(update_ctas);
  qsel::g_update_stages.store(update_stages == 0 ? 2 : update_stages);
  qsel::g_pivot_shared.store(shared_pivot ? 1 : 0);
  return QSEL_OK;
}
