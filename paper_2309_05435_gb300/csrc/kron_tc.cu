// Kronecker preconditioner on the tcgen05 tensor cores (mixed form).
//
// The apply z = Dh (U (x) V (x) V) S (U (x) V (x) V)^T Dh r of kron.cu as one
// transposition and six contractions.  Every contraction multiplies along the
// axis that is contiguous in memory, so both MMA operands are K-major and the
// sample block is never transposed in shared memory: the 128 rows of a tile
// run along the axis that the NEXT pass contracts (a 4-D TMA box), and the
// epilogue writes that axis contiguously.  Axes s (samples, ld), t (n_t),
// i, j (m); layouts slowest axis first:
//   r (t, i, j, s)  --transpose, x Dh_i Dh_j-->                  (s, t, i, j)
//   P1  V^T over j, rows along i (32) x t (4)                ->  (s, t, j, i)
//   P2  V^T over i, rows along t (128)                        ->  (s, j, i, t)
//   P3  U^T over t, x spectral scaling, rows along i x j     ->  (s, t, j, i)
//       (the scaling 1 / (tau mu_t (kappa^2 + lambda_i + lambda_j)^2 + omega)
//       is formed in the epilogue from mu and lambda, in binary32)
//   P4  V over i, rows along j (32) x t (4)                   ->  (s, t, i, j)
//   P5  V over j, rows along t (128)                          ->  (s, i, j, t)
//   P6  U over t, x Dh_i Dh_j, rows along s (128)             ->  z (t, i, j, s)
// A pass computes D[row][o] = sum_k X[row][k] op(B)[o][k] for every tile of
// 128 rows, N = dim rounded up to 16, 3xTF32 (hi*hi + hi*lo + lo*hi, FP32
// accumulation): the tables are split into TF32 parts once per theta, the
// sample tiles by converter warps.  Persistent CTAs, one per SM:
//   warp 0     one thread issues the TMA loads (X tile, op(B) hi / lo chunks)
//              into a 2- or 3-stage ring;
//   warp 1     owns two accumulators of N TMEM columns; one thread issues the
//              MMAs of tile i into accumulator i % 2;
//   warps 2-5  split each X chunk into hi (in place) and lo;
//   warps 6-9  epilogue, while the MMAs of the next tile run: tcgen05.ld of
//              32 columns, output scaling, the values written to a shared
//              staging tile laid out as the output box (double-buffered), and
//              one TMA tensor store per 32 columns (the TMA writes full lines
//              and leaves out what lies outside the tensor).
// Every wait is bounded: after the limit the CTA raises bit 1 of *err, stops
// issuing work, waits (bounded) for its loads and MMAs in flight, frees its
// tensor memory and returns.
#include <mutex>

#include "qsel.h"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace qsel {
namespace ktc {
using namespace tc;

constexpr int MR = 128;                  // rows per tile (MMA M)
constexpr int ATILE = MR * BK * 4;       // 16 KiB: 128 rows x 128 bytes
constexpr int THREADS = 320;
constexpr int kMaxSmem = 227 * 1024;
constexpr int OCH = 32;                  // output columns per staged store
constexpr int YTILE = MR * OCH * 4;      // 16 KiB staging tile

struct Params {
  CUtensorMap tmX;            // input: dims {K, d1, d2, d3}, box {32, box1, box2, box3}
  CUtensorMap tmB[2];         // op(B) hi, lo: K rows x K (row o, column k), boxes of np rows
  CUtensorMap tmY;            // output: 4-D, no swizzle, box = the tile's rows x 32 columns
  // output scaling: 0 none; 1 spectral 1 / (tau mu_o (kappa^2 + lambda_i +
  // lambda_j)^2 + omega), formed here from mu, lambda; 2 dh_i dh_j
  int smode, dim_i, dim_j;    // input dims (1..3) that hold the spatial indices i, j of a row
  const double *mu, *lam;
  const float *dhdh;
  float tau, kappa2, omega;
  int m;
  int K, np, stages;
  int size[4], box[4], ntile[4];
  int ysrc[4];                // output dim e (innermost first) is input dim ysrc[e] (0 = the new index o)
  int ystage[4];              // staging-tile element stride of input dim a (0 = o)
  int tiles;
  int32_t *err;
  long long wait_cycles;
};

__host__ __device__ constexpr int stage_bytes(int np) { return 2 * ATILE + 2 * np * BK * 4; }
__host__ __device__ constexpr uint32_t tmem_cols(int np) {
  return np <= 32 ? 32u : np <= 64 ? 64u : np <= 128 ? 128u : 256u;
}
__host__ __device__ constexpr int smem_bytes(int np, int stages) {
  return stages * stage_bytes(np) + 2 * YTILE + 256 + 1024;
}

__device__ __forceinline__ void conv_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 2, 128;" ::: "memory"); }

// kind::tf32 instruction descriptor for M = 128 and N = n (multiple of 16)
__device__ __forceinline__ uint32_t idesc_n(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(MR >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32_n(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tile_origin(const Params &p, int L, int &x1, int &x2, int &x3) {
  const int c1 = L % p.ntile[1];
  const int rest = L / p.ntile[1];
  const int c2 = rest % p.ntile[2];
  const int c3 = rest / p.ntile[2];
  x1 = c1 * p.box[1];
  x2 = c2 * p.box[2];
  x3 = c3 * p.box[3];
}

// Bounded wait used after an abort (no error is raised a second time).
__device__ __forceinline__ void drain(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  uint32_t done = 0;
  while (!done && clock64() - t0 < kWaitCycles) {
    asm volatile(
        "{\n\t.reg .pred r;\n\tmbarrier.try_wait.parity.shared::cta.b64 r, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, r;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
  }
}

__global__ void __launch_bounds__(THREADS, 1) k_kron_tc(const __grid_constant__ Params p) {
  extern __shared__ unsigned char smem_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int S = p.stages;
  const int SB = stage_bytes(p.np), BT = p.np * BK * 4;
  float *ystage = reinterpret_cast<float *>(base + S * SB);   // two staging tiles
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + S * SB + 2 * YTILE);
  // bars: [0, S) full, [S, 2S) converted, [2S, 3S) empty, [3S, 3S+2) accumulator
  // full, [3S+2, 3S+4) accumulator empty, [3S+4] all MMAs done
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 3 * S + 5);
  volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
  volatile int *cv_ok = abort + 1;
  volatile int *ep_ok = abort + 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto conv_bar = [&](int s) { return bar0 + 8u * (S + s); };
  auto empty_bar = [&](int s) { return bar0 + 8u * (2 * S + s); };
  auto accf_bar = [&](int b) { return bar0 + 8u * (3 * S + b); };
  auto acce_bar = [&](int b) { return bar0 + 8u * (3 * S + 2 + b); };
  const uint32_t fin_bar = bar0 + 8u * (3 * S + 4);
  const uint32_t ncols = tmem_cols(p.np);
  const int nk = (p.K + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(conv_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf_bar(b), 1);
      mbar_init(acce_bar(b), 1);
    }
    mbar_init(fin_bar, 1);
    *abort = 0;
    *cv_ok = 1;
    *ep_ok = 1;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      long long g = 0;   // chunks issued
      bool go = true;
      for (int L = blockIdx.x; L < p.tiles && go; L += gridDim.x) {
        int x1, x2, x3;
        tile_origin(p, L, x1, x2, x3);
        for (int kc = 0; kc < nk; ++kc) {
          const int s = (int)(g % S);
          const uint32_t u = (uint32_t)(g / S);
          if (!mbar_wait(empty_bar(s), (u & 1) ^ 1, abort, p.err, p.wait_cycles)) {
            go = false;
            break;
          }
          uint8_t *st = base + s * SB;
          mbar_expect_tx(full_bar(s), ATILE + 2 * BT);
          tma_load_4d(smem_u32(st), &p.tmX, kc * BK, x1, x2, x3, full_bar(s));
          tma_load_2d(smem_u32(st + 2 * ATILE), &p.tmB[0], kc * BK, 0, full_bar(s));
          tma_load_2d(smem_u32(st + 2 * ATILE + BT), &p.tmB[1], kc * BK, 0, full_bar(s));
          ++g;
        }
      }
      if (*abort) {
        // let the loads already issued land before the CTA's shared memory goes away
        for (long long q = (g > S ? g - S : 0); q < g; ++q)
          drain(full_bar((int)(q % S)), (uint32_t)((q / S) & 1));
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_n(p.np);
      long long g = 0;
      int i = 0;
      bool go = true;
      for (int L = blockIdx.x; L < p.tiles && go; L += gridDim.x, ++i) {
        const int b = i & 1;
        const uint32_t ub = (uint32_t)(i >> 1);
        if (!mbar_wait(acce_bar(b), (ub & 1) ^ 1, abort, p.err, p.wait_cycles)) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)b * ncols;
        for (int kc = 0; kc < nk; ++kc, ++g) {
          const int s = (int)(g % S);
          const uint32_t u = (uint32_t)(g / S);
          // the converters arrive only after the stage's TMA has landed
          if (!mbar_wait(conv_bar(s), u & 1, abort, p.err, p.wait_cycles)) {
            go = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(base + s * SB);
          const uint32_t a_hi = st, a_lo = st + ATILE, b_hi = st + 2 * ATILE, b_lo = b_hi + BT;
#pragma unroll
          for (int j = 0; j < BK / 8; ++j) {
            const uint32_t off = j * 32;
            mma_tf32_n(d, smem_desc(a_hi + off), smem_desc(b_hi + off), idesc, (kc | j) != 0);
            mma_tf32_n(d, smem_desc(a_hi + off), smem_desc(b_lo + off), idesc, 1u);
            mma_tf32_n(d, smem_desc(a_lo + off), smem_desc(b_hi + off), idesc, 1u);
          }
          mma_commit(empty_bar(s));
        }
        if (!go) break;
        mma_commit(accf_bar(b));
      }
      mma_commit(fin_bar);   // arrives once every MMA issued above has completed
    }
  } else if (warp < 6) {
    // converters: hi = rn(x) in place, lo = rn(x - hi) at the same swizzled
    // position of the lo tile
    const int ct = threadIdx.x - 64;
    long long g = 0;
    bool stop = false;
    for (int L = blockIdx.x; L < p.tiles && !stop; L += gridDim.x) {
      for (int kc = 0; kc < nk; ++kc, ++g) {
        const int s = (int)(g % S);
        const uint32_t u = (uint32_t)(g / S);
        if (ct == 0) *cv_ok = (mbar_wait(full_bar(s), u & 1, abort, p.err, p.wait_cycles) && !*abort) ? 1 : 0;
        conv_sync();
        if (!*cv_ok) {
          stop = true;
          break;
        }
        float4 *raw = reinterpret_cast<float4 *>(base + s * SB);
        float4 *lo = reinterpret_cast<float4 *>(base + s * SB + ATILE);
#pragma unroll 4
        for (int e = ct; e < ATILE / 16; e += 128) {
          const float4 v = raw[e];
          float4 h;
          h.x = tf32_rn(v.x);
          h.y = tf32_rn(v.y);
          h.z = tf32_rn(v.z);
          h.w = tf32_rn(v.w);
          raw[e] = h;
          lo[e] = make_float4(tf32_rn(v.x - h.x), tf32_rn(v.y - h.y), tf32_rn(v.z - h.z), tf32_rn(v.w - h.w));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        conv_sync();
        if (ct == 0) mbar_arrive(conv_bar(s));
      }
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 = tile rows
    const int q = warp & 3;
    const int et = threadIdx.x - 192;
    const int r = 32 * q + lane;
    const int r1 = r % p.box[1], r2 = (r / p.box[1]) % p.box[2], r3 = r / (p.box[1] * p.box[2]);
    // this row's place in a staging tile; consecutive lanes are consecutive
    // elements of the output's innermost dimension
    const int yrow = r1 * p.ystage[1] + r2 * p.ystage[2] + r3 * p.ystage[3];
    const int ycol = p.ystage[0];
    int i = 0, ec = 0;
    for (int L = blockIdx.x; L < p.tiles; L += gridDim.x, ++i) {
      const int b = i & 1;
      const uint32_t ub = (uint32_t)(i >> 1);
      if (et == 0) *ep_ok = (mbar_wait(accf_bar(b), ub & 1, abort, p.err, p.wait_cycles) && !*abort) ? 1 : 0;
      epi_sync();
      if (!*ep_ok) break;   // uniform across the four warps: tcgen05.ld is warp-collective
      tc_fence_after();
      int x[4];
      tile_origin(p, L, x[1], x[2], x[3]);
      const int c1 = x[1] + r1, c2 = x[2] + r2, c3 = x[3] + r3;
      const bool valid = c1 < p.size[1] && c2 < p.size[2] && c3 < p.size[3];
      // the row's spatial indices and its part of the scaling
      const int cc[4] = {0, c1, c2, c3};
      float s2sq = 0.0f, rs = 1.0f;
      if (valid && p.smode == 1) {
        const float s2 = p.kappa2 + (float)p.lam[cc[p.dim_i]] + (float)p.lam[cc[p.dim_j]];
        s2sq = s2 * s2;
      } else if (valid && p.smode == 2) {
        rs = p.dhdh[cc[p.dim_i] * p.m + cc[p.dim_j]];
      }
      for (int oc = 0; oc < p.np; oc += OCH, ++ec) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)b * ncols + (uint32_t)oc, v);
        float *yt = ystage + (ec & 1) * (YTILE / 4);
        // tau mu_o of column oc + lane, passed along the warp below
        const float tmu = (p.smode == 1 && oc + lane < p.K) ? p.tau * (float)p.mu[oc + lane] : 0.0f;
        // the store that last used this staging tile has read it
        if (ec >= 2 && et == 0) bulk_wait_read<1>();
        epi_sync();
        if (p.smode == 1) {
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) {
            // a preconditioner's scaling: the fast divide (a few ulp) suffices
            const float den = fmaf(__shfl_sync(0xffffffffu, tmu, jj), s2sq, p.omega);
            yt[yrow + jj * ycol] = __fdividef(__uint_as_float(v[jj]), den);
          }
        } else {
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) yt[yrow + jj * ycol] = __uint_as_float(v[jj]) * rs;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        epi_sync();
        if (et == 0) {
          x[0] = oc;
          tma_store_4d(&p.tmY, smem_u32(yt), x[p.ysrc[0]], x[p.ysrc[1]], x[p.ysrc[2]], x[p.ysrc[3]]);
          bulk_commit();
        }
      }
      tc_fence_before();
      epi_sync();   // every epilogue thread has read the accumulator
      if (et == 0) mbar_arrive(acce_bar(b));
    }
    if (et == 0) bulk_wait_all();   // the staged stores are complete before the CTA exits
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    if (lane == 0) drain(fin_bar, 0u);   // no MMA may still write the accumulators
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * ncols) : "memory");
  }
}

// x[s][row] = r[row][s] dh_i dh_j (row = (t m + i) m + j): the sample block
// transposed so that the samples become the slowest axis; 32 x 32 tiles
// through shared memory, both sides coalesced.
__global__ void __launch_bounds__(256) k_kron_transpose_in(const float *__restrict__ r, float *__restrict__ x,
                                                           const float *__restrict__ dhdh, int64_t n, int ld,
                                                           int mm) {
  __shared__ float tile[32][33];
  const int64_t row0 = (int64_t)blockIdx.x * 32;
  const int s0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int k = ty; k < 32; k += 8) {
    const int64_t row = row0 + k;
    tile[k][tx] = row < n ? r[row * ld + s0 + tx] * dhdh[row % mm] : 0.0f;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int64_t row = row0 + tx;
    if (row < n) x[(int64_t)(s0 + k) * n + row] = tile[tx][k];
  }
}

std::once_flag g_attr_once;
bool g_attr_ok = false;

// Axes of the sample block and one pass of the chain above.
enum Axis { AS = 0, AT = 1, AI = 2, AJ = 3 };
struct PassSpec {
  int in[4], out[4];    // layouts, slowest axis first; in[3] is contracted
  int box[4];           // tile rows per axis (product 128), indexed by axis
  int table;            // KronOperator::split index of op(B)
  int scale;            // 0 none, 1 spectral, 2 dh_i dh_j
};

}  // namespace ktc

bool kron_tc_supported(int dim, int ld) { return dim >= 4 && dim <= 256 && dim % 4 == 0 && ld % 32 == 0; }

bool launch_kron_apply_tc(cudaStream_t s, const KronOperator &op, const float *r, float *q, float *z) {
  using namespace ktc;
  const int m = op.m, n_t = op.n_t, ld = op.ld;
  if (!kron_tc_supported(m, ld) || !kron_tc_supported(n_t, ld) || !tc_gemm_available()) return false;
  std::call_once(g_attr_once, [] {
    g_attr_ok = cudaFuncSetAttribute(k_kron_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) == cudaSuccess;
    if (!g_attr_ok) cudaGetLastError();
  });
  if (!g_attr_ok) return false;
  const int64_t sz[4] = {ld, n_t, m, m};
  const int64_t n = (int64_t)n_t * m * m;
  auto strides = [&](const int *lay, int64_t *st) {
    int64_t acc = 1;
    for (int a = 3; a >= 0; --a) {
      st[lay[a]] = acc;
      acc *= sz[lay[a]];
    }
  };
  // the chain of the header, P1 .. P6; box[] is indexed by axis (s, t, i, j)
  static const PassSpec chain[6] = {
      {{AS, AT, AI, AJ}, {AS, AT, AJ, AI}, {1, 4, 32, 1}, 1, 0},
      {{AS, AT, AJ, AI}, {AS, AJ, AI, AT}, {1, 128, 1, 1}, 1, 0},
      {{AS, AJ, AI, AT}, {AS, AT, AJ, AI}, {1, 1, 32, 4}, 3, 1},
      {{AS, AT, AJ, AI}, {AS, AT, AI, AJ}, {1, 4, 1, 32}, 0, 0},
      {{AS, AT, AI, AJ}, {AS, AI, AJ, AT}, {1, 128, 1, 1}, 0, 0},
      {{AS, AI, AJ, AT}, {AT, AI, AJ, AS}, {128, 1, 1, 1}, 2, 2},
  };
  Params ps[6];
  for (int k = 0; k < 6; ++k) {
    const PassSpec &sp = chain[k];
    Params &p = ps[k];
    memset(&p, 0, sizeof(p));
    int64_t sin[4], sout[4];
    strides(sp.in, sin);
    strides(sp.out, sout);
    // tensor dims innermost first: d0 = contracted axis, d1 = in[2], d2 = in[1], d3 = in[0]
    const int dax[4] = {sp.in[3], sp.in[2], sp.in[1], sp.in[0]};
    const int K = (int)sz[dax[0]];
    uint64_t dims[4], bst[3];
    uint32_t box[4];
    int rows = 1;
    for (int a = 0; a < 4; ++a) {
      dims[a] = (uint64_t)sz[dax[a]];
      p.size[a] = (int)sz[dax[a]];
      box[a] = a == 0 ? (uint32_t)BK : (uint32_t)sp.box[dax[a]];
      if (a > 0) {
        bst[a - 1] = (uint64_t)sin[dax[a]] * sizeof(float);
        p.box[a] = (int)box[a];
        p.ntile[a] = (int)((sz[dax[a]] + box[a] - 1) / box[a]);
        rows *= (int)box[a];
      }
    }
    if (rows != MR) return false;
    p.box[0] = BK;
    p.ntile[0] = 1;
    const int64_t tiles = (int64_t)p.ntile[1] * p.ntile[2] * p.ntile[3];
    if (tiles > INT32_MAX) return false;
    p.tiles = (int)tiles;
    // output map: dims innermost first are the out layout's axes reversed;
    // the new index o takes the contracted axis' place
    {
      const int oax[4] = {sp.out[3], sp.out[2], sp.out[1], sp.out[0]};
      uint64_t od[4], ost[3];
      uint32_t obox[4];
      int cum = 1;
      for (int e = 0; e < 4; ++e) {
        int src = -1;
        for (int a = 0; a < 4; ++a)
          if (dax[a] == oax[e]) src = a;
        if (src < 0) return false;
        p.ysrc[e] = src;
        od[e] = (uint64_t)sz[oax[e]];
        if (e > 0) ost[e - 1] = (uint64_t)sout[oax[e]] * sizeof(float);
        obox[e] = src == 0 ? (uint32_t)OCH : (uint32_t)box[src];
        p.ystage[src] = cum;
        cum *= (int)obox[e];
      }
      if (cum != MR * OCH || obox[0] % 4 != 0) return false;
      if (!tc::encode_4d_plain(&p.tmY, (k % 2 == 0) ? q : z, od, ost, obox)) return false;
    }
    p.smode = sp.scale;
    p.dim_i = p.dim_j = 1;
    for (int a = 1; a < 4; ++a) {
      if (dax[a] == AI) p.dim_i = a;
      if (dax[a] == AJ) p.dim_j = a;
    }
    p.mu = op.mu;
    p.lam = op.lam;
    p.dhdh = static_cast<const float *>(op.dhdh);
    p.tau = (float)op.tau;
    p.kappa2 = (float)op.kappa2;
    p.omega = (float)op.omega;
    p.m = m;
    p.K = K;
    p.np = (K + 15) / 16 * 16;
    p.stages = smem_bytes(p.np, 3) <= kMaxSmem ? 3 : 2;
    p.err = op.err;
    p.wait_cycles = tc::wait_limit();
    // the transposition writes z; P1 z -> q, P2 q -> z, ..., P6 q -> z
    const float *xin = (k % 2 == 0) ? z : q;
    if (!tc::encode_4d(&p.tmX, xin, dims, bst, box)) return false;
    const float *bh = op.split[sp.table][0], *bl = op.split[sp.table][1];
    if (!tc::encode_2d(&p.tmB[0], bh, K, K, K, p.np) || !tc::encode_2d(&p.tmB[1], bl, K, K, K, p.np)) return false;
  }
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  g_launch_count += 7;
  k_kron_transpose_in<<<dim3((unsigned)((n + 31) / 32), ld / 32), 256, 0, s>>>(
      r, z, static_cast<const float *>(op.dhdh), n, ld, m * m);
  for (int k = 0; k < 6; ++k) {
    const int grid = std::min(ps[k].tiles, sms);
    k_kron_tc<<<grid, THREADS, smem_bytes(ps[k].np, ps[k].stages), s>>>(ps[k]);
  }
  return true;
}

}  // namespace qsel
