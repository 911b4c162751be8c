// Persistent tensor-core GEMM on pre-split operands (mixed form; the
// Takahashi recursion's products):
//
//   C = alpha A B^T + beta C0    A: M x K, B: N x K, row-major (K-major)
//
// with A and B given as TF32 parts (hi = rn(x), lo = rn(x - hi), k_split_tf32)
// and 3xTF32 products (hi*hi + hi*lo + lo*hi) accumulated in FP32 in tensor
// memory.  Output tiles of 128 x 256: per 32-wide K block a CTA loads 96 KB
// (A hi / lo 16 KB each, B hi / lo 32 KB each) for three 128 x 256 x 32
// products, half the shared-memory and L2 bytes per MMA of 128 x 128 tiles
// whose CTA also splits its operands (the split then costs one pass over each
// operand in HBM).  One CTA per SM walks a static list of tiles: full tiles
// in groups of 8 tile rows (a group's A panels stay in L2 while B streams),
// or the tiles on or below the diagonal.
//   warp 0      one thread issues the TMA loads into a 2-stage ring;
//   warp 1      owns 512 TMEM columns = two 256-column accumulators; one
//               thread issues tcgen05.mma.kind::tf32 (M = 128, N = 256, K = 8)
//               for tile i into accumulator i % 2;
//   warps 2-5   epilogue of the other accumulator: tcgen05.ld, alpha / beta,
//               row-contiguous 16-byte stores.
// Every wait is bounded: after the limit the CTA raises bit 1 of *err, stops
// issuing work, waits (bounded) for its loads and MMAs in flight, frees its
// tensor memory and returns.
#include <mutex>

#include "qsel.h"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace qsel {
namespace tcw {
using namespace tc;

constexpr int BN = 256;
constexpr int STAGES = 2;
constexpr int GROUP = 16;
constexpr int TA = BM * BK * 4;              // 16 KiB
constexpr int TB = BN * BK * 4;              // 32 KiB
constexpr int STAGE_BYTES = 2 * TA + 2 * TB;  // A_hi, A_lo, B_hi, B_lo
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 256 + 1024;
constexpr uint32_t kTmemCols = 2 * BN;

struct Params {
  CUtensorMap tm[kMaxBatch][4];   // A_hi, A_lo (boxes 128 rows), B_hi, B_lo (boxes 256 rows)
  float *C[kMaxBatch];
  const float *C0[kMaxBatch];
  float alpha[kMaxBatch], beta[kMaxBatch];
  int M, N, K, ldc, lower;
  int tiles_m, tiles_n, tiles_per_matrix, total_tiles;
  // ragged batches: every entry its own M and N (full tiles), its tiles at
  // tstart[z] .. tstart[z + 1] - 1 of the static list
  int ragged, count;
  int Mz[kMaxBatch], Nz[kMaxBatch], tm_z[kMaxBatch], tn_z[kMaxBatch], tstart[kMaxBatch + 1];
  int32_t *err;
  long long wait_cycles;
  int skip_loads;
};

// Tile l of one matrix: full tiles in groups of GROUP tile rows (column by
// column inside a group), or the lower tiles row by row.
__device__ __forceinline__ void tile_of(const Params &p, int l, int &bm, int &bn) {
  if (!p.lower) {
    const int per_group = GROUP * p.tiles_n;
    const int g = l / per_group;
    const int g0 = g * GROUP;
    const int rows = min(GROUP, p.tiles_m - g0);
    const int w = l - g * per_group;
    bn = w / rows;
    bm = g0 + (w - bn * rows);
    return;
  }
  int r = 0;
  for (;;) {
    const int cnt = min(p.tiles_n, (r * BM + BM - 1) / BN + 1);
    if (l < cnt) break;
    l -= cnt;
    ++r;
  }
  bm = r;
  bn = l;
}

// Entry z and tile (bm, bn) of static tile L.
__device__ __forceinline__ void tile_at(const Params &p, int L, int &z, int &bm, int &bn) {
  if (!p.ragged) {
    z = L / p.tiles_per_matrix;
    tile_of(p, L - z * p.tiles_per_matrix, bm, bn);
    return;
  }
  z = 0;
  while (z + 1 < p.count && L >= p.tstart[z + 1]) ++z;
  const int l = L - p.tstart[z];
  const int tiles_m = p.tm_z[z], tiles_n = p.tn_z[z];
  const int per_group = GROUP * tiles_n;
  const int g = l / per_group;
  const int g0 = g * GROUP;
  const int rows = min(GROUP, tiles_m - g0);
  const int w = l - g * per_group;
  bn = w / rows;
  bm = g0 + (w - bn * rows);
}

__device__ __forceinline__ void epilogue_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

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

__global__ void __launch_bounds__(192, 1) k_tc_gemm256(const __grid_constant__ Params p) {
  extern __shared__ unsigned char smem_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + STAGES * STAGE_BYTES);
  // bars: [0, S) full, [S, 2S) empty, [2S, 2S+2) accumulator full,
  // [2S+2, 2S+4) accumulator empty, [2S+4] all MMAs done
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 5);
  volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
  volatile int *ep_ok = abort + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = p.K / BK;
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
  auto accf_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
  auto acce_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + 2 + b); };
  const uint32_t fin_bar = bar0 + 8u * (2 * STAGES + 4);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf_bar(b), 1);
      mbar_init(acce_bar(b), 1);
    }
    mbar_init(fin_bar, 1);
    *abort = 0;
    *ep_ok = 1;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      long long g = 0;   // K-blocks issued
      bool go = !p.skip_loads;
      for (int L = blockIdx.x; L < p.total_tiles && go; L += gridDim.x) {
        int z, bm, bn;
        tile_at(p, L, z, bm, bn);
        for (int kb = 0; kb < nk; ++kb) {
          const int s = (int)(g % STAGES);
          const uint32_t u = (uint32_t)(g / STAGES);
          if (!mbar_wait(empty_bar(s), (u & 1) ^ 1, abort, p.err, p.wait_cycles)) {
            go = false;
            break;
          }
          uint8_t *st = base + s * STAGE_BYTES;
          mbar_expect_tx(full_bar(s), STAGE_BYTES);
          tma_load_2d(smem_u32(st), &p.tm[z][0], kb * BK, bm * BM, full_bar(s));
          tma_load_2d(smem_u32(st + TA), &p.tm[z][1], kb * BK, bm * BM, full_bar(s));
          tma_load_2d(smem_u32(st + 2 * TA), &p.tm[z][2], kb * BK, bn * BN, full_bar(s));
          tma_load_2d(smem_u32(st + 2 * TA + TB), &p.tm[z][3], kb * BK, bn * BN, full_bar(s));
          ++g;
        }
      }
      if (*abort) {
        // let the loads already issued land before the CTA's shared memory goes away
        for (long long q = (g > STAGES ? g - STAGES : 0); q < g; ++q)
          drain(full_bar((int)(q % STAGES)), (uint32_t)((q / STAGES) & 1));
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      long long g = 0;
      int i = 0;
      bool go = true;
      for (int L = blockIdx.x; L < p.total_tiles && go; L += gridDim.x, ++i) {
        const int b = i & 1;
        const uint32_t ub = (uint32_t)(i >> 1);
        if (!mbar_wait(acce_bar(b), (ub & 1) ^ 1, abort, p.err, p.wait_cycles)) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * BN);
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = (int)(g % STAGES);
          const uint32_t u = (uint32_t)(g / STAGES);
          if (!mbar_wait(full_bar(s), u & 1, abort, p.err, p.wait_cycles)) {
            go = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(base + s * STAGE_BYTES);
          const uint32_t ah = st, al = st + TA, bh = st + 2 * TA, bl = st + 2 * TA + TB;
#pragma unroll
          for (int j = 0; j < BK / 8; ++j) {
            const uint32_t off = j * 32;
            mma_tf32<BN>(d, smem_desc(ah + off), smem_desc(bh + off), (kb | j) != 0);
            mma_tf32<BN>(d, smem_desc(ah + off), smem_desc(bl + off), 1u);
            mma_tf32<BN>(d, smem_desc(al + off), smem_desc(bh + off), 1u);
          }
          mma_commit(empty_bar(s));
        }
        if (!go) break;
        mma_commit(accf_bar(b));
      }
      mma_commit(fin_bar);   // arrives once every MMA issued above has completed
    }
  } else {
    // epilogue (warps 2-5): warp w reads TMEM lanes 32 (w % 4) .. +31 = tile rows
    const int q = warp & 3;
    int i = 0;
    for (int L = blockIdx.x; L < p.total_tiles; L += gridDim.x, ++i) {
      const int b = i & 1;
      const uint32_t ub = (uint32_t)(i >> 1);
      int z, bm, bn;
      tile_at(p, L, z, bm, bn);
      const int Mlim = p.ragged ? p.Mz[z] : p.M, Nlim = p.ragged ? p.Nz[z] : p.N;
      const int row = bm * BM + 32 * q + lane;
      float *C = p.C[z];
      const float *C0 = p.C0[z];
      const float alpha = p.alpha[z], beta = p.beta[z];
      // a whole row segment in range with C0: C0 is read a chunk ahead, the
      // first chunk while the tile's MMAs still run (it does not depend on them)
      const bool full = row < Mlim && (bn + 1) * BN <= Nlim && C0 != nullptr && beta != 0.0f;
      const float *c0row0 = full ? C0 + (int64_t)row * p.ldc + bn * BN : nullptr;
      float4 cb[2][8];
      if (full) {
#pragma unroll
        for (int j = 0; j < 8; ++j) cb[0][j] = *reinterpret_cast<const float4 *>(c0row0 + 4 * j);
      }
      if (threadIdx.x == 64) *ep_ok = (mbar_wait(accf_bar(b), ub & 1, abort, p.err, p.wait_cycles) && !*abort) ? 1 : 0;
      epilogue_sync();
      if (!*ep_ok) break;   // uniform across the four warps: tcgen05.ld is warp-collective
      tc_fence_after();
      if (full) {
        float *crow0 = C + (int64_t)row * p.ldc + bn * BN;
#pragma unroll
        for (int cc = 0; cc < BN / 32; ++cc) {
          if (cc + 1 < BN / 32) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
              cb[(cc + 1) & 1][j] = *reinterpret_cast<const float4 *>(c0row0 + (cc + 1) * 32 + 4 * j);
          }
          uint32_t v[32];
          tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * BN + cc * 32), v);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float4 c = cb[cc & 1][j];
            float4 o;
            o.x = fmaf(beta, c.x, alpha * __uint_as_float(v[4 * j]));
            o.y = fmaf(beta, c.y, alpha * __uint_as_float(v[4 * j + 1]));
            o.z = fmaf(beta, c.z, alpha * __uint_as_float(v[4 * j + 2]));
            o.w = fmaf(beta, c.w, alpha * __uint_as_float(v[4 * j + 3]));
            *reinterpret_cast<float4 *>(crow0 + cc * 32 + 4 * j) = o;
          }
        }
      } else {
#pragma unroll 1
      for (int cc = 0; cc < BN / 32; ++cc) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * BN + cc * 32), v);
        const int col0 = bn * BN + cc * 32;
        if (row < Mlim && col0 < Nlim) {
          float *crow = C + (int64_t)row * p.ldc + col0;
          const float *c0row = (C0 != nullptr && beta != 0.0f) ? C0 + (int64_t)row * p.ldc + col0 : nullptr;
          const int ncol = min(32, Nlim - col0);
          if (ncol == 32) {
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
              float4 o = make_float4(alpha * __uint_as_float(v[j]), alpha * __uint_as_float(v[j + 1]),
                                     alpha * __uint_as_float(v[j + 2]), alpha * __uint_as_float(v[j + 3]));
              if (c0row) {
                const float4 c = *reinterpret_cast<const float4 *>(c0row + j);
                o.x = fmaf(beta, c.x, o.x);
                o.y = fmaf(beta, c.y, o.y);
                o.z = fmaf(beta, c.z, o.z);
                o.w = fmaf(beta, c.w, o.w);
              }
              *reinterpret_cast<float4 *>(crow + j) = o;
            }
          } else {
            for (int j = 0; j < ncol; ++j) {
              float o = alpha * __uint_as_float(v[j]);
              if (c0row) o = fmaf(beta, c0row[j], o);
              crow[j] = o;
            }
          }
        }
      }
      }
      tc_fence_before();
      epilogue_sync();   // every epilogue thread has read the accumulator
      if (threadIdx.x == 64) mbar_arrive(acce_bar(b));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    if (lane == 0) drain(fin_bar, 0u);   // no MMA may still write the accumulators
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

std::once_flag g_attr_once;
bool g_attr_ok = false;

}  // namespace tcw

bool launch_tc_gemm_split(cudaStream_t s, const SplitGemmBatch &b, int M, int N, int K, int lda, int ldb, int ldc,
                          bool lower, int32_t *err, int max_ctas) {
  if (b.count <= 0) return true;
  if (K % tc::BK != 0 || !tc_gemm_available()) return false;
  std::call_once(tcw::g_attr_once, [] {
    tcw::g_attr_ok = cudaFuncSetAttribute(tcw::k_tc_gemm256, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          tcw::SMEM_BYTES) == cudaSuccess;
    if (!tcw::g_attr_ok) cudaGetLastError();
  });
  if (!tcw::g_attr_ok) return false;
  tcw::Params p;
  memset(&p, 0, sizeof(p));
  bool ragged = false;
  for (int q = 0; q < b.count; ++q) ragged |= b.e[q].rows > 0 || b.e[q].cols > 0;
  if (ragged && lower) return false;
  int tiles_sum = 0;
  for (int q = 0; q < b.count; ++q) {
    const SplitGemmEntry &e = b.e[q];
    const int Mq = e.rows > 0 ? e.rows : M, Nq = e.cols > 0 ? e.cols : N;
    if (!tc::encode_2d(&p.tm[q][0], e.Ah, Mq, K, lda, tc::BM) ||
        !tc::encode_2d(&p.tm[q][1], e.Al, Mq, K, lda, tc::BM) ||
        !tc::encode_2d(&p.tm[q][2], e.Bh, Nq, K, ldb, tcw::BN) || !tc::encode_2d(&p.tm[q][3], e.Bl, Nq, K, ldb, tcw::BN))
      return false;
    p.C[q] = e.C;
    p.C0[q] = e.C0;
    p.alpha[q] = e.alpha;
    p.beta[q] = e.beta;
    p.Mz[q] = Mq;
    p.Nz[q] = Nq;
    p.tm_z[q] = (Mq + tc::BM - 1) / tc::BM;
    p.tn_z[q] = (Nq + tcw::BN - 1) / tcw::BN;
    p.tstart[q] = tiles_sum;
    tiles_sum += p.tm_z[q] * p.tn_z[q];
  }
  p.tstart[b.count] = tiles_sum;
  p.ragged = ragged ? 1 : 0;
  p.count = b.count;
  p.M = M;
  p.N = N;
  p.K = K;
  p.ldc = ldc;
  p.lower = lower ? 1 : 0;
  p.tiles_m = (M + tc::BM - 1) / tc::BM;
  p.tiles_n = (N + tcw::BN - 1) / tcw::BN;
  double tiles = 0.0;
  if (!lower) {
    p.tiles_per_matrix = p.tiles_m * p.tiles_n;
  } else {
    int t = 0;
    for (int r = 0; r < p.tiles_m; ++r) t += std::min(p.tiles_n, (r * tc::BM + tc::BM - 1) / tcw::BN + 1);
    p.tiles_per_matrix = t;
  }
  tiles = (double)p.tiles_per_matrix;
  p.total_tiles = p.tiles_per_matrix * b.count;
  if (ragged) {
    p.total_tiles = tiles_sum;
    tiles = (double)tiles_sum / b.count;
  }
  p.err = err;
  p.wait_cycles = tc::wait_limit();
  p.skip_loads = tc::skip_loads();
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (max_ctas > 0) sms = std::min(sms, max_ctas);
  const int grid = std::min(p.total_tiles, sms);
  ++g_launch_count;
  Profiler::Rec rec{PROF_GEMM, nullptr, nullptr, 2.0 * tc::BM * tcw::BN * (double)K * tiles * b.count};
  if (g_prof) g_prof->begin(s, rec);
  tcw::k_tc_gemm256<<<grid, 192, tcw::SMEM_BYTES, s>>>(p);
  if (g_prof) g_prof->end(s, rec);
  return true;
}

}  // namespace qsel
