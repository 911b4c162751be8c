// Persistent tensor-core kernel of the sweep's panel updates (mixed form):
//
//   C = alpha U V^T + beta C   on the lower 128 x 128 tiles of every matrix of
//                              a batch (C n x n, U and V n x K row-major),
//
// with U and V already split into TF32 parts (hi = rn(x), lo = rn(x - hi)) by
// k_split_tf32, once per panel for all tiles, so that every tile only loads
// and multiplies: the three products hi*hi + hi*lo + lo*hi ("3xTF32") run
// with FP32 accumulation in tensor memory.
//
// One CTA per SM walks a static list of (matrix, tile row, tile column)
// lower tiles:
//   warp 0      one thread issues the TMA loads of the four 128 x 32 operand
//               tiles of every K-block into a 2-stage ring (129 KB of shared
//               memory: the sweep's pivot and panel kernels, and its compact
//               look-ahead GEMM, fit on the same SM and run beside it);
//   warp 1      owns 256 TMEM columns = two 128-column accumulators; one
//               thread issues tcgen05.mma.kind::tf32 (M = N = 128, K = 8) for
//               tile i into accumulator i % 2 while the epilogue drains the
//               other one;
//   warps 2-5   epilogue: tcgen05.ld of the accumulator, alpha / beta, store.
// Every wait is bounded: after the limit the CTA raises bit 1 of *err, stops
// issuing work, waits (bounded) for its loads and MMAs in flight, frees its
// tensor memory and returns.
#include <mutex>

#include "qsel.h"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace qsel {
namespace tcu {
using namespace tc;

constexpr int BN = 128;
constexpr int TILE = BM * BK * 4;            // 16 KiB: 128 rows x 32 floats
constexpr int STAGE_BYTES = 4 * TILE;        // U_hi, U_lo, V_hi, V_lo
// Two stages (129 KB) leave room on the SM for the sweep's pivot and panel
// CTAs beside the update; three (193 KB) do not, so those run on the SMs
// that a capped update grid leaves free.
template <int STAGES>
constexpr int smem_bytes() { return STAGES * STAGE_BYTES + 256 + 1024; }
constexpr uint32_t kTmemCols = 2 * BN;

struct Params {
  CUtensorMap tm[kMaxBatch][4];   // U_hi, U_lo, V_hi, V_lo
  float *C[kMaxBatch];
  int n, K, ldc;
  int tiles_per_matrix, total_tiles;
  float alpha, beta;
  int32_t *err;
  long long wait_cycles;
  int skip_loads;
};

// Lower tile r of a matrix (row-major over the lower triangle): row bm,
// column bn <= bm.
__device__ __forceinline__ void lower_tile(int r, int &bm, int &bn) {
  int m = (int)((sqrtf(8.0f * (float)r + 1.0f) - 1.0f) * 0.5f);
  while ((m + 1) * (m + 2) / 2 <= r) ++m;
  while (m * (m + 1) / 2 > r) --m;
  bm = m;
  bn = r - m * (m + 1) / 2;
}

__device__ __forceinline__ void epilogue_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

template <int STAGES>
__global__ void __launch_bounds__(192, 1) k_tc_update(const __grid_constant__ Params p) {
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
        const int z = L / p.tiles_per_matrix;
        int bm, bn;
        lower_tile(L - z * p.tiles_per_matrix, bm, bn);
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
          tma_load_2d(smem_u32(st + TILE), &p.tm[z][1], kb * BK, bm * BM, full_bar(s));
          tma_load_2d(smem_u32(st + 2 * TILE), &p.tm[z][2], kb * BK, bn * BN, full_bar(s));
          tma_load_2d(smem_u32(st + 3 * TILE), &p.tm[z][3], kb * BK, bn * BN, full_bar(s));
          ++g;
        }
      }
      if (*abort) {
        // let the loads already issued land before the CTA's shared memory goes away
        for (long long q = (g > STAGES ? g - STAGES : 0); q < g; ++q) {
          const long long t0 = clock64();
          uint32_t done = 0;
          while (!done && clock64() - t0 < kWaitCycles) {
            asm volatile(
                "{\n\t.reg .pred r;\n\tmbarrier.try_wait.parity.shared::cta.b64 r, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, r;\n\t}\n"
                : "=r"(done)
                : "r"(full_bar((int)(q % STAGES))), "r"((uint32_t)((q / STAGES) & 1))
                : "memory");
          }
        }
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
          const uint32_t uh = st, ul = st + TILE, vh = st + 2 * TILE, vl = st + 3 * TILE;
#pragma unroll
          for (int j = 0; j < BK / 8; ++j) {
            const uint32_t off = j * 32;
            mma_tf32<BN>(d, smem_desc(uh + off), smem_desc(vh + off), (kb | j) != 0);
            mma_tf32<BN>(d, smem_desc(uh + off), smem_desc(vl + off), 1u);
            mma_tf32<BN>(d, smem_desc(ul + off), smem_desc(vh + off), 1u);
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
      const int z = L / p.tiles_per_matrix;
      int bm, bn;
      lower_tile(L - z * p.tiles_per_matrix, bm, bn);
      const int row = bm * BM + 32 * q + lane;
      float *C = p.C[z];
      // a whole row segment in range: C is read a chunk ahead, the first chunk
      // while the tile's MMAs still run (C does not depend on them)
      const bool full = row < p.n && (bn + 1) * BN <= p.n && p.beta != 0.0f;
      float *crow0 = C + (int64_t)row * p.ldc + bn * BN;
      float4 cb[2][8];
      if (full) {
#pragma unroll
        for (int j = 0; j < 8; ++j) cb[0][j] = *reinterpret_cast<const float4 *>(crow0 + 4 * j);
      }
      if (threadIdx.x == 64) *ep_ok = (mbar_wait(accf_bar(b), ub & 1, abort, p.err, p.wait_cycles) && !*abort) ? 1 : 0;
      epilogue_sync();
      if (!*ep_ok) break;   // uniform across the four warps: tcgen05.ld is warp-collective
      tc_fence_after();
      if (full) {
#pragma unroll
        for (int cc = 0; cc < BN / 32; ++cc) {
          if (cc + 1 < BN / 32) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
              cb[(cc + 1) & 1][j] = *reinterpret_cast<const float4 *>(crow0 + (cc + 1) * 32 + 4 * j);
          }
          uint32_t v[32];
          tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * BN + cc * 32), v);
          float *crow = crow0 + cc * 32;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float4 c = cb[cc & 1][j];
            float4 o;
            o.x = fmaf(p.beta, c.x, p.alpha * __uint_as_float(v[4 * j]));
            o.y = fmaf(p.beta, c.y, p.alpha * __uint_as_float(v[4 * j + 1]));
            o.z = fmaf(p.beta, c.z, p.alpha * __uint_as_float(v[4 * j + 2]));
            o.w = fmaf(p.beta, c.w, p.alpha * __uint_as_float(v[4 * j + 3]));
            *reinterpret_cast<float4 *>(crow + 4 * j) = o;
          }
        }
      } else {
#pragma unroll 1
      for (int cc = 0; cc < BN / 32; ++cc) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * BN + cc * 32), v);
        const int col0 = bn * BN + cc * 32;
        if (row < p.n && col0 < p.n) {
          float *crow = C + (int64_t)row * p.ldc + col0;
          const int ncol = min(32, p.n - col0);
          if (ncol == 32) {
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
              const float4 c = *reinterpret_cast<const float4 *>(crow + j);
              float4 o;
              o.x = fmaf(p.beta, c.x, p.alpha * __uint_as_float(v[j]));
              o.y = fmaf(p.beta, c.y, p.alpha * __uint_as_float(v[j + 1]));
              o.z = fmaf(p.beta, c.z, p.alpha * __uint_as_float(v[j + 2]));
              o.w = fmaf(p.beta, c.w, p.alpha * __uint_as_float(v[j + 3]));
              *reinterpret_cast<float4 *>(crow + j) = o;
            }
          } else {
            for (int j = 0; j < ncol; ++j) crow[j] = fmaf(p.beta, crow[j], p.alpha * __uint_as_float(v[j]));
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
    if (lane == 0) {
      // no MMA may still write the accumulators when they are freed
      const long long t0 = clock64();
      uint32_t done = 0;
      while (!done && clock64() - t0 < kWaitCycles) {
        asm volatile(
            "{\n\t.reg .pred r;\n\tmbarrier.try_wait.parity.shared::cta.b64 r, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, r;\n\t}\n"
            : "=r"(done)
            : "r"(fin_bar), "r"(0u)
            : "memory");
      }
    }
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// hi = rn_tf32(x), lo = rn_tf32(x - hi) for `count` floats (16-byte vectors,
// then the last count % 4 one by one).
__global__ void __launch_bounds__(256) k_split_tf32(const float4 *__restrict__ src, float4 *__restrict__ hi,
                                                    float4 *__restrict__ lo, int64_t count4, int tail) {
  if (blockIdx.x == 0 && (int)threadIdx.x < tail) {
    const int64_t i = 4 * count4 + threadIdx.x;
    const float v = reinterpret_cast<const float *>(src)[i];
    const float h = tf32_rn(v);
    reinterpret_cast<float *>(hi)[i] = h;
    reinterpret_cast<float *>(lo)[i] = tf32_rn(v - h);
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count4; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = src[i];
    float4 h, l;
    h.x = tf32_rn(v.x);
    h.y = tf32_rn(v.y);
    h.z = tf32_rn(v.z);
    h.w = tf32_rn(v.w);
    l.x = tf32_rn(v.x - h.x);
    l.y = tf32_rn(v.y - h.y);
    l.z = tf32_rn(v.z - h.z);
    l.w = tf32_rn(v.w - h.w);
    hi[i] = h;
    lo[i] = l;
  }
}

// The same split for several arrays of count4 16-byte vectors each (one per
// grid row): the sweep's U and W of every matrix of a batch in one launch.
__global__ void __launch_bounds__(256) k_split_tf32_jobs(SplitJobs jobs, int64_t count4_all) {
  const SplitJob jb = jobs.j[blockIdx.y];
  const int64_t count4 = jb.count > 0 ? jb.count / 4 : count4_all;
  const float4 *__restrict__ src = reinterpret_cast<const float4 *>(jb.src);
  float4 *__restrict__ hi = reinterpret_cast<float4 *>(jb.hi);
  float4 *__restrict__ lo = reinterpret_cast<float4 *>(jb.lo);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count4; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = src[i];
    float4 h, l;
    h.x = tf32_rn(v.x);
    h.y = tf32_rn(v.y);
    h.z = tf32_rn(v.z);
    h.w = tf32_rn(v.w);
    l.x = tf32_rn(v.x - h.x);
    l.y = tf32_rn(v.y - h.y);
    l.z = tf32_rn(v.z - h.z);
    l.w = tf32_rn(v.w - h.w);
    hi[i] = h;
    lo[i] = l;
  }
}

std::once_flag g_attr_once;
bool g_attr_ok = false;

}  // namespace tcu

void launch_split_tf32(cudaStream_t s, const float *src, float *hi, float *lo, int64_t count) {
  ++g_launch_count;
  const int64_t c4 = count / 4;
  const int grid = (int)std::min<int64_t>((c4 + 255) / 256, 152 * 4);
  tcu::k_split_tf32<<<grid < 1 ? 1 : grid, 256, 0, s>>>(reinterpret_cast<const float4 *>(src),
                                                         reinterpret_cast<float4 *>(hi),
                                                         reinterpret_cast<float4 *>(lo), c4,
                                                         (int)(count - 4 * c4));
}

void launch_split_tf32_jobs(cudaStream_t s, const SplitJobs &jobs, int64_t count) {
  if (jobs.count <= 0) return;
  ++g_launch_count;
  const int64_t c4 = count / 4;
  const int gx = (int)std::max<int64_t>(1, std::min<int64_t>((c4 + 255) / 256, (152 * 4 + jobs.count - 1) / jobs.count));
  tcu::k_split_tf32_jobs<<<dim3(gx, jobs.count), 256, 0, s>>>(jobs, c4);
}

bool launch_tc_update(cudaStream_t s, const UpdateBatch &b, int n, int K, int ldp, float alpha, float beta,
                      int32_t *err, int max_ctas) {
  if (b.count <= 0) return true;
  if (!tc_gemm_available()) return false;
  std::call_once(tcu::g_attr_once, [] {
    tcu::g_attr_ok = cudaFuncSetAttribute(tcu::k_tc_update<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          tcu::smem_bytes<2>()) == cudaSuccess &&
                     cudaFuncSetAttribute(tcu::k_tc_update<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          tcu::smem_bytes<3>()) == cudaSuccess;
    if (!tcu::g_attr_ok) cudaGetLastError();
  });
  if (!tcu::g_attr_ok) return false;
  tcu::Params p;
  memset(&p, 0, sizeof(p));
  for (int q = 0; q < b.count; ++q) {
    const UpdateEntry &e = b.e[q];
    const float *ops[4] = {e.Uh, e.Ul, e.Vh, e.Vl};
    for (int o = 0; o < 4; ++o)
      if (!tc::encode_2d(&p.tm[q][o], ops[o], n, K, ldp, tc::BM)) return false;
    p.C[q] = e.C;
  }
  const int gm = (n + tc::BM - 1) / tc::BM;
  p.n = n;
  p.K = K;
  p.ldc = n;
  p.tiles_per_matrix = gm * (gm + 1) / 2;
  p.total_tiles = p.tiles_per_matrix * b.count;
  p.alpha = alpha;
  p.beta = beta;
  p.err = err;
  p.wait_cycles = tc::wait_limit();
  p.skip_loads = tc::skip_loads();
  int sms = 152;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (max_ctas > 0) sms = std::min(sms, max_ctas);
  const int grid = std::min(p.total_tiles, sms);
  ++g_launch_count;
  if (update_stages() == 3)
    tcu::k_tc_update<3><<<grid, 192, tcu::smem_bytes<3>(), s>>>(p);
  else
    tcu::k_tc_update<2><<<grid, 192, tcu::smem_bytes<2>(), s>>>(p);
  return true;
}

}  // namespace qsel
