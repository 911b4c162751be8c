// Tensor-core GEMM for the mixed path (sm_100a/sm_103a tcgen05 + TMA).
//
//   C = alpha A B^T + beta C0,   A: M x K, B: N x K, C: M x N, all FP32 row-major
//
// Both operands are K-major ("TN"), which is what the Takahashi products of
// the mixed path need: Y^T = W^T Sigma_{t+1} (Sigma symmetric) and
// Sigma_t = D_t^-1 + Y^T W (B stored as W^T).
//
// One CTA computes a 128 x 128 tile of C:
//   warp 0      one thread issues the TMA loads of 128 x 32 FP32 tiles of A and
//               B (128-byte rows, 128B swizzle) into a 3-stage ring;
//   warps 2-5   split every loaded tile into TF32 hi = rn(x) and lo =
//               rn(x - hi) parts (rn = round to nearest TF32, so hi + lo
//               holds x to about 2^-23) in shared memory, then run the
//               epilogue (tcgen05.ld of the accumulator, alpha/beta, store);
//   warp 1      owns the 128-column TMEM accumulator; one thread issues
//               tcgen05.mma.kind::tf32 (M=128, N=128, K=8) for hi*hi, hi*lo and
//               lo*hi ("3xTF32", FP32-level accuracy with FP32 accumulation) or
//               for the raw values only (1 pass).
// Every wait is bounded: after ~2 s (or the limit set by the test hook
// qsel_debug_tc_wait) the CTA raises bit 1 of *err, stops issuing work, waits
// (bounded) for what it already issued, frees TMEM and returns.
#include <cuda.h>

#include <atomic>
#include <mutex>

#include "qsel.h"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace qsel {
namespace tc {

constexpr int TILE_A = BM * BK * 4;              // 16 KiB A tile
constexpr int BAR_BYTES = 256;
// Configurations: <3 stages, BN = 128> (one CTA per SM) for K > 64, and
// <2 stages, BN = 64> for K = 64 (the last, one-tile panel of the sweep and
// the one-pivot sweep): the two K-blocks fit without reusing a stage and two
// CTAs share an SM, so one CTA's epilogue overlaps the other's loads and MMAs.
// <2 stages, BN = 32> (compact) for the sweep's look-ahead products, which
// run beside the persistent panel update and must fit on its SMs.
template <int BN>
__host__ __device__ constexpr int tile_b() {
  return BN * BK * 4;
}
template <int STAGES, int BN>
__host__ __device__ constexpr int stage_bytes() {
  return 2 * (TILE_A + tile_b<BN>());            // A, B, A_lo, B_lo
}
template <int STAGES, int BN>
__host__ __device__ constexpr int smem_bytes() {
  return STAGES * stage_bytes<STAGES, BN>() + BAR_BYTES + 1024;
}
struct Params {
  CUtensorMap tmA[kMaxBatch];
  CUtensorMap tmB[kMaxBatch];
  float *C[kMaxBatch];
  const float *C0[kMaxBatch];
  float alpha[kMaxBatch], beta[kMaxBatch];
  int M, N, K, ldc, lower, passes;
  int32_t *err;
  long long wait_cycles;   // limit of every wait on a stage or the accumulator
  int skip_loads;          // test hook: the producer issues no TMA load
};

__device__ __forceinline__ void named_sync_converters() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

template <int STAGES, int BN>
__global__ void __launch_bounds__(192) k_tc_gemm(const __grid_constant__ Params p) {
  constexpr int TILE_B = tile_b<BN>();
  constexpr int STAGE_BYTES = stage_bytes<STAGES, BN>();
  constexpr uint32_t kTmemCols = BN;
  extern __shared__ unsigned char smem_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + STAGES * STAGE_BYTES);
  // bars[0..S): full (TMA landed), [S..2S): converted, [2S..3S): empty, [3S]: accumulator ready
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 3 * STAGES + 1);
  volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
  volatile int *conv_ok = abort + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bn = blockIdx.x, bm = blockIdx.y, z = blockIdx.z;
  if (p.lower && bn * BN >= (bm + 1) * BM) return;   // tile entirely above the diagonal
  const int nk = p.K / BK;
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto conv_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
  auto empty_bar = [&](int s) { return bar0 + 8u * (2 * STAGES + s); };
  const uint32_t accum_bar = bar0 + 8u * (3 * STAGES);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(conv_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    mbar_init(accum_bar, 1);
    *abort = 0;
    *conv_ok = 1;
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
      const CUtensorMap *tma = &p.tmA[z];
      const CUtensorMap *tmb = &p.tmB[z];
      int issued = 0;
      for (int kb = 0; kb < nk && !p.skip_loads; ++kb) {
        const int s = kb % STAGES, u = kb / STAGES;
        if (!mbar_wait(empty_bar(s), (u & 1) ^ 1, abort, p.err, p.wait_cycles)) break;
        uint8_t *st = base + s * STAGE_BYTES;
        mbar_expect_tx(full_bar(s), TILE_A + TILE_B);
        tma_load_2d(smem_u32(st), tma, kb * BK, bm * BM, full_bar(s));
        tma_load_2d(smem_u32(st + TILE_A), tmb, kb * BK, bn * BN, full_bar(s));
        issued = kb + 1;
      }
      if (*abort) {
        // let the loads already issued land before the CTA's shared memory goes away
        for (int kb = max(0, issued - STAGES); kb < issued; ++kb) {
          const long long t0 = clock64();
          uint32_t done = 0;
          while (!done && clock64() - t0 < kWaitCycles) {
            asm volatile(
                "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, q;\n\t}\n"
                : "=r"(done)
                : "r"(full_bar(kb % STAGES)), "r"((uint32_t)((kb / STAGES) & 1))
                : "memory");
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES, u = kb / STAGES;
        if (!mbar_wait(conv_bar(s), u & 1, abort, p.err, p.wait_cycles)) break;
        tc_fence_after();
        const uint32_t st = smem_u32(base + s * STAGE_BYTES);
        const uint32_t a_hi = st, b_hi = st + TILE_A, a_lo = st + TILE_A + TILE_B, b_lo = a_lo + TILE_A;
#pragma unroll
        for (int j = 0; j < BK / 8; ++j) {
          const uint32_t off = j * 32;
          mma_tf32<BN>(tmem, smem_desc(a_hi + off), smem_desc(b_hi + off), (kb | j) != 0);
          if (p.passes == 3) {
            mma_tf32<BN>(tmem, smem_desc(a_hi + off), smem_desc(b_lo + off), 1u);
            mma_tf32<BN>(tmem, smem_desc(a_lo + off), smem_desc(b_hi + off), 1u);
          }
        }
        mma_commit(empty_bar(s));
      }
      // signals the epilogue when every MMA issued so far has completed
      mma_commit(accum_bar);
    }
  } else {
    // converters (warps 2-5): split the raw tiles into TF32 hi / lo parts
    const int ct = threadIdx.x - 64;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES, u = kb / STAGES;
      if (ct == 0) *conv_ok = (mbar_wait(full_bar(s), u & 1, abort, p.err, p.wait_cycles) && !*abort) ? 1 : 0;
      named_sync_converters();
      if (!*conv_ok) break;
      if (p.passes == 3) {
        float4 *raw = reinterpret_cast<float4 *>(base + s * STAGE_BYTES);
        float4 *lo = reinterpret_cast<float4 *>(base + s * STAGE_BYTES + TILE_A + TILE_B);
        // A then B (16-byte chunks); lo mirrors raw at +(A + B)
        for (int i = ct; i < (TILE_A + TILE_B) / 16; i += 128) {
          float4 v = raw[i];
          float4 h;
          h.x = tf32_rn(v.x);
          h.y = tf32_rn(v.y);
          h.z = tf32_rn(v.z);
          h.w = tf32_rn(v.w);
          raw[i] = h;
          lo[i] = make_float4(tf32_rn(v.x - h.x), tf32_rn(v.y - h.y), tf32_rn(v.z - h.z), tf32_rn(v.w - h.w));
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      named_sync_converters();
      if (ct == 0) mbar_arrive(conv_bar(s));
    }
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 = rows of the tile
    if (ct == 0) *conv_ok = (mbar_wait(accum_bar, 0, abort, p.err, p.wait_cycles) && !*abort) ? 1 : 0;
    named_sync_converters();
    if (*conv_ok) {  // uniform across the four warps: tcgen05.ld is warp-collective
      tc_fence_after();
      const int q = warp & 3;
      const int row = bm * BM + 32 * q + lane;
      float *C = p.C[z];
      const float *C0 = p.C0[z];
      const float alpha = p.alpha[z], beta = p.beta[z];
#pragma unroll 1
      for (int cc = 0; cc < BN / 32; ++cc) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(cc * 32), v);
        const int col0 = bn * BN + cc * 32;
        if (row < p.M && col0 < p.N) {
          float *crow = C + (int64_t)row * p.ldc + col0;
          const float *c0row = C0 ? C0 + (int64_t)row * p.ldc + col0 : nullptr;
          const int ncol = min(32, p.N - col0);
          if (ncol == 32) {
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
              float4 o = make_float4(alpha * __uint_as_float(v[j]), alpha * __uint_as_float(v[j + 1]),
                                     alpha * __uint_as_float(v[j + 2]), alpha * __uint_as_float(v[j + 3]));
              if (c0row != nullptr && beta != 0.0f) {
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
              if (c0row != nullptr && beta != 0.0f) o = fmaf(beta, c0row[j], o);
              crow[j] = o;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    if (*abort && lane == 0) {
      // wait (bounded) for MMAs still in flight before the accumulator is freed
      const long long t0 = clock64();
      uint32_t done = 0;
      while (!done && clock64() - t0 < kWaitCycles) {
        asm volatile(
            "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, q;\n\t}\n"
            : "=r"(done)
            : "r"(accum_bar), "r"(0u)
            : "memory");
      }
    }
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::mutex g_mu;
EncodeFn g_encode = nullptr;
int g_state = 0;  // 0 unknown, 1 available, -1 unavailable
// test hook (qsel_debug_tc_wait): skip the loads and / or shorten the waits
std::atomic<int> g_skip_loads{0};
std::atomic<long long> g_wait_cycles{0};

long long wait_limit() {
  const long long wc = g_wait_cycles.load();
  return wc > 0 ? wc : kWaitCycles;
}

int skip_loads() { return g_skip_loads.load(); }

bool encode_2d(CUtensorMap *tm, const float *ptr, int rows, int cols, int ld, int box_rows) {
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(ptr), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool encode_4d(CUtensorMap *tm, const float *ptr, const uint64_t dims[4], const uint64_t strides[3],
               const uint32_t box[4]) {
  cuuint64_t d[4] = {dims[0], dims[1], dims[2], dims[3]};
  cuuint64_t st[3] = {strides[0], strides[1], strides[2]};
  cuuint32_t bx[4] = {(cuuint32_t)BK, box[1], box[2], box[3]};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(ptr), d, st, bx, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool encode_4d_plain(CUtensorMap *tm, const float *ptr, const uint64_t dims[4], const uint64_t strides[3],
                     const uint32_t box[4]) {
  cuuint64_t d[4] = {dims[0], dims[1], dims[2], dims[3]};
  cuuint64_t st[3] = {strides[0], strides[1], strides[2]};
  cuuint32_t bx[4] = {box[0], box[1], box[2], box[3]};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(ptr), d, st, bx, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace tc

// True when the current device runs tcgen05 (compute capability 10.x) and the
// driver provides cuTensorMapEncodeTiled.
bool tc_gemm_available() {
  std::lock_guard<std::mutex> lock(tc::g_mu);
  if (tc::g_state != 0) return tc::g_state > 0;
  int dev = 0, major = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess || major != 10) {
    tc::g_state = -1;
    return false;
  }
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || fn == nullptr) {
    cudaGetLastError();
    tc::g_state = -1;
    return false;
  }
  tc::g_encode = reinterpret_cast<tc::EncodeFn>(fn);
  if (cudaFuncSetAttribute(tc::k_tc_gemm<3, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           tc::smem_bytes<3, 128>()) != cudaSuccess ||
      cudaFuncSetAttribute(tc::k_tc_gemm<2, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           tc::smem_bytes<2, 64>()) != cudaSuccess ||
      cudaFuncSetAttribute(tc::k_tc_gemm<2, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           tc::smem_bytes<2, 32>()) != cudaSuccess) {
    cudaGetLastError();
    tc::g_state = -1;
    return false;
  }
  tc::g_state = 1;
  return true;
}

// C = alpha A B^T + beta C0 with A (M x K, lda) and B (N x K, ldb) row-major;
// K a multiple of 32, lda/ldb/ldc multiples of 4.  Returns false when a tensor
// map cannot be encoded (nothing is launched then).
bool launch_tc_gemm(cudaStream_t s, const GemmBatch<float> &b, int M, int N, int K, int lda, int ldb, int ldc,
                    bool lower, int passes, int32_t *err, bool compact) {
  // K = 64 (the sweep updates): two stages, 128 x 64 tiles, two CTAs per SM
  const bool narrow = K <= 64 && !compact;
  const int bn_w = compact ? 32 : narrow ? 64 : 128;
  if (b.count <= 0) return true;
  if (!tc_gemm_available()) return false;
  tc::Params p;
  memset(&p, 0, sizeof(p));
  for (int q = 0; q < b.count; ++q) {
    if (!tc::encode_2d(&p.tmA[q], b.e[q].A, M, K, lda, tc::BM) ||
        !tc::encode_2d(&p.tmB[q], b.e[q].B, N, K, ldb, bn_w))
      return false;
    p.C[q] = b.e[q].C;
    p.C0[q] = b.e[q].C0;
    p.alpha[q] = (float)b.e[q].alpha;
    p.beta[q] = (float)b.e[q].beta;
  }
  p.M = M;
  p.N = N;
  p.K = K;
  p.ldc = ldc;
  p.lower = lower ? 1 : 0;
  p.passes = passes;
  p.err = err;
  p.wait_cycles = tc::wait_limit();
  p.skip_loads = tc::skip_loads();
  ++g_launch_count;
  Profiler::Rec rec{PROF_GEMM, nullptr, nullptr, 0.0};
  const int gm = (M + tc::BM - 1) / tc::BM, gn = (N + bn_w - 1) / bn_w;
  if (g_prof) {
    double tiles = 0.0;
    for (int bm = 0; bm < gm; ++bm)
      for (int bn = 0; bn < gn; ++bn)
        if (!lower || bn * bn_w < (bm + 1) * tc::BM) tiles += 1.0;
    rec.work = 2.0 * tc::BM * bn_w * (double)K * tiles * b.count;
    g_prof->begin(s, rec);
  }
  if (compact)
    tc::k_tc_gemm<2, 32><<<dim3(gn, gm, b.count), 192, tc::smem_bytes<2, 32>(), s>>>(p);
  else if (narrow)
    tc::k_tc_gemm<2, 64><<<dim3(gn, gm, b.count), 192, tc::smem_bytes<2, 64>(), s>>>(p);
  else
    tc::k_tc_gemm<3, 128><<<dim3(gn, gm, b.count), 192, tc::smem_bytes<3, 128>(), s>>>(p);
  if (g_prof) g_prof->end(s, rec);
  return true;
}

}  // namespace qsel

extern "C" qsel_status qsel_debug_tc_wait(int32_t skip_loads, int64_t wait_cycles) {
  if (wait_cycles < 0) return QSEL_EINVAL;
  qsel::tc::g_skip_loads.store(skip_loads ? 1 : 0);
  qsel::tc::g_wait_cycles.store((long long)wait_cycles);
  return QSEL_OK;
}
