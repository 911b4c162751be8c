// Kronecker preconditioner passes on the tcgen05 tensor cores (mixed form).
//
// A pass computes, for every group g and every block of 128 sample columns,
//   Y_g[o, c] = sc_out(o) sum_k op(B)[o, k] sc_in(k) X_g[k, c],   o, k < dim,
// where X_g gathers the rows base(g) + k kstride of the n x ld sample block
// (see KronPass in kernels.cuh).  As an MMA, D[c, o] = sum_k A[c, k] B[o, k]
// with M = 128 sample columns, N = dim rounded up to 16 (<= 256) and K = dim
// in chunks of 32: both operands K-major, as kind::tf32 reads them.
//   warp 0      one thread loads the op(B) hi / lo chunks (tables split into
//               TF32 parts once per theta) by TMA into a 2-stage ring;
//   warps 2-5   gather the X_g chunk (coalesced along the samples), scale it,
//               split it into TF32 hi / lo and write it transposed into the
//               K-major 128B-swizzled layout, then run the epilogue
//               (tcgen05.ld, output scaling, stores coalesced along the samples);
//   warp 1      owns the accumulator (N TMEM columns); one thread issues the
//               3xTF32 MMAs (hi*hi + hi*lo + lo*hi, FP32 accumulation).
// Every wait is bounded (the same abort protocol as the GEMM kernels).
#include <mutex>

#include "qsel.h"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace qsel {
namespace ktc {
using namespace tc;

constexpr int MC = 128;                 // sample columns per work item (MMA M)
constexpr int STAGES = 2;
constexpr int ATILE = MC * BK * 4;      // 16 KiB: 128 rows x 128 bytes

struct Params {
  CUtensorMap tmB[2];                   // op(B) hi, lo: dim x dim row-major (row o, column k)
  const float *x;
  float *y;
  const float *scale;
  int dim, np, ld, m, mode, col_blocks, n_inner;
  int64_t kstride, outer_stride, inner_stride, items;
  int32_t *err;
  long long wait_cycles;
};

__host__ __device__ constexpr int btile_bytes(int np) { return np * BK * 4; }
__host__ __device__ constexpr int stage_bytes(int np) { return 2 * ATILE + 2 * btile_bytes(np); }
__host__ __device__ constexpr int smem_bytes(int np) { return STAGES * stage_bytes(np) + 256 + 1024; }
__host__ __device__ constexpr uint32_t tmem_cols(int np) {
  return np <= 32 ? 32u : np <= 64 ? 64u : np <= 128 ? 128u : 256u;
}

__device__ __forceinline__ void conv_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// kind::tf32 instruction descriptor for M = 128 and a runtime N (multiple of 16)
__device__ __forceinline__ uint32_t idesc_n(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(MC >> 4) << 24);
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

// Byte offset of element (row r, column k < 32) of a K-major tile with
// 128-byte rows and the 128B swizzle: the 16-byte unit k / 4 of row r is
// stored at unit (k / 4) ^ (r % 8).
__device__ __forceinline__ uint32_t sw128(int r, int k) {
  return (uint32_t)(r * 128 + ((((k >> 2) ^ (r & 7)) & 7) << 4) + ((k & 3) << 2));
}

__global__ void __launch_bounds__(192) k_kron_tc(const __grid_constant__ Params p) {
  extern __shared__ unsigned char smem_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int SB = stage_bytes(p.np), BT = btile_bytes(p.np);
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + STAGES * SB);
  // bars: [0, S) B landed, [S, 2S) A converted, [2S, 3S) stage empty, [3S] accumulator ready
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 3 * STAGES + 1);
  volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
  volatile int *cv_ok = abort + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto conv_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
  auto empty_bar = [&](int s) { return bar0 + 8u * (2 * STAGES + s); };
  const uint32_t accum_bar = bar0 + 8u * (3 * STAGES);
  const uint32_t ncols = tmem_cols(p.np);

  const int64_t item = blockIdx.x;
  const int cb = (int)(item % p.col_blocks);
  const int64_t g = item / p.col_blocks;
  const int g_inner = (int)(g % p.n_inner);
  const int64_t row0 = (g / p.n_inner) * p.outer_stride + (int64_t)g_inner * p.inner_stride;
  const int c0 = cb * MC;
  const int nk = (p.dim + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(conv_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    mbar_init(accum_bar, 1);
    *abort = 0;
    *cv_ok = 1;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int kc = 0; kc < nk; ++kc) {
        const int s = kc % STAGES;
        const uint32_t u = (uint32_t)(kc / STAGES);
        if (!mbar_wait(empty_bar(s), (u & 1) ^ 1, abort, p.err, p.wait_cycles)) break;
        uint8_t *st = base + s * SB;
        mbar_expect_tx(full_bar(s), 2 * BT);
        tma_load_2d(smem_u32(st + 2 * ATILE), &p.tmB[0], kc * BK, 0, full_bar(s));
        tma_load_2d(smem_u32(st + 2 * ATILE + BT), &p.tmB[1], kc * BK, 0, full_bar(s));
        issued = kc + 1;
      }
      if (*abort) {
        for (int kc = max(0, issued - STAGES); kc < issued; ++kc) {
          const long long t0 = clock64();
          uint32_t done = 0;
          while (!done && clock64() - t0 < kWaitCycles) {
            asm volatile(
                "{\n\t.reg .pred r;\n\tmbarrier.try_wait.parity.shared::cta.b64 r, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, r;\n\t}\n"
                : "=r"(done)
                : "r"(full_bar(kc % STAGES)), "r"((uint32_t)((kc / STAGES) & 1))
                : "memory");
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_n(p.np);
      for (int kc = 0; kc < nk; ++kc) {
        const int s = kc % STAGES;
        const uint32_t u = (uint32_t)(kc / STAGES);
        if (!mbar_wait(conv_bar(s), u & 1, abort, p.err, p.wait_cycles)) break;
        if (!mbar_wait(full_bar(s), u & 1, abort, p.err, p.wait_cycles)) break;
        tc_fence_after();
        const uint32_t st = smem_u32(base + s * SB);
        const uint32_t a_hi = st, a_lo = st + ATILE, b_hi = st + 2 * ATILE, b_lo = b_hi + BT;
#pragma unroll
        for (int j = 0; j < BK / 8; ++j) {
          const uint32_t off = j * 32;
          mma_tf32_n(tmem, smem_desc(a_hi + off), smem_desc(b_hi + off), idesc, (kc | j) != 0);
          mma_tf32_n(tmem, smem_desc(a_hi + off), smem_desc(b_lo + off), idesc, 1u);
          mma_tf32_n(tmem, smem_desc(a_lo + off), smem_desc(b_hi + off), idesc, 1u);
        }
        mma_commit(empty_bar(s));
      }
      mma_commit(accum_bar);
    }
  } else {
    // gather, scale, split and transpose X_g into A (row = sample column c,
    // column = k within the chunk); thread t takes column c = t for 32 rows k
    const int t = threadIdx.x - 64;
    const bool in_dh = p.mode == KRON_IN_DH;
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % STAGES;
      const uint32_t u = (uint32_t)(kc / STAGES);
      if (t == 0) *cv_ok = (mbar_wait(empty_bar(s), (u & 1) ^ 1, abort, p.err, p.wait_cycles) && !*abort) ? 1 : 0;
      conv_sync();
      if (!*cv_ok) break;
      uint8_t *st = base + s * SB;
      float *ahi = reinterpret_cast<float *>(st);
      float *alo = reinterpret_cast<float *>(st + ATILE);
#pragma unroll 4
      for (int kk = 0; kk < BK; ++kk) {
        const int k = kc * BK + kk;
        float v = 0.0f;
        if (k < p.dim) {
          v = p.x[(row0 + (int64_t)k * p.kstride) * p.ld + c0 + t];
          if (in_dh) v *= p.scale[k * p.m + g_inner];
        }
        const float h = tf32_rn(v);
        const uint32_t off = sw128(t, kk) >> 2;
        ahi[off] = h;
        alo[off] = tf32_rn(v - h);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      conv_sync();
      if (t == 0) mbar_arrive(conv_bar(s));
    }
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 = sample columns
    if (t == 0) *cv_ok = (mbar_wait(accum_bar, 0, abort, p.err, p.wait_cycles) && !*abort) ? 1 : 0;
    conv_sync();
    if (*cv_ok) {
      tc_fence_after();
      const int q = warp & 3;
      const int c = c0 + 32 * q + lane;
#pragma unroll 1
      for (int oc = 0; oc < p.np; oc += 32) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)oc, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int o = oc + j;
          if (o < p.dim) {
            float sc = 1.0f;
            if (p.mode == KRON_OUT_DH)
              sc = p.scale[o * p.m + g_inner];
            else if (p.mode == KRON_OUT_SPEC)   // group = spatial index, o = temporal index
              sc = p.scale[(int64_t)o * p.m * p.m + g_inner];
            p.y[(row0 + (int64_t)o * p.kstride) * p.ld + c] = __uint_as_float(v[j]) * sc;
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
      const long long t0 = clock64();
      uint32_t done = 0;
      while (!done && clock64() - t0 < kWaitCycles) {
        asm volatile(
            "{\n\t.reg .pred r;\n\tmbarrier.try_wait.parity.shared::cta.b64 r, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, r;\n\t}\n"
            : "=r"(done)
            : "r"(accum_bar), "r"(0u)
            : "memory");
      }
    }
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

std::mutex g_mu;
int g_attr_np = 0;   // largest np whose shared memory has been opted in

}  // namespace ktc

// dim rows of 16-byte multiples (the tables' tensor maps), at most 256 (one MMA N)
bool kron_tc_supported(int dim, int ld) { return dim >= 4 && dim <= 256 && dim % 4 == 0 && ld % ktc::MC == 0; }

bool launch_kron_pass_tc(cudaStream_t s, const KronPass &p, const float *Bop_hi, const float *Bop_lo, const float *x,
                         float *y, int32_t *err) {
  if (!kron_tc_supported(p.dim, p.ld) || !tc_gemm_available()) return false;
  const int np = (p.dim + 15) / 16 * 16;
  {
    std::lock_guard<std::mutex> lock(ktc::g_mu);
    if (np > ktc::g_attr_np) {
      if (cudaFuncSetAttribute(ktc::k_kron_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, ktc::smem_bytes(np)) !=
          cudaSuccess) {
        cudaGetLastError();
        return false;
      }
      ktc::g_attr_np = np;
    }
  }
  ktc::Params kp;
  memset(&kp, 0, sizeof(kp));
  if (!tc::encode_2d(&kp.tmB[0], Bop_hi, p.dim, p.dim, p.dim, np) ||
      !tc::encode_2d(&kp.tmB[1], Bop_lo, p.dim, p.dim, p.dim, np))
    return false;
  kp.x = x;
  kp.y = y;
  kp.scale = static_cast<const float *>(p.scale);
  kp.dim = p.dim;
  kp.np = np;
  kp.ld = p.ld;
  kp.m = p.m;
  kp.mode = p.mode;
  kp.col_blocks = p.ld / ktc::MC;
  kp.n_inner = p.n_inner;
  kp.kstride = p.kstride;
  kp.outer_stride = p.outer_stride;
  kp.inner_stride = p.inner_stride;
  kp.items = (int64_t)p.n_outer * p.n_inner * kp.col_blocks;
  kp.err = err;
  kp.wait_cycles = tc::wait_limit();
  ++g_launch_count;
  ktc::k_kron_tc<<<(unsigned)kp.items, 192, ktc::smem_bytes(np), s>>>(kp);
  return true;
}

}  // namespace qsel
