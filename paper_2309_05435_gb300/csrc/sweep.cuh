// Scalar symmetric sweep (Gauss-Jordan on an SPD matrix without pivoting),
// in shared memory, by all threads of the block.
#pragma once

namespace qsel {

// After pivoting on every index 0..b-1, S (b x b, row stride ld_s) holds
// -S^-1.  Each pivot p: S_pp <- -1/d, row and column p scaled by 1/d, the
// rest updated by S_ij - S_ip S_pj / d, all from the values before the pivot.
// A non-positive pivot sets bit 0 of *err_flag.  At most 16 entries per thread.
__device__ inline void sym_sweep_inverse_smem(double *S, int ld_s, int b, int32_t *err_flag) {
  for (int p = 0; p < b; ++p) {
    const double d = S[p * ld_s + p];
    if (!(d > 0.0) && threadIdx.x == 0 && err_flag) atomicOr(err_flag, 1);
    const double inv = (d > 0.0) ? 1.0 / d : 0.0;
    double nv[16];
    int cnt = 0;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
      const int i = e / b, j = e - (e / b) * b;
      double v;
      if (i == p && j == p)
        v = -inv;
      else if (i == p)
        v = S[p * ld_s + j] * inv;
      else if (j == p)
        v = S[i * ld_s + p] * inv;
      else
        v = S[i * ld_s + j] - S[i * ld_s + p] * S[p * ld_s + j] * inv;
      nv[cnt++] = v;
    }
    __syncthreads();
    cnt = 0;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
      const int i = e / b, j = e - (e / b) * b;
      S[i * ld_s + j] = nv[cnt++];
    }
    __syncthreads();
  }
}

// 64 x 64 version of the sweep above for an SPD tile held in its lower
// triangle: each pivot snapshots column p (c_i = S_ip) and w_j = c_j / d, then
// every lower entry is updated with one FMA, S_ij - c_i w_j, by the thread
// that owns it (2080 entries, ceil(2080 / NT) per thread; blockDim.x == NT).
// Only the 64 column threads form 1 / d; thread 0 leaves it in col[64] for the
// owner of the diagonal entry (col holds 65 doubles).  After the 64 pivots the
// lower triangle holds that of -S^-1.
template <int NT>
__device__ inline void sym_sweep_inverse64_lower(double *S, int ld_s, double *col, double *wv, int32_t *err_flag) {
  constexpr int EPT = (2080 + NT - 1) / NT;
  int ei[EPT], ej[EPT];
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int e = (int)threadIdx.x + q * NT;
    ei[q] = -1;
    ej[q] = 0;
    if (e < 2080) {
      // float estimate of the row, made exact by the two corrections
      int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
      while ((i + 1) * (i + 2) / 2 <= e) ++i;
      while (i * (i + 1) / 2 > e) --i;
      ei[q] = i;
      ej[q] = e - i * (i + 1) / 2;
    }
  }
  for (int p = 0; p < 64; ++p) {
    if (threadIdx.x < 64) {
      const double d = S[p * ld_s + p];
      const double inv = (d > 0.0) ? 1.0 / d : 0.0;
      const int i = threadIdx.x;
      const double c = (i >= p) ? S[i * ld_s + p] : S[p * ld_s + i];
      col[i] = c;
      wv[i] = c * inv;
      if (i == 0) {
        col[64] = inv;
        if (!(d > 0.0) && err_flag) atomicOr(err_flag, 1);
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      if (ei[q] >= 0) {
        const int i = ei[q], j = ej[q];
        double v;
        if (i == p && j == p)
          v = -col[64];
        else if (i == p)
          v = wv[j];
        else if (j == p)
          v = wv[i];
        else
          v = fma(-col[i], wv[j], S[i * ld_s + j]);
        S[i * ld_s + j] = v;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Double-float arithmetic (Dekker 1971, "A floating-point technique for
// extending the available precision"; Knuth, TAOCP vol. 2, 4.2.2): a value is
// hi + lo with |lo| <= ulp(hi) / 2, about 48 significant bits, on the FP32
// pipe.  The _rn intrinsics keep the compiler from contracting or
// reassociating the error terms.
// ---------------------------------------------------------------------------
struct dfloat {
  float hi, lo;
};
// s + e = a + b exactly (Knuth's two-sum)
__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// the same for |a| >= |b| (Dekker's fast two-sum)
__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);  // exact error of the product
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ dfloat df_sub(dfloat a, dfloat b) {
  dfloat s = df_two_sum(a.hi, -b.hi);
  s.lo = __fadd_rn(s.lo, __fsub_rn(a.lo, b.lo));
  return df_fast_two_sum(s.hi, s.lo);
}
// 1 / d: the float reciprocal and one Newton step r + r (1 - d r), whose
// residual is formed exactly enough with two fused multiply-adds
__device__ __forceinline__ dfloat df_recip(dfloat d) {
  const float r = 1.0f / d.hi;
  float t = __fmaf_rn(-d.hi, r, 1.0f);
  t = __fmaf_rn(-d.lo, r, t);
  return df_fast_two_sum(r, __fmul_rn(r, t));
}

// sym_sweep_inverse64_lower in double-float: S (64 x 64 lower triangle, row
// stride ld_s) ends as the lower triangle of -S^-1; col holds 65 entries
// (col[64] = 1 / d), wv 64.  blockDim.x == NT.
template <int NT>
__device__ inline void sym_sweep_inverse64_lower_df(dfloat *S, int ld_s, dfloat *col, dfloat *wv,
                                                    int32_t *err_flag) {
  constexpr int EPT = (2080 + NT - 1) / NT;
  int ei[EPT], ej[EPT];
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int e = (int)threadIdx.x + q * NT;
    ei[q] = -1;
    ej[q] = 0;
    if (e < 2080) {
      int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
      while ((i + 1) * (i + 2) / 2 <= e) ++i;
      while (i * (i + 1) / 2 > e) --i;
      ei[q] = i;
      ej[q] = e - i * (i + 1) / 2;
    }
  }
  for (int p = 0; p < 64; ++p) {
    if (threadIdx.x < 64) {
      const dfloat d = S[p * ld_s + p];
      const bool pos = d.hi > 0.0f;
      const dfloat inv = pos ? df_recip(d) : dfloat{0.0f, 0.0f};
      const int i = threadIdx.x;
      const dfloat c = (i >= p) ? S[i * ld_s + p] : S[p * ld_s + i];
      col[i] = c;
      wv[i] = df_mul(c, inv);
      if (i == 0) {
        col[64] = inv;
        if (!pos && err_flag) atomicOr(err_flag, 1);
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      if (ei[q] >= 0) {
        const int i = ei[q], j = ej[q];
        dfloat v;
        if (i == p && j == p)
          v = dfloat{-col[64].hi, -col[64].lo};
        else if (i == p)
          v = wv[j];
        else if (j == p)
          v = wv[i];
        else
          v = df_sub(S[i * ld_s + j], df_mul(col[i], wv[j]));
        S[i * ld_s + j] = v;
      }
    }
    __syncthreads();
  }
}

// acc += a b in double-float: the product's rounding error (exact through the
// FMA) and the two-sum error of the addition collect in acc.lo, which stays a
// few ulp of acc.hi over a short sum; df_renorm makes the pair canonical.
__device__ __forceinline__ void df_fma_acc(dfloat &acc, dfloat a, dfloat b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const dfloat s = df_two_sum(acc.hi, p);
  acc.hi = s.hi;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, e));
}
__device__ __forceinline__ dfloat df_renorm(dfloat a) { return df_two_sum(a.hi, a.lo); }

// Scalar sweep of a 32 x 32 SPD block held in the lower triangle of S (row
// stride 33) in double-float: after the 32 pivots the lower triangle holds that
// of -S^-1, then both halves are filled.  Each pivot reads the block as it
// stood before the pivot from one buffer and writes the new values to the
// other (S and T alternate; 32 pivots end in S), so a pivot costs one block
// barrier: every thread forms 1 / d and reads column p itself, then updates
// the lower entries it owns (528 entries, about one per thread):
//   S_pp <- -1/d,  S_ip <- c_i / d,  S_ij <- S_ij - c_i (c_j / d).
// A non-positive pivot sets bit 0 of *err_flag.  blockDim.x == NT.
template <int NT>
__device__ inline void df_sweep32(dfloat *S, dfloat *T, int32_t *err_flag) {
  constexpr int EPT = (528 + NT - 1) / NT;
  int ei[EPT], ej[EPT];
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int e = (int)threadIdx.x + q * NT;
    ei[q] = -1;
    ej[q] = 0;
    if (e < 528) {
      int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
      while ((i + 1) * (i + 2) / 2 <= e) ++i;
      while (i * (i + 1) / 2 > e) --i;
      ei[q] = i;
      ej[q] = e - i * (i + 1) / 2;
    }
  }
  dfloat *src = S, *dst = T;
  for (int p = 0; p < 32; ++p) {
    const dfloat d = src[p * 33 + p];
    const bool pos = d.hi > 0.0f;
    const dfloat inv = pos ? df_recip(d) : dfloat{0.0f, 0.0f};
    if (threadIdx.x == 0 && !pos && err_flag) atomicOr(err_flag, 1);
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int i = ei[q], j = ej[q];
      if (i < 0) continue;
      const dfloat ci = (i >= p) ? src[i * 33 + p] : src[p * 33 + i];
      const dfloat cj = (j >= p) ? src[j * 33 + p] : src[p * 33 + j];
      const dfloat wj = df_mul(cj, inv);
      dfloat v;
      if (i == p && j == p)
        v = dfloat{-inv.hi, -inv.lo};
      else if (i == p)
        v = wj;
      else if (j == p)
        v = df_mul(ci, inv);
      else
        v = df_sub(src[i * 33 + j], df_mul(ci, wj));
      dst[i * 33 + j] = v;
    }
    __syncthreads();
    dfloat *t = src;
    src = dst;
    dst = t;
  }
  // 32 pivots: the result is in S
  for (int e = threadIdx.x; e < 1024; e += NT) {
    const int i = e >> 5, j = e & 31;
    if (i < j) S[i * 33 + j] = S[j * 33 + i];
  }
  __syncthreads();
}

// Shared scratch of sym_inverse64_df_2x2: the three blocks of the tile and
// the two products, 32 x 32 each with row stride 33.
struct Inverse64Smem {
  dfloat B11[32 * 33], B21[32 * 33], B22[32 * 33], U[32 * 33], X[32 * 33];
};

// P = Tk^-1 (64 x 64 float, both halves) for the SPD tile whose lower half is
// at Tk (row stride ld), in double-float, as a 2 x 2 block sweep: sweeping the
// index blocks K1 = [0, 32) and then K2 = [32, 64) is the same as sweeping the
// 64 indices one by one, and reads (N = -inverse of a swept block)
//   N11 = -B11^-1,  U = B21 B11^-1 = -B21 N11,  B22' = B22 - U B21^T,
//   N22 = -B22'^-1, X = B22'^-1 U = -N22 U,
//   -Tk^-1 = [[N11 - U^T X, X^T], [X, N22]].
// The 32 x 32 sweeps take one barrier per pivot with about one entry per
// thread; the four 32-term block products run on all threads with their
// sums in double-float.  A non-positive pivot sets bit 0 of *err_flag.
// blockDim.x == NT >= 512.
template <int NT>
__device__ inline void sym_inverse64_df_2x2(const float *Tk, int ld, float *P, Inverse64Smem &S,
                                             int32_t *err_flag) {
  const int tid = threadIdx.x;
  for (int e = tid; e < 1024; e += NT) {
    const int i = e >> 5, j = e & 31;
    S.B11[i * 33 + j] = dfloat{Tk[(int64_t)max(i, j) * ld + min(i, j)], 0.0f};
    S.B21[i * 33 + j] = dfloat{Tk[(int64_t)(32 + i) * ld + j], 0.0f};
    if (i >= j) S.B22[i * 33 + j] = dfloat{Tk[(int64_t)(32 + i) * ld + 32 + j], 0.0f};
  }
  __syncthreads();
  df_sweep32<NT>(S.B11, S.U, err_flag);   // B11 <- N11 (both halves; U as the second buffer)
  // U = -B21 N11
  for (int e = tid; e < 1024; e += NT) {
    const int i = e >> 5, j = e & 31;
    dfloat acc{0.0f, 0.0f};
#pragma unroll 8
    for (int k = 0; k < 32; ++k) df_fma_acc(acc, S.B21[i * 33 + k], S.B11[k * 33 + j]);
    acc = df_renorm(acc);
    S.U[i * 33 + j] = dfloat{-acc.hi, -acc.lo};
  }
  __syncthreads();
  // B22 <- B22 - U B21^T (lower)
  for (int e = tid; e < 1024; e += NT) {
    const int i = e >> 5, j = e & 31;
    if (i < j) continue;
    dfloat acc{0.0f, 0.0f};
#pragma unroll 8
    for (int k = 0; k < 32; ++k) df_fma_acc(acc, S.U[i * 33 + k], S.B21[j * 33 + k]);
    S.B22[i * 33 + j] = df_sub(S.B22[i * 33 + j], df_renorm(acc));
  }
  __syncthreads();
  df_sweep32<NT>(S.B22, S.X, err_flag);   // B22 <- N22 (both halves; X as the second buffer)
  // X = -N22 U
  for (int e = tid; e < 1024; e += NT) {
    const int i = e >> 5, j = e & 31;
    dfloat acc{0.0f, 0.0f};
#pragma unroll 8
    for (int k = 0; k < 32; ++k) df_fma_acc(acc, S.B22[i * 33 + k], S.U[k * 33 + j]);
    acc = df_renorm(acc);
    S.X[i * 33 + j] = dfloat{-acc.hi, -acc.lo};
  }
  __syncthreads();
  // N11 <- N11 - U^T X (lower), and the output
  for (int e = tid; e < 1024; e += NT) {
    const int i = e >> 5, j = e & 31;
    if (i < j) continue;
    dfloat acc{0.0f, 0.0f};
#pragma unroll 8
    for (int k = 0; k < 32; ++k) df_fma_acc(acc, S.U[k * 33 + i], S.X[k * 33 + j]);
    const dfloat v = df_sub(S.B11[i * 33 + j], df_renorm(acc));
    const float f = -__fadd_rn(v.hi, v.lo);
    P[i * 64 + j] = f;
    P[j * 64 + i] = f;
  }
  for (int e = tid; e < 1024; e += NT) {
    const int i = e >> 5, j = e & 31;
    const dfloat x = S.X[i * 33 + j];
    const float fx = -__fadd_rn(x.hi, x.lo);
    P[(32 + i) * 64 + j] = fx;
    P[j * 64 + 32 + i] = fx;
    const dfloat n = S.B22[i * 33 + j];
    P[(32 + i) * 64 + 32 + j] = -__fadd_rn(n.hi, n.lo);
  }
}

}  // namespace qsel
