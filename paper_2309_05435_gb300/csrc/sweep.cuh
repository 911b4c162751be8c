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

// Register-resident double-float sweep of a 64 x 64 SPD tile (the lower
// triangle of Tk, row stride ld), written as -(Tk^-1) in float to P (64 x 64,
// both halves).  Thread t owns up to R = 5 consecutive entries of one column
// j of the lower triangle (442 segments) and keeps them in registers for the
// whole sweep.  Pivot p needs only column p of the matrix before the pivot
// (c_k = A_kp, both halves by symmetry) and 1 / A_pp: the owners publish them
// in shared memory at the end of pivot p - 1 (double-buffered), so a pivot
// costs one block barrier.  Its update
//   A_pp <- -1/d,  A_ip <- c_i / d,  A_ij <- A_ij - c_i (c_j / d)
// takes one double-float product per entry; the sum keeps its rounding error
// in the low word without renormalising (the value stays exact to the
// double-float level; only the published column, the multiplicand of the next
// pivot, is renormalised).  A non-positive pivot sets bit 0 of *err_flag.
// blockDim.x == NT >= 442.
template <int NT>
__device__ inline void sym_sweep_inverse64_reg_df(const float *Tk, int ld, float *P, int32_t *err_flag) {
  static_assert(NT >= 442, "one thread per column segment");
  constexpr int R = 5;
  __shared__ dfloat colbuf[2][64];
  __shared__ dfloat invbuf[2];
  const int t = threadIdx.x;
  int j = -1, r0 = 64, cnt = 0;
  {
    int base = 0;
    for (int jj = 0; jj < 64; ++jj) {
      const int segs = (64 - jj + R - 1) / R;
      if (t < base + segs) {
        j = jj;
        r0 = jj + (t - base) * R;
        cnt = min(R, 64 - r0);
        break;
      }
      base += segs;
    }
  }
  float ah[R], al[R];
#pragma unroll
  for (int u = 0; u < R; ++u) {
    ah[u] = (u < cnt) ? Tk[(int64_t)(r0 + u) * ld + j] : 0.0f;
    al[u] = 0.0f;
  }
  // column 0 and 1 / A_00 for the first pivot
  if (j == 0) {
#pragma unroll
    for (int u = 0; u < R; ++u)
      if (u < cnt) colbuf[0][r0 + u] = dfloat{ah[u], 0.0f};
    if (r0 == 0) {
      const dfloat d{ah[0], 0.0f};
      const bool pos = d.hi > 0.0f;
      invbuf[0] = pos ? df_recip(d) : dfloat{0.0f, 0.0f};
      if (!pos && err_flag) atomicOr(err_flag, 1);
    }
  }
  __syncthreads();
  for (int p = 0; p < 64; ++p) {
    const int b = p & 1;
    if (j >= 0) {
      const dfloat inv = invbuf[b];
      if (j == p) {
#pragma unroll
        for (int u = 0; u < R; ++u) {
          if (u >= cnt) continue;
          const dfloat v = (r0 + u == p) ? dfloat{-inv.hi, -inv.lo} : df_mul(dfloat{ah[u], al[u]}, inv);
          ah[u] = v.hi;
          al[u] = v.lo;
        }
      } else {
        const dfloat w = df_mul(colbuf[b][j], inv);
#pragma unroll
        for (int u = 0; u < R; ++u) {
          if (u >= cnt) continue;
          const int i = r0 + u;
          const dfloat c = colbuf[b][i];
          const float pr = __fmul_rn(c.hi, w.hi);
          float e = __fmaf_rn(c.hi, w.hi, -pr);
          e = __fmaf_rn(c.hi, w.lo, e);
          e = __fmaf_rn(c.lo, w.hi, e);
          const dfloat sm = df_two_sum(ah[u], -pr);
          const float lo = __fadd_rn(al[u], __fsub_rn(sm.lo, e));
          const bool on_row = i == p;   // entry (p, j), j < p: c_j / d
          ah[u] = on_row ? w.hi : sm.hi;
          al[u] = on_row ? w.lo : lo;
        }
      }
      // column p + 1 for the next pivot (renormalised), and its 1 / d
      const int q = p + 1;
      if (q < 64) {
        if (j == q) {
#pragma unroll
          for (int u = 0; u < R; ++u) {
            if (u >= cnt) continue;
            const dfloat v = df_two_sum(ah[u], al[u]);
            ah[u] = v.hi;
            al[u] = v.lo;
            colbuf[b ^ 1][r0 + u] = v;
          }
          if (r0 == q) {
            const dfloat d{ah[0], al[0]};
            const bool pos = d.hi > 0.0f;
            invbuf[b ^ 1] = pos ? df_recip(d) : dfloat{0.0f, 0.0f};
            if (!pos && err_flag) atomicOr(err_flag, 1);
          }
        } else if (j < q) {
#pragma unroll
          for (int u = 0; u < R; ++u) {
            if (u >= cnt || r0 + u != q) continue;
            const dfloat v = df_two_sum(ah[u], al[u]);
            ah[u] = v.hi;
            al[u] = v.lo;
            colbuf[b ^ 1][j] = v;
          }
        }
      }
    }
    __syncthreads();
  }
  if (j >= 0) {
#pragma unroll
    for (int u = 0; u < R; ++u) {
      if (u >= cnt) continue;
      const int i = r0 + u;
      const float v = -__fadd_rn(ah[u], al[u]);
      P[i * 64 + j] = v;
      P[j * 64 + i] = v;
    }
  }
}

}  // namespace qsel
