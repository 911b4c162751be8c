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

}  // namespace qsel
