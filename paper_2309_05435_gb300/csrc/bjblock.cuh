// Diagonal blocks of Q for the block-Jacobi preconditioners: rows
// [r0, r0 + b) of the global order, assembled from the spatial pattern and
// the time coefficients (Q = c_{t,t+d} Q_s blocks + diag(obs) / sigma^2).
#pragma once

#include "kernels.cuh"

namespace qsel {

// S (b x b, row stride ld_s, shared memory) <- Q[r0:r0+b, r0:r0+b]; rows past
// n get the identity.  All threads of the block take part.
__device__ inline void assemble_diag_block(double *S, int ld_s, const SellPattern &pat, const double *qs,
                                           const double *a0, const double *a1, const uint8_t *obs, double obs_w,
                                           int n_s, int n_t, int r0, int b) {
  const int n = n_s * n_t;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e - (e / b) * b;
    S[i * ld_s + j] = (i == j && r0 + i >= n) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int rr = threadIdx.x; rr < b; rr += blockDim.x) {
    const int row = r0 + rr;
    if (row >= n) continue;
    const int t = row / n_s, i = row - t * n_s;
    const int sl = i >> 5, li = i & 31;
    const int w = pat.slice_width[sl];
    const int base = pat.slice_ptr[sl] + li;
    for (int s = 0; s < w; ++s) {
      const int j = pat.col[base + s * kSlice];
      const double v = qs[base + s * kSlice];
      for (int d = -1; d <= 1; ++d) {
        const int u = t + d;
        if (u < 0 || u >= n_t) continue;
        const int colg = u * n_s + j;
        if (colg < r0 || colg >= r0 + b) continue;
        const double c = (d == 0) ? a0[t] : (d < 0 ? a1[t - 1] : a1[t]);
        S[rr * ld_s + (colg - r0)] += c * v;
      }
    }
    if (obs != nullptr && obs[row]) S[rr * ld_s + rr] += obs_w;
  }
  __syncthreads();
}

}  // namespace qsel
