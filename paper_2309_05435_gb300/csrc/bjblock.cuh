// Diagonal blocks of Q for the block-Jacobi preconditioners: rows
// [r0, r0 + b) of the global order, assembled from the spatial pattern and
// the block values of the model (diagonal blocks A_t, couplings B_t and the
// observation diagonal).
#pragma once

#include "kernels.cuh"

namespace qsel {

// S (b x b, row stride ld_s, shared memory) <- Q[r0:r0+b, r0:r0+b]; rows past
// n get the identity.  All threads of the block take part.
__device__ inline void assemble_diag_block(double *S, int ld_s, const SellPattern &pat, const BtModel &m, int n_s,
                                           int n_t, int r0, int b) {
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
    const double c0 = m.diag.scale(t);
    const double cm = t > 0 ? m.off.scale(t - 1) : 0.0, cp = t + 1 < n_t ? m.off.scale(t) : 0.0;
    const double *v0 = m.diag.at(t);
    const double *vm = t > 0 ? m.off.at(t - 1) : nullptr;
    const double *vp = t + 1 < n_t ? m.off.at(t) : nullptr;
    for (int s = 0; s < w; ++s) {
      const int idx = base + s * kSlice;
      const int j = pat.col[idx];
      for (int d = -1; d <= 1; ++d) {
        const int u = t + d;
        if (u < 0 || u >= n_t) continue;
        const int colg = u * n_s + j;
        if (colg < r0 || colg >= r0 + b) continue;
        const double v = (d == 0) ? c0 * v0[idx] : (d < 0 ? cm * vm[idx] : cp * vp[idx]);
        S[rr * ld_s + (colg - r0)] += v;
      }
    }
    if (m.obs != nullptr && m.obs[row]) S[rr * ld_s + rr] += m.obs_w;
  }
  __syncthreads();
}

}  // namespace qsel
