// Rao-Blackwell correction terms of the overlapping RBMC estimator
// (Section 3.2.3, Algorithm 4) and the trace estimator (Section 3.4.2,
// Eq. hyperpar:4).
//
// For subdomain p with local slabs 0..T-1 (global e0 + tau) and own slabs
// [lo, hi], the correction samples w = Q_{**}^-1 Q_{*S} x_S are given
// (T x n_pad x ld, zero beyond n_s rows / k columns).  For every own row i of
// slab tau this kernel adds
//   diag:   (1/k) sum_s w_i^2
//   traces: (1/k) sum_s w_i (dQ_j w)_i,
// with dQ_j the block-tridiagonal derivative of theta_j: diagonal blocks
// dA_j(t), couplings dB_j(t) on the spatial pattern.
#include "kernels.cuh"

namespace qsel {

constexpr int kCorrGrid = 152 * 2;

int corr_grid() { return kCorrGrid; }

// (w_i^T dQ_j w) = sum over pattern entries l of row i and time offsets d of
// M_{j,d}[i, l] * sum_c w_i(c) w_{l, t+d}(c): the column sums q_d are formed
// once per entry and shared by every j.
template <typename T>
__global__ void __launch_bounds__(256) k_correction_terms(CorrBatch<T> bt, SellPattern pat, DerivModels dm, int n_s,
                                                          int n_pad, int ld, int k) {
  __shared__ double red[8][kMaxTheta];
  const CorrEntry<T> e = bt.e[blockIdx.y];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double inv_k = 1.0 / (double)k;
  const int n_own = (e.hi - e.lo + 1) * n_s;
  const int64_t slab = (int64_t)n_pad * ld;
  double tr[kMaxTheta] = {0.0, 0.0, 0.0, 0.0};
  for (int item = blockIdx.x * 8 + warp; item < n_own; item += gridDim.x * 8) {
    const int tl = e.lo + item / n_s;      // local slab
    const int i = item - (item / n_s) * n_s;
    const int t = e.e0 + tl;               // global slab
    const bool has_m = tl > 0, has_p = tl + 1 < e.T_;
    const int sl = i >> 5, li = i & 31;
    const int w = pat.slice_width[sl];
    const int base = pat.slice_ptr[sl] + li;
    const T *wrow = e.w + tl * slab + (int64_t)i * ld;
    double sq = 0.0, q4 = 0.0;
    for (int c = lane; c < ld; c += 32) {
      const double wi = (double)wrow[c];
      sq = fma(wi, wi, sq);
      q4 = fma(wi * wi, wi * wi, q4);
    }
    double p[kMaxTheta] = {0.0, 0.0, 0.0, 0.0};
    for (int s = 0; s < w; ++s) {
      const int idx = base + s * kSlice;
      const T *wc = e.w + tl * slab + (int64_t)pat.col[idx] * ld;
      double q0 = 0.0, qm = 0.0, qp = 0.0;
      for (int c = lane; c < ld; c += 32) {
        const double wi = (double)wrow[c];
        q0 = fma(wi, (double)wc[c], q0);
        if (has_m) qm = fma(wi, (double)wc[c - slab], qm);
        if (has_p) qp = fma(wi, (double)wc[c + slab], qp);
      }
#pragma unroll
      for (int j = 0; j < kMaxTheta; ++j) {
        if (j >= dm.n) break;
        double acc = dm.diag[j].scale(t) * dm.diag[j].at(t)[idx] * q0;
        if (has_m) acc = fma(dm.off[j].scale(t - 1) * dm.off[j].at(t - 1)[idx], qm, acc);
        if (has_p) acc = fma(dm.off[j].scale(t) * dm.off[j].at(t)[idx], qp, acc);
        p[j] += acc;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      sq += __shfl_down_sync(0xffffffffu, sq, o);
      q4 += __shfl_down_sync(0xffffffffu, q4, o);
#pragma unroll
      for (int j = 0; j < kMaxTheta; ++j) p[j] += __shfl_down_sync(0xffffffffu, p[j], o);
    }
    if (lane == 0) {
      e.corr_out[(int64_t)t * n_s + i] = sq * inv_k;
      if (e.corr4_out) e.corr4_out[(int64_t)t * n_s + i] = q4 * inv_k;
#pragma unroll
      for (int j = 0; j < kMaxTheta; ++j) tr[j] += p[j];
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < kMaxTheta; ++j) red[warp][j] = tr[j];
  }
  __syncthreads();
  if (threadIdx.x < kMaxTheta) {
    double s = 0.0;
    for (int ww = 0; ww < 8; ++ww) s += red[ww][threadIdx.x];
    e.partial[blockIdx.x * kMaxTheta + threadIdx.x] = s * inv_k;
  }
}

template <typename T>
void launch_correction_terms(cudaStream_t s, const CorrBatch<T> &b, const SellPattern &pat, const DerivModels &dm,
                             int n_s, int n_pad, int ld, int k) {
  if (b.count <= 0) return;
  ++g_launch_count;
  ProfScope ps_(s, PROF_CORR);
  k_correction_terms<T><<<dim3(kCorrGrid, b.count), 256, 0, s>>>(b, pat, dm, n_s, n_pad, ld, k);
}
template void launch_correction_terms<double>(cudaStream_t, const CorrBatch<double> &, const SellPattern &,
                                              const DerivModels &, int, int, int, int);
template void launch_correction_terms<float>(cudaStream_t, const CorrBatch<float> &, const SellPattern &,
                                             const DerivModels &, int, int, int, int);

// tr_j = sum over own row slabs t of
//   <dA_j(t), Sigma_tt> - <dB_j(t), Y_t> - <dB_j(t-1), Y_{t-1}>
// (Sigma_{t,t+1} = -Y_t^T, Sigma_{t,t-1} = -Y_{t-1}, the blocks symmetric;
// sums hold the pattern inner products without the scales) plus the
// correction partials.  One thread, fixed order.
__global__ void k_trace_combine(const TraceSlab *__restrict__ slabs, int n_slabs,
                                const double *__restrict__ sums, const double *__restrict__ partials,
                                int n_partials, DerivModels dm, double *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double acc[kMaxTheta] = {0.0, 0.0, 0.0, 0.0};
  for (int q = 0; q < n_slabs; ++q) {
    const TraceSlab sl = slabs[q];
    const int t = sl.t;
    for (int j = 0; j < dm.n; ++j) {
      acc[j] += dm.diag[j].scale(t) * sums[kMaxTheta * sl.sd + j];
      if (sl.sy >= 0) acc[j] -= dm.off[j].scale(t) * sums[kMaxTheta * sl.sy + j];
      if (sl.sym >= 0) acc[j] -= dm.off[j].scale(t - 1) * sums[kMaxTheta * sl.sym + j];
    }
  }
  for (int q = 0; q < n_partials; ++q)
    for (int j = 0; j < dm.n; ++j) acc[j] += partials[kMaxTheta * q + j];
  for (int j = 0; j < dm.n; ++j) out[j] = acc[j];
}

void launch_trace_combine(cudaStream_t s, const TraceSlab *slabs_dev, int n_slabs, const double *sums,
                          const double *partials, int n_partials, const DerivModels &dm, double *out) {
  ++g_launch_count;
  k_trace_combine<<<1, 32, 0, s>>>(slabs_dev, n_slabs, sums, partials, n_partials, dm, out);
}

template <typename T>
__global__ void k_add(T *__restrict__ y, const T *__restrict__ x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += x[i];
}

template <typename T>
void launch_add(cudaStream_t s, T *y, const T *x, int64_t n) {
  if (n <= 0) return;
  ++g_launch_count;
  int64_t grid = (n + 255) / 256;
  if (grid > 152 * 8) grid = 152 * 8;
  k_add<T><<<(int)grid, 256, 0, s>>>(y, x, n);
}
template void launch_add<double>(cudaStream_t, double *, const double *, int64_t);
template void launch_add<float>(cudaStream_t, float *, const float *, int64_t);

// Per part p: sum over the rows of Omega_p of Var_hat / v_i^2 with
// Var_hat = (m4_i - m2_i^2) / (k - 1), the estimated variance of the mean of
// the k values w_i^2.  One CTA per part.
__global__ void k_part_error_sums(const double *__restrict__ m2, const double *__restrict__ m4,
                                  const double *__restrict__ v, const int32_t *__restrict__ slab_start, int n_s,
                                  int k, double *__restrict__ out) {
  __shared__ double red[256];
  const int p = blockIdx.x;
  const int64_t r0 = (int64_t)slab_start[p] * n_s, r1 = (int64_t)slab_start[p + 1] * n_s;
  const double inv = 1.0 / (double)(k - 1);
  double a = 0.0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const double var = fmax(m4[r] - m2[r] * m2[r], 0.0) * inv;
    a += var / (v[r] * v[r]);
  }
  red[threadIdx.x] = a;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[p] = red[0];
}

void launch_part_error_sums(cudaStream_t s, const double *m2, const double *m4, const double *v,
                            const int32_t *slab_start_dev, int n_parts, int n_s, int k, double *out) {
  ++g_launch_count;
  k_part_error_sums<<<n_parts, 256, 0, s>>>(m2, m4, v, slab_start_dev, n_s, k, out);
}

__global__ void k_sum(double *__restrict__ out, const double *__restrict__ a, const double *__restrict__ b, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = a[i] + b[i];
}

void launch_sum(cudaStream_t s, double *out, const double *a, const double *b, int n) {
  if (n <= 0) return;
  ++g_launch_count;
  int grid = (n + 255) / 256;
  if (grid > 152 * 8) grid = 152 * 8;
  k_sum<<<grid, 256, 0, s>>>(out, a, b, n);
}

}  // namespace qsel
