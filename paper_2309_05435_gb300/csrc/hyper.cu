// Posterior mean and the gradient of the hyperparameter marginal (no fixed
// effects):
//   mu = Q^-1 b,  b = A^T y / sigma^2                         (Eq. mean:5)
//   d log p(y|theta) / d theta_j = 1/2 tr(Q_x^-1 dQ_x_j) - 1/2 tr(Q^-1 dQ_j)
//                                  - 1/2 mu^T dQ_x_j mu       (Eqs. hyperpar:1, 3, 4)
// with dQ_j = dQ_x_j and the prior log-determinant derivatives in closed
// form: d/dlog kappa = 4 n_t kappa^2 tr(K^-1 C), d/dlog tau = n,
// d/dlogit rho = n_s 2 rho^2 (n_t - 1) / (1 + rho).  The solve for mu is
// the sampler's PCG; the quadratic forms are the block-tridiagonal SpMM with
// the derivative coefficients and its fused per-column dot partials; K^-1
// comes from the blocked sweep on the dense K.
#include "kernels.cuh"

namespace qsel {

// R[:, 0] = A^T y / sigma^2 (R zeroed before): node r observed (obs[r])
// receives y[obs_index[r]], its rank among the observed nodes.
__global__ void __launch_bounds__(256) k_data_rhs(double *R, int ld, const uint8_t *obs, const int32_t *obs_index,
                                                  const double *y, int n, double inv_s2) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
    if (obs[r]) R[(int64_t)r * ld] = y[obs_index[r]] * inv_s2;
}

void launch_data_rhs(cudaStream_t s, double *R, int ld, const uint8_t *obs, const int32_t *obs_index,
                     const double *y, int n, double inv_s2) {
  ++g_launch_count;
  k_data_rhs<<<std::min(152 * 8, (n + 255) / 256), 256, 0, s>>>(R, ld, obs, obs_index, y, n, inv_s2);
}

// out = sum_r partial[r * ld + col] in a fixed order (one block).
__global__ void __launch_bounds__(256) k_column_sum(const double *partial, int rows, int ld, int col, double *out) {
  __shared__ double red[256];
  double a = 0.0;
  for (int r = threadIdx.x; r < rows; r += 256) a += partial[(int64_t)r * ld + col];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

void launch_column_sum(cudaStream_t s, const double *partial, int rows, int ld, int col, double *out) {
  ++g_launch_count;
  k_column_sum<<<1, 256, 0, s>>>(partial, rows, ld, col, out);
}

// Dense K = kappa^2 C + G (n_pad x n_pad, zeroed before) from the values of C
// and G on the SELL pattern of Q_s, which contains theirs; padding slots
// repeat the diagonal with zero values.  Padded rows get a unit diagonal.
// kappa from theta[0] = log kappa.
__global__ void __launch_bounds__(256) k_dense_K(double *K, int n_pad, SellPattern pat, const double *c_pat,
                                                 const double *g_pat, const double *theta, int n_s) {
  const double kappa2 = exp(2.0 * theta[0]);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += gridDim.x * blockDim.x) {
    if (i >= n_s) {
      K[(int64_t)i * n_pad + i] = 1.0;
      continue;
    }
    const int sl = i >> 5, li = i & 31;
    const int w = pat.slice_width[sl];
    const int base = pat.slice_ptr[sl] + li;
    for (int s = 0; s < w; ++s) {
      const int e = base + s * kSlice;
      K[(int64_t)i * n_pad + pat.col[e]] += kappa2 * c_pat[e] + g_pat[e];
    }
  }
}

void launch_dense_K(cudaStream_t s, double *K, int n_pad, const SellPattern &pat, const double *c_pat,
                    const double *g_pat, const double *theta, int n_s) {
  ++g_launch_count;
  k_dense_K<<<std::min(152 * 4, (n_pad + 255) / 256), 256, 0, s>>>(K, n_pad, pat, c_pat, g_pat, theta, n_s);
}

// grad[j] = 1/2 prior_j - 1/2 traces[j] - 1/2 quad[j]; terms = (prior,
// traces, quad) for the record.  tr_kc = tr(K^-1 C) = sum_i C_ii (K^-1)_ii,
// summed here in a fixed order over the diagonal of Kinv.
__global__ void __launch_bounds__(256) k_loglik_combine(const double *Kinv, int n_pad, const double *c_diag, int n_s,
                                                        int n_t, const double *theta, const double *traces,
                                                        const double *quad, double *grad, double *terms) {
  __shared__ double red[256];
  double a = 0.0;
  for (int i = threadIdx.x; i < n_s; i += 256) a += c_diag[i] * Kinv[(int64_t)i * n_pad + i];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double kappa2 = exp(2.0 * theta[0]);
    const double rho = 1.0 / (1.0 + exp(-theta[2]));
    double prior[3];
    prior[0] = 4.0 * n_t * kappa2 * red[0];
    prior[1] = (double)n_s * n_t;
    prior[2] = n_s * 2.0 * rho * rho * (n_t - 1) / (1.0 + rho);
    for (int j = 0; j < 3; ++j) {
      grad[j] = 0.5 * prior[j] - 0.5 * traces[j] - 0.5 * quad[j];
      terms[j] = prior[j];
      terms[3 + j] = traces[j];
      terms[6 + j] = quad[j];
    }
  }
}

void launch_loglik_combine(cudaStream_t s, const double *Kinv, int n_pad, const double *c_diag, int n_s, int n_t,
                           const double *theta, const double *traces, const double *quad, double *grad,
                           double *terms) {
  ++g_launch_count;
  k_loglik_combine<<<1, 256, 0, s>>>(Kinv, n_pad, c_diag, n_s, n_t, theta, traces, quad, grad, terms);
}

}  // namespace qsel
