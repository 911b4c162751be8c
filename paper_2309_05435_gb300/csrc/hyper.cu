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
#include "sweep.cuh"

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

// grad[j] = 1/2 prior_j - 1/2 (traces[j] + extra[j]) - 1/2 quad[j] (extra:
// the fixed effects' tr(S^-1 dS_j), or null); terms = (prior, traces + extra,
// quad) for the record.  tr_kc = tr(K^-1 C) = sum_i C_ii (K^-1)_ii,
// summed here in a fixed order over the diagonal of Kinv.
__global__ void __launch_bounds__(256) k_loglik_combine(const double *Kinv, int n_pad, const double *c_diag, int n_s,
                                                        int n_t, const double *theta, const double *traces,
                                                        const double *extra, const double *quad, double *grad,
                                                        double *terms) {
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
      // the log-determinant of the joint precision adds tr(S^-1 dS_j) with fixed effects
      const double tr = traces[j] + (extra ? extra[j] : 0.0);
      grad[j] = 0.5 * prior[j] - 0.5 * tr - 0.5 * quad[j];
      terms[j] = prior[j];
      terms[3 + j] = tr;
      terms[6 + j] = quad[j];
    }
  }
}

void launch_loglik_combine(cudaStream_t s, const double *Kinv, int n_pad, const double *c_diag, int n_s, int n_t,
                           const double *theta, const double *traces, const double *extra, const double *quad,
                           double *grad, double *terms) {
  ++g_launch_count;
  k_loglik_combine<<<1, 256, 0, s>>>(Kinv, n_pad, c_diag, n_s, n_t, theta, traces, extra, quad, grad, terms);
}

}  // namespace qsel

// ---------------------------------------------------------------------------
// Fixed effects y = A_u u + Z beta + eps, beta ~ N(0, I / beta_prec) (Section
// 2.3, Eqs. mean:4-5, var:1; Eq. hyperpar:3).  With Q_ub = A_u^T Z / sigma^2
// solved next to the data column (X[:, 0] = Q_uu^-1 A_u^T y / sigma^2,
// X[:, 1 + a] = W[:, a] = (Q_uu^-1 Q_ub)[:, a]):
//   S = beta_prec I + Z^T Z / sigma^2 - Q_bu W,   m = Z^T (y - A_u X[:, 0]) / sigma^2,
//   mu_beta = S^-1 m,  mu_u = X[:, 0] - W mu_beta,  diag Var(u) += diag(W S^-1 W^T),
//   d log|Q| / d theta_j += tr(S^-1 W^T dQ_j W).
// obs_nodes[q] is the q-th observed node; Z is n_obs x n_beta row-major.
// ---------------------------------------------------------------------------
namespace qsel {

// R[obs_nodes[q], 1 + a] = Z[q, a] / sigma^2 (the rest of those columns zero).
__global__ void __launch_bounds__(256) k_fe_rhs(double *R, int ld, const int32_t *obs_nodes, const double *Z,
                                                int n_obs, int n_beta, double inv_s2) {
  const int64_t total = (int64_t)n_obs * n_beta;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(i / n_beta), a = (int)(i % n_beta);
    R[(int64_t)obs_nodes[q] * ld + 1 + a] = Z[i] * inv_s2;
  }
}

void launch_fe_rhs(cudaStream_t s, double *R, int ld, const int32_t *obs_nodes, const double *Z, int n_obs,
                   int n_beta, double inv_s2) {
  ++g_launch_count;
  const int64_t total = (int64_t)n_obs * n_beta;
  k_fe_rhs<<<(int)std::min<int64_t>(152 * 8, (total + 255) / 256), 256, 0, s>>>(R, ld, obs_nodes, Z, n_obs, n_beta,
                                                                              inv_s2);
}

// Block (a, b), b < n_beta: S[a, b]; block (a, n_beta): m[a].  Fixed-order
// reduction over the observed nodes.
__global__ void __launch_bounds__(256) k_fe_schur(const double *X, int ld, const int32_t *obs_nodes, const double *Z,
                                                  const double *y, int n_obs, int n_beta, double inv_s2,
                                                  double beta_prec, double *S, double *m) {
  __shared__ double red[256];
  const int a = blockIdx.y, b = blockIdx.x;
  double acc = 0.0;
  for (int q = threadIdx.x; q < n_obs; q += 256) {
    const int64_t r = obs_nodes[q];
    const double za = Z[(int64_t)q * n_beta + a];
    if (b < n_beta)
      acc += za * (Z[(int64_t)q * n_beta + b] - X[r * ld + 1 + b]);
    else
      acc += za * (y[q] - X[r * ld]);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (b < n_beta)
      S[a * n_beta + b] = red[0] * inv_s2 + (a == b ? beta_prec : 0.0);
    else
      m[a] = red[0] * inv_s2;
  }
}

void launch_fe_schur(cudaStream_t s, const double *X, int ld, const int32_t *obs_nodes, const double *Z,
                     const double *y, int n_obs, int n_beta, double inv_s2, double beta_prec, double *S, double *m) {
  ++g_launch_count;
  k_fe_schur<<<dim3(n_beta + 1, n_beta), 256, 0, s>>>(X, ld, obs_nodes, Z, y, n_obs, n_beta, inv_s2, beta_prec, S, m);
}

// Sinv = S^-1 (the symmetric sweep in shared memory, which leaves -S^-1),
// mu_beta = Sinv m.  One block; n_beta <= 64.
__global__ void __launch_bounds__(256) k_fe_solve(const double *S, const double *m, int n_beta, double *Sinv,
                                                  double *mu_beta, int32_t *err_flag) {
  __shared__ double Sm[64 * 65];
  for (int i = threadIdx.x; i < n_beta * n_beta; i += 256) Sm[(i / n_beta) * 65 + i % n_beta] = S[i];
  __syncthreads();
  sym_sweep_inverse_smem(Sm, 65, n_beta, err_flag);
  for (int i = threadIdx.x; i < n_beta * n_beta; i += 256) Sinv[i] = -Sm[(i / n_beta) * 65 + i % n_beta];
  __syncthreads();
  for (int a = threadIdx.x; a < n_beta; a += 256) {
    double acc = 0.0;
    for (int b = 0; b < n_beta; ++b) acc += -Sm[a * 65 + b] * m[b];
    mu_beta[a] = acc;
  }
}

void launch_fe_solve(cudaStream_t s, const double *S, const double *m, int n_beta, double *Sinv, double *mu_beta,
                     int32_t *err_flag) {
  ++g_launch_count;
  k_fe_solve<<<1, 256, 0, s>>>(S, m, n_beta, Sinv, mu_beta, err_flag);
}

// mu_u[r] = X[r, 0] - sum_a W[r, a] mu_beta[a] (also written back to X[r, 0]);
// corr[r] = sum_ab W[r, a] Sinv[a, b] W[r, b].
__global__ void __launch_bounds__(256) k_fe_mean(double *X, int ld, int n, int n_beta, const double *mu_beta,
                                                 const double *Sinv, double *mu, double *corr) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const double *w = X + (int64_t)r * ld + 1;
    double v = X[(int64_t)r * ld], c = 0.0;
    for (int a = 0; a < n_beta; ++a) {
      v -= w[a] * mu_beta[a];
      double t = 0.0;
      for (int b = 0; b < n_beta; ++b) t += Sinv[a * n_beta + b] * w[b];
      c += w[a] * t;
    }
    mu[r] = v;
    X[(int64_t)r * ld] = v;
    corr[r] = c;
  }
}

void launch_fe_mean(cudaStream_t s, double *X, int ld, int n, int n_beta, const double *mu_beta, const double *Sinv,
                    double *mu, double *corr) {
  ++g_launch_count;
  k_fe_mean<<<std::min(152 * 8, (n + 255) / 256), 256, 0, s>>>(X, ld, n, n_beta, mu_beta, Sinv, mu, corr);
}

// C[a, b] = sum_r X[r, 1 + a] Y[r, 1 + b] (Y = dQ_j X), fixed-order reduction
// per block (a, b); then out = sum_ab Sinv[a, b] C[a, b] (k_fe_trace_sum).
__global__ void __launch_bounds__(256) k_fe_cross(const double *X, const double *Y, int ld, int n, int n_beta,
                                                  double *C) {
  __shared__ double red[256];
  const int a = blockIdx.y, b = blockIdx.x;
  double acc = 0.0;
  for (int r = threadIdx.x; r < n; r += 256) acc += X[(int64_t)r * ld + 1 + a] * Y[(int64_t)r * ld + 1 + b];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) C[a * n_beta + b] = red[0];
}

__global__ void k_fe_trace_sum(const double *Sinv, const double *C, int n_beta, double *out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double acc = 0.0;
    for (int i = 0; i < n_beta * n_beta; ++i) acc += Sinv[i] * C[i];
    *out = acc;
  }
}

void launch_fe_schur_trace(cudaStream_t s, const double *X, const double *Y, int ld, int n, int n_beta,
                           const double *Sinv, double *C, double *out) {
  g_launch_count += 2;
  k_fe_cross<<<dim3(n_beta, n_beta), 256, 0, s>>>(X, Y, ld, n, n_beta, C);
  k_fe_trace_sum<<<1, 32, 0, s>>>(Sinv, C, n_beta, out);
}

}  // namespace qsel
