// Theta-dependent model values (Sections 2.1-2.3).
//
// The spatial pattern and the theta-free parts C, G and H = G C^-1 G are
// built once at context creation; here the device turns theta into
//   Q_s = kappa^4 C + 2 kappa^2 G + H            (alpha = 2, lumped mass)
//   dQ_s/dlog kappa = 4 kappa^4 C + 4 kappa^2 G
//   M = (kappa^2 C + G) C^-1/2                    (factor of Q_s = M M^T)
// and the scalars of the unit-variance AR(1) time structure.
#include "kernels.cuh"

namespace qsel {

thread_local int64_t g_launch_count = 0;
thread_local Profiler *g_prof = nullptr;

__global__ void k_time_coeffs(const double *__restrict__ theta, int n_t, TimeCoeffs tc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double log_kappa = theta[0], log_tau = theta[1], logit_rho = theta[2];
  const double kappa = exp(log_kappa);
  const double tau = exp(log_tau);
  const double rho = 1.0 / (1.0 + exp(-logit_rho));
  const double om = 1.0 - rho * rho;            // 1 - rho^2
  const double drho_deta = rho * (1.0 - rho);   // d rho / d logit rho
  for (int t = 0; t < n_t; ++t) {
    // R = B^T B: 1 at both ends, 1 + rho^2 inside (1 - rho^2 for one slab)
    double R, dR;
    if (n_t == 1) {
      R = om;
      dR = -2.0 * rho;
    } else if (t == 0 || t == n_t - 1) {
      R = 1.0;
      dR = 0.0;
    } else {
      R = 1.0 + rho * rho;
      dR = 2.0 * rho;
    }
    tc.a0[t] = tau * R / om;
    tc.r0[t] = tau * drho_deta * (dR / om + R * 2.0 * rho / (om * om));
    tc.bdiag[t] = (t == 0) ? sqrt(om) : 1.0;
    if (t + 1 < n_t) {
      // off-diagonal of R is -rho, of dR/drho is -1
      tc.a1[t] = -tau * rho / om;
      tc.r1[t] = tau * drho_deta * (-1.0 / om - rho * 2.0 * rho / (om * om));
    }
  }
  tc.scalars[0] = kappa;
  tc.scalars[1] = tau;
  tc.scalars[2] = rho;
  tc.scalars[3] = sqrt(tau / om);
  tc.scalars[4] = -rho;
}

void launch_time_coeffs(cudaStream_t s, const double *theta_dev, int n_t, TimeCoeffs tc) {
  ++g_launch_count;
  k_time_coeffs<<<1, 32, 0, s>>>(theta_dev, n_t, tc);
}

__global__ void k_qs_values(int n_ent, const double *__restrict__ c_pat,
                            const double *__restrict__ g_pat, const double *__restrict__ h_pat,
                            const double *__restrict__ isqc_pat, const double *__restrict__ scalars,
                            double *__restrict__ qs, double *__restrict__ dqs,
                            double *__restrict__ kc) {
  const double kappa = scalars[0];
  const double k2 = kappa * kappa;
  const double k4 = k2 * k2;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_ent; e += gridDim.x * blockDim.x) {
    const double c = c_pat[e], g = g_pat[e];
    qs[e] = k4 * c + 2.0 * k2 * g + h_pat[e];
    dqs[e] = 4.0 * k4 * c + 4.0 * k2 * g;
    kc[e] = (k2 * c + g) * isqc_pat[e];
  }
}

void launch_qs_values(cudaStream_t s, int n_ent, const double *c_pat, const double *g_pat,
                      const double *h_pat, const double *isqc_pat, const double *scalars,
                      double *qs, double *dqs, double *kc) {
  ++g_launch_count;
  int grid = (n_ent + 255) / 256;
  if (grid > 1024) grid = 1024;
  if (grid < 1) grid = 1;
  k_qs_values<<<grid, 256, 0, s>>>(n_ent, c_pat, g_pat, h_pat, isqc_pat, scalars, qs, dqs, kc);
}

}  // namespace qsel
