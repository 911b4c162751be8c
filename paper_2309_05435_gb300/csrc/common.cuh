// Internal helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>

namespace qsel {

// Dense tiles are 64 x 64; dense matrices are padded to a multiple of 64 with
// an identity block on the padded diagonal, which leaves every inverse and
// product exact on the leading n_s x n_s part.
constexpr int kTile = 64;
// Sample columns are padded to a multiple of 64 with zero right-hand sides.
constexpr int kColPad = 64;
// Width of a slice of the sliced-ELL spatial pattern.
constexpr int kSlice = 32;

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }
inline int64_t round_up64(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Status carried through host code.
struct Err {
  int code = 0;        // qsel_status
  std::string msg;
};

// Sliced-ELL (SELL-32) spatial pattern of Q_s: the union of the patterns of
// C, G and G C^-1 G.  Slice s covers rows [32 s, 32 s + 32); entry (slot, lane)
// of slice s sits at slice_ptr[s] + slot * 32 + lane.  Padding entries point
// at the row itself with zero coefficients.
struct SellPattern {
  int n_rows = 0;
  int n_slices = 0;
  int max_width = 0;
  const int32_t *slice_ptr = nullptr;   // n_slices + 1
  const int32_t *slice_width = nullptr; // n_slices
  const int32_t *col = nullptr;         // entries
};

// Spatial blocks of a block-tridiagonal precision on the common SELL pattern:
// block t has the entries scale(t) * v[t * stride + e] (stride 0: one array
// for every block, scaled per block by coef; coef null: scale 1).  The
// separable model stores Q_s once with the time coefficients as scales; the
// diffusion model and user-given block-tridiagonal matrices store one array
// per block.
struct BlockVals {
  const double *v = nullptr;
  int64_t stride = 0;
  const double *coef = nullptr;
  __host__ __device__ const double *at(int t) const { return v + (int64_t)t * stride; }
  __host__ __device__ const double *scale_ptr(int t) const { return coef ? coef + t : nullptr; }
#ifdef __CUDACC__
  __device__ double scale(int t) const { return coef ? coef[t] : 1.0; }
#endif
};
// A block-tridiagonal precision with symmetric blocks on one spatial pattern:
// diagonal blocks A_t (t < n_t) plus obs_w on the diagonal of observed nodes,
// couplings B_t = Q[t, t+1] = Q[t+1, t] (t < n_t - 1).
struct BtModel {
  BlockVals diag, off;
  const uint8_t *obs = nullptr;   // may be null: no observation diagonal
  double obs_w = 0.0;
};
// Largest number of hyperparameters with a trace gradient.
constexpr int kMaxTheta = 4;
// dQ/dtheta_j as block-tridiagonal matrices on the same pattern (no
// observation term).
struct DerivModels {
  BlockVals diag[kMaxTheta], off[kMaxTheta];
  int n = 0;
};

// Theta-dependent scalars of the time structure, written by a device kernel.
//   a0[t] = tau Q_t[t,t], a1[t] = tau Q_t[t,t+1]
//   r0[t], r1[t]: the same for d/dlogit rho
//   bdiag[t] = B[t,t]; boff = B[t+1,t] = -rho; fscale = sqrt(tau/(1-rho^2))
struct TimeCoeffs {
  double *a0, *a1, *r0, *r1, *bdiag;
  double *scalars;  // [0] kappa, [1] tau, [2] rho, [3] fscale, [4] boff
};

}  // namespace qsel

#define QSEL_CUDA_TRY(expr)                                                        \
  do {                                                                             \
    cudaError_t _e = (expr);                                                       \
    if (_e != cudaSuccess) {                                                       \
      return ::qsel::cuda_fail(_e, #expr, __FILE__, __LINE__);                     \
    }                                                                              \
  } while (0)

namespace qsel {
Err cuda_fail(cudaError_t e, const char *what, const char *file, int line);
}
