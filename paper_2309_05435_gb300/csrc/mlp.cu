// Learned control variate: per-node features, a 14-64-64-1 GELU MLP with
// BF16 weights and FP32 accumulation (forward, backward, Adam) and the
// qsel_cv object of the C ABI.
//
// The network predicts log(c_i / v_i), the relative Rao-Blackwell correction
// of node i (Algorithm 4: v_i = Sigma*_ii + c_i).  A planner (qsel_cv_plan in
// api.cu) uses it to choose the overlap and the number of samples; the
// estimate itself stays plain RBMC.
//
// Parameter vector (FP32 master copy): W1 (64 x 14), b1 (64), W2 (64 x 64),
// b2 (64), W3 (64), b3 (1) = 5185 values, then the input mean (14) and scale
// (14).  The forward pass reads BF16 copies of W1, W2, W3.
#include <cuda_bf16.h>

#include <cmath>
#include <string>
#include <vector>

#include "qsel.h"
#include "kernels.cuh"

namespace qsel {
namespace mlp {

constexpr int NF = QSEL_CV_FEATURES;   // 14
constexpr int H = 64;
constexpr int OFF_W1 = 0, OFF_B1 = H * NF, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H, OFF_W3 = OFF_B2 + H,
              OFF_B3 = OFF_W3 + H, N_TRAIN = OFF_B3 + 1, OFF_MU = N_TRAIN, OFF_SC = OFF_MU + NF,
              N_ALL = OFF_SC + NF;
static_assert(N_TRAIN == QSEL_CV_PARAMS, "parameter count");
constexpr int TILE = 64;   // samples per backward CTA

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * __expf(-0.5f * x * x);
}

struct Weights {
  const __nv_bfloat16 *w1, *w2, *w3;
  const float *p;   // master parameters: biases, mean, scale
};

// Weights, biases, mean and scale staged in shared memory as float.
struct SmemW {
  float w1[H * NF], b1[H], w2[H * H], b2[H], w3[H], b3, mu[NF], sc[NF];
};

__device__ void stage_weights(const Weights &W, SmemW &s) {
  for (int i = threadIdx.x; i < H * NF; i += blockDim.x) s.w1[i] = __bfloat162float(W.w1[i]);
  for (int i = threadIdx.x; i < H * H; i += blockDim.x) s.w2[i] = __bfloat162float(W.w2[i]);
  for (int i = threadIdx.x; i < H; i += blockDim.x) {
    s.w3[i] = __bfloat162float(W.w3[i]);
    s.b1[i] = W.p[OFF_B1 + i];
    s.b2[i] = W.p[OFF_B2 + i];
  }
  for (int i = threadIdx.x; i < NF; i += blockDim.x) {
    s.mu[i] = W.p[OFF_MU + i];
    s.sc[i] = W.p[OFF_SC + i];
  }
  if (threadIdx.x == 0) s.b3 = W.p[OFF_B3];
  __syncthreads();
}

// One sample per thread.  With act set, a1 and a2 are stored (training).
__global__ void __launch_bounds__(256) k_mlp_forward(Weights W, const float *__restrict__ X, int n,
                                                     float *__restrict__ y, float *__restrict__ act) {
  __shared__ SmemW s;
  stage_weights(W, s);
  for (int smp = blockIdx.x * blockDim.x + threadIdx.x; smp < n; smp += gridDim.x * blockDim.x) {
    float xn[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) xn[k] = (X[(int64_t)smp * NF + k] - s.mu[k]) / s.sc[k];
    float h1[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
      float a = s.b1[j];
#pragma unroll
      for (int k = 0; k < NF; ++k) a = fmaf(s.w1[j * NF + k], xn[k], a);
      if (act) act[(int64_t)smp * 2 * H + j] = a;
      h1[j] = gelu(a);
    }
    float out = s.b3;
    for (int j = 0; j < H; ++j) {
      float a = s.b2[j];
#pragma unroll
      for (int k = 0; k < H; ++k) a = fmaf(s.w2[j * H + k], h1[k], a);
      if (act) act[(int64_t)smp * 2 * H + H + j] = a;
      out = fmaf(s.w3[j], gelu(a), out);
    }
    y[smp] = out;
  }
}

// Backward for TILE samples per CTA: per-sample deltas in shared memory, then
// the tile's partial weight gradients (mean-squared loss, 2 (y - t) / n).
struct SmemB {
  float xn[TILE][NF + 1];
  float h1[TILE][H + 1];
  float h2[TILE][H + 1];
  float d2[TILE][H + 1];
  float d1[TILE][H + 1];   // holds a1 first, then delta1
  float dy[TILE];
  float lsum[TILE];
};

__global__ void __launch_bounds__(256) k_mlp_backward(Weights W, const float *__restrict__ X,
                                                      const float *__restrict__ target, const float *__restrict__ y,
                                                      const float *__restrict__ act, int n,
                                                      float *__restrict__ partial, float *__restrict__ loss_partial) {
  extern __shared__ __align__(16) unsigned char smem_b[];
  SmemW &s = *reinterpret_cast<SmemW *>(smem_b);
  SmemB &b = *reinterpret_cast<SmemB *>(smem_b + ((sizeof(SmemW) + 15) / 16) * 16);
  stage_weights(W, s);
  const int s0 = blockIdx.x * TILE;
  const float inv_n = 2.0f / (float)n;
  for (int e = threadIdx.x; e < TILE * H; e += blockDim.x) {
    const int q = e / H, j = e - q * H;
    const int smp = s0 + q;
    float a1 = 0.f, a2 = 0.f;
    if (smp < n) {
      a1 = act[(int64_t)smp * 2 * H + j];
      a2 = act[(int64_t)smp * 2 * H + H + j];
    }
    b.h1[q][j] = (smp < n) ? gelu(a1) : 0.f;
    b.h2[q][j] = (smp < n) ? gelu(a2) : 0.f;
    b.d1[q][j] = a1;
    b.d2[q][j] = (smp < n) ? s.w3[j] * gelu_grad(a2) : 0.f;   // times dy below
  }
  for (int e = threadIdx.x; e < TILE * NF; e += blockDim.x) {
    const int q = e / NF, k = e - q * NF;
    const int smp = s0 + q;
    b.xn[q][k] = (smp < n) ? (X[(int64_t)smp * NF + k] - s.mu[k]) / s.sc[k] : 0.f;
  }
  if (threadIdx.x < TILE) {
    const int smp = s0 + threadIdx.x;
    const float diff = (smp < n) ? y[smp] - target[smp] : 0.f;
    b.dy[threadIdx.x] = diff * inv_n;
    b.lsum[threadIdx.x] = diff * diff;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TILE * H; e += blockDim.x) {
    const int q = e / H, j = e - q * H;
    b.d2[q][j] *= b.dy[q];
  }
  __syncthreads();
  // delta1[q][k] = (sum_j delta2[q][j] W2[j][k]) gelu'(a1[q][k])
  for (int e = threadIdx.x; e < TILE * H; e += blockDim.x) {
    const int q = e / H, k = e - q * H;
    float acc = 0.f;
#pragma unroll 8
    for (int j = 0; j < H; ++j) acc = fmaf(b.d2[q][j], s.w2[j * H + k], acc);
    b.d1[q][k] = acc * gelu_grad(b.d1[q][k]);
  }
  __syncthreads();
  float *out = partial + (int64_t)blockIdx.x * N_TRAIN;
  for (int e = threadIdx.x; e < H * H; e += blockDim.x) {   // W2[j][k]
    const int j = e / H, k = e - j * H;
    float acc = 0.f;
    for (int q = 0; q < TILE; ++q) acc = fmaf(b.d2[q][j], b.h1[q][k], acc);
    out[OFF_W2 + e] = acc;
  }
  for (int e = threadIdx.x; e < H * NF; e += blockDim.x) {  // W1[j][k]
    const int j = e / NF, k = e - j * NF;
    float acc = 0.f;
    for (int q = 0; q < TILE; ++q) acc = fmaf(b.d1[q][j], b.xn[q][k], acc);
    out[OFF_W1 + e] = acc;
  }
  for (int j = threadIdx.x; j < H; j += blockDim.x) {
    float g1 = 0.f, g2 = 0.f, g3 = 0.f;
    for (int q = 0; q < TILE; ++q) {
      g1 += b.d1[q][j];
      g2 += b.d2[q][j];
      g3 = fmaf(b.dy[q], b.h2[q][j], g3);
    }
    out[OFF_B1 + j] = g1;
    out[OFF_B2 + j] = g2;
    out[OFF_W3 + j] = g3;
  }
  if (threadIdx.x == 0) {
    float g = 0.f, l = 0.f;
    for (int q = 0; q < TILE; ++q) {
      g += b.dy[q];
      l += b.lsum[q];
    }
    out[OFF_B3] = g;
    loss_partial[blockIdx.x] = l;
  }
}

// grad[p] = sum over tiles (fixed order, double), loss = mean squared error.
__global__ void k_mlp_reduce(const float *__restrict__ partial, const float *__restrict__ loss_partial, int tiles,
                             int n, float *__restrict__ grad, float *__restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < N_TRAIN) {
    double acc = 0.0;
    for (int t = 0; t < tiles; ++t) acc += partial[(int64_t)t * N_TRAIN + p];
    grad[p] = (float)acc;
  }
  if (p == 0) {
    double l = 0.0;
    for (int t = 0; t < tiles; ++t) l += loss_partial[t];
    *loss = (float)(l / n);
  }
}

// Adam on the FP32 master parameters, then the BF16 copies of W1, W2, W3.
__global__ void k_adam(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, int step, float lr, __nv_bfloat16 *w1, __nv_bfloat16 *w2,
                       __nv_bfloat16 *w3) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N_TRAIN) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / (1.f - powf(b1, (float)step));
  const float vh = vi / (1.f - powf(b2, (float)step));
  const float pi = p[i] - lr * mh / (sqrtf(vh) + eps);
  p[i] = pi;
  if (i < OFF_B1) w1[i - OFF_W1] = __float2bfloat16(pi);
  else if (i >= OFF_W2 && i < OFF_B2) w2[i - OFF_W2] = __float2bfloat16(pi);
  else if (i >= OFF_W3 && i < OFF_B3) w3[i - OFF_W3] = __float2bfloat16(pi);
}

__global__ void k_sync_bf16(const float *__restrict__ p, __nv_bfloat16 *w1, __nv_bfloat16 *w2, __nv_bfloat16 *w3) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < H * NF) w1[i] = __float2bfloat16(p[OFF_W1 + i]);
  if (i < H * H) w2[i] = __float2bfloat16(p[OFF_W2 + i]);
  if (i < H) w3[i] = __float2bfloat16(p[OFF_W3 + i]);
}

// Per-feature mean and scale (standard deviation, floored) of X, one block
// per feature, written to the parameter vector.
__global__ void k_feature_stats(const float *__restrict__ X, int n, float *__restrict__ p) {
  __shared__ double s1[256], s2[256];
  const int k = blockIdx.x;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = X[(int64_t)i * NF + k];
    a += x;
    b += x * x;
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double mean = s1[0] / n;
    const double var = fmax(s2[0] / n - mean * mean, 0.0);
    p[OFF_MU + k] = (float)mean;
    p[OFF_SC + k] = (float)fmax(sqrt(var), 1e-3);
  }
}

}  // namespace mlp

// ---------------------------------------------------------------------------
// Per-node features of the current model for a given overlap (see the oracle
// documentation for the definition).  One thread per node.
// ---------------------------------------------------------------------------
__global__ void k_cv_features(SellPattern pat, BtModel m, int n_s, int n_t, const float *__restrict__ sep_dist,
                              const float *__restrict__ bnd_dist, double th0, double th1, double th2,
                              float *__restrict__ F) {
  const int n = n_s * n_t;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const int t = r / n_s, i = r - t * n_s;
    const int sl = i >> 5, li = i & 31;
    const int w = pat.slice_width[sl];
    const int base = pat.slice_ptr[sl] + li;
    double diag = (m.obs && m.obs[r]) ? m.obs_w : 0.0;
    double top[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) top[q] = 0.0;
    auto push = [&](double v) {
      if (!(v > top[7])) return;
      int q = 7;
      while (q > 0 && top[q - 1] < v) {
        top[q] = top[q - 1];
        --q;
      }
      top[q] = v;
    };
    const double c0 = m.diag.scale(t);
    const double cm = t > 0 ? m.off.scale(t - 1) : 0.0, cp = t + 1 < n_t ? m.off.scale(t) : 0.0;
    const double *v0 = m.diag.at(t);
    const double *vm = m.off.at(t > 0 ? t - 1 : 0);
    const double *vp = m.off.at(t + 1 < n_t ? t : 0);
    for (int s = 0; s < w; ++s) {
      const int idx = base + s * kSlice;
      const int j = pat.col[idx];
      const double v = c0 * v0[idx];
      if (j == i)
        diag += v;
      else if (v != 0.0)
        push(fabs(v));
      if (t > 0 && vm[idx] != 0.0) push(fabs(cm * vm[idx]));
      if (t + 1 < n_t && vp[idx] != 0.0) push(fabs(cp * vp[idx]));
    }
    float *f = F + (int64_t)r * mlp::NF;
    f[0] = (float)log(diag);
#pragma unroll
    for (int q = 0; q < 8; ++q) f[1 + q] = (float)log(top[q] > 1e-30 ? top[q] : 1e-30);
    f[9] = sep_dist[t];
    f[10] = bnd_dist[i];
    f[11] = (float)th0;
    f[12] = (float)th1;
    f[13] = (float)th2;
  }
}

void launch_cv_features(cudaStream_t s, const SellPattern &pat, const BtModel &m, int n_s, int n_t,
                        const float *sep_dist, const float *bnd_dist, const double th[3], float *F) {
  ++g_launch_count;
  const int n = n_s * n_t;
  int grid = (n + 255) / 256;
  if (grid > 152 * 8) grid = 152 * 8;
  k_cv_features<<<grid, 256, 0, s>>>(pat, m, n_s, n_t, sep_dist, bnd_dist, th[0], th[1], th[2], F);
}

// Per part p: sum over the rows of Omega_p (slabs [slab_start[p],
// slab_start[p+1])) of exp(2 y_i), the squared predicted ratio c_i / v_i.
// One CTA per part, double accumulation.
__global__ void k_cv_part_m2(const float *__restrict__ y, const int32_t *__restrict__ slab_start, int n_s,
                             double *__restrict__ out) {
  __shared__ double red[256];
  const int p = blockIdx.x;
  const int64_t r0 = (int64_t)slab_start[p] * n_s, r1 = (int64_t)slab_start[p + 1] * n_s;
  double a = 0.0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const double v = (double)y[r];
    a += exp(2.0 * v);
  }
  red[threadIdx.x] = a;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[p] = red[0];
}

void launch_cv_part_m2(cudaStream_t s, const float *y, const int32_t *slab_start_dev, int n_parts, int n_s,
                       double *out) {
  ++g_launch_count;
  k_cv_part_m2<<<n_parts, 256, 0, s>>>(y, slab_start_dev, n_s, out);
}

// y_i = log(cbar_i / (sel_i + cbar_i)), cbar_i the mean of the corrections,
// ratio clamped below at 1e-9 (a node below it adds less than 1e-18 to any
// planned squared error).
__global__ void k_cv_targets(CvTargetArgs a, const double *__restrict__ sel, int n, float *__restrict__ y) {
  const double inv = 1.0 / a.count;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double c = 0.0;
    for (int q = 0; q < a.count; ++q) c += a.corr[q][i];
    c *= inv;
    const double v = sel[i] + c;
    double r = c / v;
    if (!(r > 1e-9)) r = 1e-9;
    y[i] = (float)log(r);
  }
}

void launch_cv_targets(cudaStream_t s, const CvTargetArgs &a, const double *sel, int n, float *y) {
  ++g_launch_count;
  int grid = (n + 255) / 256;
  if (grid > 152 * 8) grid = 152 * 8;
  k_cv_targets<<<grid, 256, 0, s>>>(a, sel, n, y);
}

}  // namespace qsel

using namespace qsel;

struct qsel_cv {
  cudaStream_t stream = nullptr;
  float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr, *loss = nullptr;
  __nv_bfloat16 *w1 = nullptr, *w2 = nullptr, *w3 = nullptr;
  float *act = nullptr, *y = nullptr, *partial = nullptr, *loss_partial = nullptr;
  int cap = 0;      // samples the training buffers hold
  int step = 0;
  std::vector<void *> allocs;
  ~qsel_cv() {
    for (void *q : allocs) cudaFree(q);
  }
  bool alloc(void **q, size_t bytes) {
    if (cudaMalloc(q, bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    allocs.push_back(*q);
    return true;
  }
  bool ensure(int n) {
    if (n <= cap) return true;
    for (void **q : {(void **)&act, (void **)&y, (void **)&partial, (void **)&loss_partial}) {
      if (*q) {
        cudaFree(*q);
        for (auto &a : allocs)
          if (a == *q) a = nullptr;
        *q = nullptr;
      }
    }
    const int tiles = (n + mlp::TILE - 1) / mlp::TILE;
    if (!alloc((void **)&act, (size_t)n * 2 * mlp::H * sizeof(float)) || !alloc((void **)&y, (size_t)n * sizeof(float)) ||
        !alloc((void **)&partial, (size_t)tiles * mlp::N_TRAIN * sizeof(float)) ||
        !alloc((void **)&loss_partial, (size_t)tiles * sizeof(float)))
      return false;
    cap = n;
    return true;
  }
  mlp::Weights weights() const { return mlp::Weights{w1, w2, w3, p}; }
};

namespace {
thread_local std::string g_cv_error;

qsel_status cv_fail(qsel_status st, const std::string &m) {
  g_cv_error = m;
  set_context_free_error(m);
  return st;
}

int backward_smem() {
  return (int)(((sizeof(mlp::SmemW) + 15) / 16) * 16 + sizeof(mlp::SmemB));
}

qsel_status cv_forward_backward(qsel_cv *cv, const float *X, const float *target, int n) {
  using namespace mlp;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, backward_smem());
    attr = true;
  }
  if (!cv->ensure(n)) return cv_fail(QSEL_ENOMEM, "qsel_cv: device allocation failed");
  const int tiles = (n + TILE - 1) / TILE;
  g_launch_count += 3;
  k_mlp_forward<<<std::min((n + 255) / 256, 152 * 4), 256, 0, cv->stream>>>(cv->weights(), X, n, cv->y, cv->act);
  k_mlp_backward<<<tiles, 256, backward_smem(), cv->stream>>>(cv->weights(), X, target, cv->y, cv->act, n,
                                                              cv->partial, cv->loss_partial);
  k_mlp_reduce<<<(N_TRAIN + 255) / 256, 256, 0, cv->stream>>>(cv->partial, cv->loss_partial, tiles, n, cv->g,
                                                               cv->loss);
  return cudaGetLastError() == cudaSuccess ? QSEL_OK : cv_fail(QSEL_ECUDA, "qsel_cv: kernel launch failed");
}
}  // namespace

extern "C" {

qsel_status qsel_cv_create(qsel_cv **out, uint64_t seed, void *cuda_stream) {
  using namespace mlp;
  if (!out) return cv_fail(QSEL_EINVAL, "qsel_cv_create: out must not be NULL");
  *out = nullptr;
  qsel_cv *cv = new (std::nothrow) qsel_cv();
  if (!cv) return cv_fail(QSEL_ENOMEM, "qsel_cv_create: host allocation failed");
  cv->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (!cv->alloc((void **)&cv->p, N_ALL * sizeof(float)) || !cv->alloc((void **)&cv->m, N_TRAIN * sizeof(float)) ||
      !cv->alloc((void **)&cv->v, N_TRAIN * sizeof(float)) || !cv->alloc((void **)&cv->g, N_TRAIN * sizeof(float)) ||
      !cv->alloc((void **)&cv->loss, sizeof(float)) || !cv->alloc((void **)&cv->w1, H * NF * 2) ||
      !cv->alloc((void **)&cv->w2, H * H * 2) || !cv->alloc((void **)&cv->w3, H * 2)) {
    delete cv;
    return cv_fail(QSEL_ENOMEM, "qsel_cv_create: device allocation failed");
  }
  // Glorot-style initial weights from a seeded host generator (initial values
  // are an input of the training, not part of the method's arithmetic)
  std::vector<float> h(N_ALL, 0.f);
  uint64_t st = seed * 6364136223846793005ull + 1442695040888963407ull;
  auto unif = [&]() {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    return (float)((st >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f;
  };
  const float s1 = std::sqrt(6.f / (NF + H)), s2 = std::sqrt(6.f / (H + H)), s3 = std::sqrt(6.f / (H + 1));
  for (int i = 0; i < H * NF; ++i) h[OFF_W1 + i] = s1 * unif();
  for (int i = 0; i < H * H; ++i) h[OFF_W2 + i] = s2 * unif();
  for (int i = 0; i < H; ++i) h[OFF_W3 + i] = s3 * unif();
  for (int k = 0; k < NF; ++k) h[OFF_SC + k] = 1.f;
  if (cudaMemcpy(cv->p, h.data(), N_ALL * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(cv->m, 0, N_TRAIN * sizeof(float)) != cudaSuccess ||
      cudaMemset(cv->v, 0, N_TRAIN * sizeof(float)) != cudaSuccess) {
    delete cv;
    return cv_fail(QSEL_ECUDA, "qsel_cv_create: copy failed");
  }
  ++g_launch_count;
  k_sync_bf16<<<(H * H + 255) / 256, 256, 0, cv->stream>>>(cv->p, cv->w1, cv->w2, cv->w3);
  if (cudaStreamSynchronize(cv->stream) != cudaSuccess) {
    delete cv;
    return cv_fail(QSEL_ECUDA, "qsel_cv_create: kernel failed");
  }
  *out = cv;
  return QSEL_OK;
}

qsel_status qsel_cv_set_params(qsel_cv *cv, const float *params) {
  using namespace mlp;
  if (!cv || !params) return cv_fail(QSEL_EINVAL, "qsel_cv_set_params: NULL argument");
  if (cudaMemcpy(cv->p, params, N_ALL * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return cv_fail(QSEL_ECUDA, "qsel_cv_set_params: copy failed");
  ++g_launch_count;
  k_sync_bf16<<<(H * H + 255) / 256, 256, 0, cv->stream>>>(cv->p, cv->w1, cv->w2, cv->w3);
  return cudaStreamSynchronize(cv->stream) == cudaSuccess ? QSEL_OK
                                                         : cv_fail(QSEL_ECUDA, "qsel_cv_set_params: kernel failed");
}

qsel_status qsel_cv_get_params(const qsel_cv *cv, float *params) {
  if (!cv || !params) return cv_fail(QSEL_EINVAL, "qsel_cv_get_params: NULL argument");
  if (cudaStreamSynchronize(cv->stream) != cudaSuccess ||
      cudaMemcpy(params, cv->p, mlp::N_ALL * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return cv_fail(QSEL_ECUDA, "qsel_cv_get_params: copy failed");
  return QSEL_OK;
}

qsel_status qsel_cv_predict(const qsel_cv *cv, const float *X_dev, float *y_dev, int32_t n) {
  if (!cv || !X_dev || !y_dev || n < 1) return cv_fail(QSEL_EINVAL, "qsel_cv_predict: invalid argument");
  ++g_launch_count;
  mlp::k_mlp_forward<<<std::min((n + 255) / 256, 152 * 4), 256, 0, cv->stream>>>(cv->weights(), X_dev, n, y_dev,
                                                                                  nullptr);
  if (cudaStreamSynchronize(cv->stream) != cudaSuccess) return cv_fail(QSEL_ECUDA, "qsel_cv_predict: kernel failed");
  return QSEL_OK;
}

qsel_status qsel_cv_grad(qsel_cv *cv, const float *X_dev, const float *y_dev, int32_t n, float *grad_host,
                         float *loss_host) {
  if (!cv || !X_dev || !y_dev || !grad_host || n < 1) return cv_fail(QSEL_EINVAL, "qsel_cv_grad: invalid argument");
  qsel_status st = cv_forward_backward(cv, X_dev, y_dev, n);
  if (st) return st;
  if (cudaStreamSynchronize(cv->stream) != cudaSuccess ||
      cudaMemcpy(grad_host, cv->g, mlp::N_TRAIN * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess ||
      (loss_host && cudaMemcpy(loss_host, cv->loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess))
    return cv_fail(QSEL_ECUDA, "qsel_cv_grad: copy failed");
  return QSEL_OK;
}

qsel_status qsel_cv_train(qsel_cv *cv, const float *X_dev, const float *y_dev, int32_t n, int32_t steps, float lr,
                          int32_t set_input_stats, float *loss_out) {
  using namespace mlp;
  if (!cv || !X_dev || !y_dev || n < 1 || steps < 0 || !(lr > 0.f))
    return cv_fail(QSEL_EINVAL, "qsel_cv_train: invalid argument");
  if (set_input_stats) {
    ++g_launch_count;
    k_feature_stats<<<NF, 256, 0, cv->stream>>>(X_dev, n, cv->p);
  }
  for (int s = 0; s < steps; ++s) {
    qsel_status st = cv_forward_backward(cv, X_dev, y_dev, n);
    if (st) return st;
    ++cv->step;
    ++g_launch_count;
    k_adam<<<(N_TRAIN + 255) / 256, 256, 0, cv->stream>>>(cv->p, cv->m, cv->v, cv->g, cv->step, lr, cv->w1, cv->w2,
                                                           cv->w3);
  }
  if (loss_out) {
    // loss of the final parameters
    qsel_status st = cv_forward_backward(cv, X_dev, y_dev, n);
    if (st) return st;
    if (cudaMemcpyAsync(loss_out, cv->loss, sizeof(float), cudaMemcpyDeviceToHost, cv->stream) != cudaSuccess)
      return cv_fail(QSEL_ECUDA, "qsel_cv_train: copy failed");
  }
  if (cudaStreamSynchronize(cv->stream) != cudaSuccess) return cv_fail(QSEL_ECUDA, "qsel_cv_train: kernel failed");
  return QSEL_OK;
}

void qsel_cv_destroy(qsel_cv *cv) {
  if (!cv) return;
  cudaStreamSynchronize(cv->stream);
  delete cv;
}

}  // extern "C"
