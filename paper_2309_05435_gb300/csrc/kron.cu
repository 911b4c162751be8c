// Kronecker preconditioner of the sampler's PCG for grid meshes:
//   M^-1 = (I (x) Dh (x) Dh) (U (x) V (x) V) diag(1 / (tau mu_k (kappa^2 +
//          lambda_a + lambda_b)^2 + omega)) (U (x) V (x) V)^T (I (x) Dh (x) Dh)
// with V, lambda the eigenpairs of the scaled 1-D Neumann stiffness
// D^-1/2 T D^-1/2, Dh = D^-1/2, U, mu those of Q_t, omega the mean
// observation weight (the prior of Sections 2.1-2.2 with the lumped mass taken
// as D (x) D, plus omega C~ for A^T A / sigma^2).
//
// Applying it is six passes of one batched, strided small-matrix product:
// for every group g (the two indices not transformed) y_g = B x_g or B^T x_g,
// where x_g gathers the rows base(g) + k * kstride, k < dim, of the n x ld
// block (all samples at once).  A CTA computes a 64-row x 64-column output
// tile, looping over 64-wide K slices staged in shared memory; each thread
// accumulates an 8 x 2 register tile.  The diagonal scalings are fused into
// the passes that touch them.
#include <type_traits>

#include "kernels.cuh"

namespace qsel {

constexpr int kKT = 64;     // output rows / K slice per tile

template <typename T, int CW>
struct KronSmem {
  static constexpr int BP = kKT + 16 / (int)sizeof(T);    // padded rows: 16-byte aligned
  static constexpr int XP = CW + 16 / (int)sizeof(T);
  static constexpr int bytes = (kKT * BP + kKT * XP) * (int)sizeof(T);
};

// CW columns per tile (64 or 128): each thread accumulates an 8-row x
// (CW / 32)-column register tile from 16-byte shared loads.
template <typename T, int CW>
__global__ void __launch_bounds__(256) k_kron_pass(const KronPass p, const T *__restrict__ x, T *__restrict__ y) {
  using SM = KronSmem<T, CW>;
  constexpr int NC = CW / 32;
  using V16 = typename std::conditional<std::is_same<T, float>::value, float4, double2>::type;
  constexpr int E16 = 16 / (int)sizeof(T);
  extern __shared__ __align__(16) unsigned char smem_kron[];
  T *Bs = reinterpret_cast<T *>(smem_kron);                 // Bs[k * BP + o] = op(B)[o][k]
  const T *Bt = static_cast<const T *>(p.Bt);
  const T *scale = static_cast<const T *>(p.scale);
  T *xs = Bs + kKT * SM::BP;                                // xs[k * XP + c]
  const int tid = threadIdx.x, rg = tid >> 5, cg = tid & 31;
  const int row_tiles = (p.dim + kKT - 1) / kKT;
  const int col_tiles = p.ld / CW;
  const int64_t n_groups = (int64_t)p.n_outer * p.n_inner;
  const int64_t items = n_groups * row_tiles * col_tiles;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int ct = (int)(it % col_tiles);
    const int64_t rest = it / col_tiles;
    const int rt = (int)(rest % row_tiles);
    const int64_t g = rest / row_tiles;
    const int64_t base = (g / p.n_inner) * p.outer_stride + (g % p.n_inner) * p.inner_stride;
    const int g_inner = (int)(g % p.n_inner);
    const int o0 = rt * kKT, c0 = ct * CW;
    T acc[8][NC];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int q = 0; q < NC; ++q) acc[a][q] = T(0);
    for (int k0 = 0; k0 < p.dim; k0 += kKT) {
      __syncthreads();
      for (int e = tid; e < kKT * kKT; e += blockDim.x) {
        const int kk = e / kKT, oo = e - kk * kKT;
        const int o = o0 + oo, k = k0 + kk;
        Bs[kk * SM::BP + oo] = (o < p.dim && k < p.dim) ? Bt[(int64_t)k * p.dim + o] : T(0);
      }
      for (int e = tid; e < kKT * CW / E16; e += blockDim.x) {
        const int kk = e / (CW / E16), q = e - kk * (CW / E16);
        const int k = k0 + kk;
        V16 v;
        T *vs = reinterpret_cast<T *>(&v);
        if (k < p.dim) {
          v = *reinterpret_cast<const V16 *>(x + (base + (int64_t)k * p.kstride) * p.ld + c0 + q * E16);
          if (p.mode == KRON_IN_DH) {
            const T sc = scale[k * p.m + g_inner];
#pragma unroll
            for (int u = 0; u < E16; ++u) vs[u] *= sc;
          }
        } else {
#pragma unroll
          for (int u = 0; u < E16; ++u) vs[u] = T(0);
        }
        *reinterpret_cast<V16 *>(xs + kk * SM::XP + q * E16) = v;
      }
      __syncthreads();
      const int kmax = min(kKT, p.dim - k0);
#pragma unroll 4
      for (int kk = 0; kk < kmax; ++kk) {
        T bv[8], xv[NC];
        const V16 *bp = reinterpret_cast<const V16 *>(Bs + kk * SM::BP + rg * 8);
#pragma unroll
        for (int u = 0; u < 8 / E16; ++u) {
          const V16 t = bp[u];
          const T *ts = reinterpret_cast<const T *>(&t);
#pragma unroll
          for (int w = 0; w < E16; ++w) bv[u * E16 + w] = ts[w];
        }
#pragma unroll
        for (int q = 0; q < NC; ++q) xv[q] = xs[kk * SM::XP + cg * NC + q];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int q = 0; q < NC; ++q) acc[a][q] = fma(bv[a], xv[q], acc[a][q]);
      }
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int o = o0 + rg * 8 + a;
      if (o >= p.dim) continue;
      T sc = T(1);
      if (p.mode == KRON_OUT_DH)
        sc = scale[o * p.m + g_inner];
      else if (p.mode == KRON_OUT_SPEC)  // group = spatial index, o = temporal index
        sc = scale[(int64_t)o * p.m * p.m + g_inner];
      T *dst = y + (base + (int64_t)o * p.kstride) * p.ld + c0 + cg * NC;
#pragma unroll
      for (int q = 0; q < NC; ++q) dst[q] = acc[a][q] * sc;
    }
  }
}

template <typename T, int CW>
static void kron_pass_cw(cudaStream_t s, const KronPass &p, const T *x, T *y) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_kron_pass<T, CW>, cudaFuncAttributeMaxDynamicSharedMemorySize, KronSmem<T, CW>::bytes);
    attr = true;
  }
  const int64_t items = (int64_t)p.n_outer * p.n_inner * ((p.dim + kKT - 1) / kKT) * (p.ld / CW);
  const int grid = (int)std::min<int64_t>(items, 152 * 6);
  k_kron_pass<T, CW><<<grid, 256, KronSmem<T, CW>::bytes, s>>>(p, x, y);
}

template <typename T>
void launch_kron_pass(cudaStream_t s, const KronPass &p, const T *x, T *y) {
  ++g_launch_count;
  if (p.ld % 128 == 0)
    kron_pass_cw<T, 128>(s, p, x, y);
  else
    kron_pass_cw<T, 64>(s, p, x, y);
}
template void launch_kron_pass<double>(cudaStream_t, const KronPass &, const double *, double *);
template void launch_kron_pass<float>(cudaStream_t, const KronPass &, const float *, float *);

// partial_a[cta][c] = sum r z, partial_b[cta][c] = sum r r over the CTA's rows
// (the layout the PCG's beta reduction reads), columns in 64-wide chunks.
template <typename T>
__global__ void __launch_bounds__(256) k_pcg_dots(PcgVec<T> v) {
  __shared__ double red[2][4][64];
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int64_t rows_per = (v.n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = blockIdx.x * rows_per, r1 = min((int64_t)v.n, r0 + rows_per);
  for (int c0 = 0; c0 < v.ld; c0 += 64) {
    const int c = c0 + tx;
    T sa = T(0), sb = T(0);
    for (int64_t r = r0 + ty; r < r1; r += 4) {
      const T rv = v.r[r * v.ld + c];
      sa = fma(rv, v.z[r * v.ld + c], sa);
      sb = fma(rv, rv, sb);
    }
    red[0][ty][tx] = (double)sa;
    red[1][ty][tx] = (double)sb;
    __syncthreads();
    if (ty == 0) {
      v.partial_a[(int64_t)blockIdx.x * v.ld + c] = red[0][0][tx] + red[0][1][tx] + red[0][2][tx] + red[0][3][tx];
      v.partial_b[(int64_t)blockIdx.x * v.ld + c] = red[1][0][tx] + red[1][1][tx] + red[1][2][tx] + red[1][3][tx];
    }
    __syncthreads();
  }
}

template <typename T>
void launch_pcg_dots(cudaStream_t s, const PcgVec<T> &v) {
  ++g_launch_count;
  k_pcg_dots<T><<<v.n_tiles, 256, 0, s>>>(v);
}
template void launch_pcg_dots<double>(cudaStream_t, const PcgVec<double> &);
template void launch_pcg_dots<float>(cudaStream_t, const PcgVec<float> &);

// The preconditioner's tables in T for one theta (see KronOperator): the
// factors and their transposes, dh_i dh_j, and the spectral scaling formed
// in double and rounded once.
template <typename T>
__global__ void __launch_bounds__(256) k_kron_tables(KronOperator op) {
  const int m = op.m, n_t = op.n_t, n_s = m * m;
  const int64_t total = 2 * (int64_t)m * m + 2 * (int64_t)n_t * n_t + (int64_t)m * m + (int64_t)n_t * n_s;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = i;
    if (r < (int64_t)m * m) {
      static_cast<T *>(op.tV)[r] = (T)op.V[r];
      continue;
    }
    r -= (int64_t)m * m;
    if (r < (int64_t)m * m) {
      const int a = (int)(r / m), b = (int)(r % m);
      static_cast<T *>(op.tVT)[r] = (T)op.V[(int64_t)b * m + a];
      continue;
    }
    r -= (int64_t)m * m;
    if (r < (int64_t)n_t * n_t) {
      static_cast<T *>(op.tU)[r] = (T)op.U[r];
      continue;
    }
    r -= (int64_t)n_t * n_t;
    if (r < (int64_t)n_t * n_t) {
      const int a = (int)(r / n_t), b = (int)(r % n_t);
      static_cast<T *>(op.tUT)[r] = (T)op.U[(int64_t)b * n_t + a];
      continue;
    }
    r -= (int64_t)n_t * n_t;
    if (r < (int64_t)m * m) {
      const int a = (int)(r / m), b = (int)(r % m);
      static_cast<T *>(op.dhdh)[r] = (T)(op.dh[a] * op.dh[b]);
      continue;
    }
    r -= (int64_t)m * m;
    const int t = (int)(r / n_s), s = (int)(r % n_s);
    const int sa = s / m, sb = s - sa * m;
    const double s2 = op.kappa2 + op.lam[sa] + op.lam[sb];
    static_cast<T *>(op.spec)[r] = (T)(1.0 / (op.tau * op.mu[t] * s2 * s2 + op.omega));
  }
}

template <typename T>
void launch_kron_tables(cudaStream_t s, const KronOperator &op) {
  ++g_launch_count;
  k_kron_tables<T><<<152, 256, 0, s>>>(op);
  if constexpr (std::is_same<T, float>::value) {
    if (op.use_tc) {
      const int64_t mm = (int64_t)op.m * op.m, tt = (int64_t)op.n_t * op.n_t;
      const void *src[4] = {op.tV, op.tVT, op.tU, op.tUT};
      const int64_t cnt[4] = {mm, mm, tt, tt};
      for (int q = 0; q < 4; ++q)
        launch_split_tf32(s, static_cast<const float *>(src[q]), op.split[q][0], op.split[q][1], cnt[q]);
    }
  }
}
template void launch_kron_tables<double>(cudaStream_t, const KronOperator &);
template void launch_kron_tables<float>(cudaStream_t, const KronOperator &);

// z = M^-1 r: six passes, ping-pong between the scratch q and z (q is free
// once the AXPY has consumed Q p); the result ends in z.  With split float
// tables the whole apply runs on the tensor cores (kron_tc.cu).
template <typename T>
void launch_kron_apply(cudaStream_t s, const KronOperator &op, const T *r, T *q, T *z) {
  if constexpr (std::is_same<T, float>::value) {
    if (op.use_tc) {
      ProfScope ps_(s, PROF_PRECOND);
      if (launch_kron_apply_tc(s, op, r, q, z)) return;
    }
  }
  const int m = op.m, n_s = m * m, n_t = op.n_t;
  KronPass p{};
  p.ld = op.ld;
  p.m = m;
  p.scale = op.dhdh;
  // spatial index s = i m + j inside slab t (row t n_s + s)
  KronPass over_i = p, over_j = p, over_t = p;
  over_i.dim = m;
  over_i.kstride = m;
  over_i.n_outer = n_t;
  over_i.outer_stride = n_s;
  over_i.n_inner = m;
  over_i.inner_stride = 1;
  over_j.dim = m;
  over_j.kstride = 1;
  over_j.n_outer = n_t;
  over_j.outer_stride = n_s;
  over_j.n_inner = m;
  over_j.inner_stride = m;
  over_t.dim = n_t;
  over_t.kstride = n_s;
  over_t.n_outer = 1;
  over_t.outer_stride = 0;
  over_t.n_inner = n_s;
  over_t.inner_stride = 1;
  ProfScope ps_(s, PROF_PRECOND);
  // op(B)^T is B for the transposed passes and B^T for the others
  KronPass a = over_i;          // (V^T over i) after the input scaling Dh (x) Dh
  a.Bt = op.tV;
  a.mode = KRON_IN_DH;
  launch_kron_pass<T>(s, a, r, q);
  KronPass b = over_j;          // V^T over j
  b.Bt = op.tV;
  b.mode = KRON_NONE;
  launch_kron_pass<T>(s, b, q, z);
  KronPass c = over_t;          // U^T over t, then the spectral scaling
  c.Bt = op.tU;
  c.mode = KRON_OUT_SPEC;
  c.scale = op.spec;
  launch_kron_pass<T>(s, c, z, q);
  KronPass d = over_t;          // U over t
  d.Bt = op.tUT;
  d.mode = KRON_NONE;
  launch_kron_pass<T>(s, d, q, z);
  KronPass e = over_j;          // V over j
  e.Bt = op.tVT;
  e.mode = KRON_NONE;
  launch_kron_pass<T>(s, e, z, q);
  KronPass f = over_i;          // V over i, then Dh (x) Dh
  f.Bt = op.tVT;
  f.mode = KRON_OUT_DH;
  launch_kron_pass<T>(s, f, q, z);
}
template void launch_kron_apply<double>(cudaStream_t, const KronOperator &, const double *, double *, double *);
template void launch_kron_apply<float>(cudaStream_t, const KronOperator &, const float *, float *, float *);

}  // namespace qsel
