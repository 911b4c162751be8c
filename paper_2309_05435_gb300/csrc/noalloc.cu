// Allocation-free SPD inverse (qsel_spd_inverse_noalloc in qsel.h).
//
// Some callers cannot let a library call cudaMalloc: code inside a framework
// whose caching allocator already owns the device memory budget (a foreign
// allocation can fail or fragment what the framework reserved), and
// long-running services that must keep their device memory footprint fixed
// after start-up.  This entry point serves them: it inverts one SPD matrix in
// place in caller-owned device memory, using as scratch only the file-scope
// array below, which every GPU that loads this module holds until the
// process exits.  The call reads its pivot status back to the host and
// synchronises the caller's stream before it returns.
#include <mutex>

#include "qsel.h"
#include "kernels.cuh"

namespace qsel {
namespace {

constexpr int kNoAllocMaxN = QSEL_NOALLOC_MAX_N;
constexpr size_t kPadMat = (size_t)kNoAllocMaxN * kNoAllocMaxN;  // padded copy of A
constexpr size_t kPanel = (size_t)kNoAllocMaxN * 64;              // sweep panels U, V
constexpr size_t kFlagOff = kPadMat + 64 * 64 + 2 * kPanel;       // error word
constexpr size_t kScratchDoubles = kFlagOff + 32;

// Shared by every call on a device: calls that overlap on the GPU race.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

__global__ void k_noalloc_pad_in(const double *__restrict__ a, int n, int lda, int n_pad,
                                 double *__restrict__ dst) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (c >= n_pad) return;
  double v;
  if (r < n && c < n)
    v = a[(int64_t)r * lda + c];
  else
    v = (r == c) ? 1.0 : 0.0;
  dst[(int64_t)r * n_pad + c] = v;
}

__global__ void k_noalloc_copy_out(const double *__restrict__ src, int n_pad, int n,
                                   double *__restrict__ a, int lda) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (c >= n) return;
  a[(int64_t)r * lda + c] = src[(int64_t)r * n_pad + c];
}

std::mutex g_mu;
double *g_dev_ptr[128] = {};

struct ErrorSink {
  ErrorSink &operator=(const std::string &m) {
    set_context_free_error(m);
    return *this;
  }
} g_noalloc_error;

// Device address of the scratch array on the current device, looked up once
// per device with that device current (the host-side symbol is only a
// stand-in and must never be passed to a kernel).  A device reset would
// invalidate the cached address; calls after one are not supported.
cudaError_t scratch_on_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev_ptr[dev]) {
    double *p = nullptr;
    e = cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_dev_ptr[dev] = p;
  }
  *out = g_dev_ptr[dev];
  return cudaSuccess;
}

}  // namespace

}  // namespace qsel

using namespace qsel;

extern "C" qsel_status qsel_spd_inverse_noalloc(double *a_dev, int32_t n, int32_t lda, void *cuda_stream) {
  if (!a_dev || n < 1 || lda < n) {
    g_noalloc_error = "qsel_spd_inverse_noalloc: a_dev must not be NULL, n >= 1 and lda >= n";
    return QSEL_EINVAL;
  }
  if (n > kNoAllocMaxN) {
    g_noalloc_error = "qsel_spd_inverse_noalloc: n = " + std::to_string(n) + " exceeds QSEL_NOALLOC_MAX_N = " +
                      std::to_string(kNoAllocMaxN);
    return QSEL_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  double *base = nullptr;
  cudaError_t e = scratch_on_current_device(&base);
  if (e != cudaSuccess) {
    g_noalloc_error = std::string("qsel_spd_inverse_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
    return QSEL_ECUDA;
  }
  const int n_pad = round_up(n, kTile);
  double *A = base;
  int32_t *flag = reinterpret_cast<int32_t *>(base + kFlagOff);
  SweepBatch<double> b{};
  b.count = 1;
  b.e[0].A = A;
  b.e[0].P = base + kPadMat;
  b.e[0].U = base + kPadMat + 64 * 64;
  b.e[0].V = base + kPadMat + 64 * 64 + kPanel;
  e = cudaMemsetAsync(flag, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) {
    ++g_launch_count;
    k_noalloc_pad_in<<<dim3((n_pad + 255) / 256, n_pad), 256, 0, s>>>(a_dev, n, lda, n_pad, A);
    spd_inverse(s, b, n_pad, flag);
    ++g_launch_count;
    k_noalloc_copy_out<<<dim3((n + 255) / 256, n), 256, 0, s>>>(A, n_pad, n, a_dev, lda);
    e = cudaGetLastError();
  }
  int32_t hflag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    g_noalloc_error = std::string("qsel_spd_inverse_noalloc: CUDA error ") + cudaGetErrorString(e);
    return QSEL_ECUDA;
  }
  if (hflag & 1) {
    g_noalloc_error = "qsel_spd_inverse_noalloc: a pivot was not positive (matrix not SPD)";
    return QSEL_ENOTSPD;
  }
  return QSEL_OK;
}
