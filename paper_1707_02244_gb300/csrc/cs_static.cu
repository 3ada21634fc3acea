// Allocation-free circulant product: y = C x or C^T x for one generating
// vector, with its FFT work space in a fixed device array of this library
// instead of memory from cudaMalloc.
//
// Some callers cannot call cudaMalloc: code whose device memory is owned
// entirely by another allocator (a framework's caching allocator, or a fixed
// pool reserved up front), and latency-critical loops that cannot afford the
// implicit device synchronisation an allocation may cause.  This entry point
// serves them: the caller passes the inputs and the output, and the work
// space is the file-scope array below.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/cs.h"
#include "cs_internal.h"

namespace csk {

namespace {

constexpr int64_t kStaticMaxN = CS_STATIC_MAX_N;

// Three FP64 complex work vectors of the largest supported length (768 KiB).
// Every GPU that loads the library holds this array until the process exits.
// All calls share it: calls that overlap on the GPU race on it.
static __device__ __align__(256) double2 g_static_scratch[3 * kStaticMaxN];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct ScratchAddr {
  void* ctx = nullptr;        // CUDA context the address belongs to
  double2* addr = nullptr;
};
ScratchAddr g_scratch_addr[kMaxDevices];

// cuCtxGetCurrent from the driver, fetched through the runtime so that the
// library needs no link against libcuda.
using CtxGetCurrentFn = int (*)(void**);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<CtxGetCurrentFn>(f);
  }();
  return fn;
}

// Device address of the array in the current context.  In host code the
// array's name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress, looked up once per device with that device current.
// The lookup is repeated when the device's current context is another one
// than at the last lookup (after cudaDeviceReset the module, and with it the
// array, can be loaded at another address).
cudaError_t scratch_address(double2** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  CtxGetCurrentFn get = ctx_get_current();
  if (!get) return cudaErrorInitializationError;
  // null before the runtime has made a context current on this thread
  void* ctx = nullptr;
  if (get(&ctx) != 0) return cudaErrorInitializationError;
  std::lock_guard<std::mutex> lock(g_mu);
  ScratchAddr& sa = g_scratch_addr[dev];
  if (!sa.addr || !ctx || sa.ctx != ctx) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);   // makes the device's primary context current if none is
    if (e != cudaSuccess) return e;
    if (get(&ctx) != 0 || !ctx) return cudaErrorInitializationError;
    sa.addr = static_cast<double2*>(p);
    sa.ctx = ctx;
  }
  *out = sa.addr;
  return cudaSuccess;
}

constexpr int NTH = 256;

__global__ void real_to_complex64_k(const double* __restrict__ c, double2* __restrict__ a, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)NTH + threadIdx.x;
  if (i < n) a[i] = make_double2(c[i], 0.0);
}

__global__ void float_to_complex64_k(const float* __restrict__ x, double2* __restrict__ a, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)NTH + threadIdx.x;
  if (i < n) a[i] = make_double2((double)x[i], 0.0);
}

// w = conj(H X) with H = conj(chat) for C x, chat for C^T x; the inverse FFT
// is then conj(FFT(w)) / n, whose real part is the product.
__global__ void spectrum_product_k(const double2* __restrict__ chat, const double2* __restrict__ X,
                                   double2* __restrict__ w, int64_t n, int transpose) {
  const int64_t i = blockIdx.x * (int64_t)NTH + threadIdx.x;
  if (i >= n) return;
  const double2 h = transpose ? chat[i] : make_double2(chat[i].x, -chat[i].y);
  const double2 x = X[i];
  const double2 p = make_double2(h.x * x.x - h.y * x.y, h.x * x.y + h.y * x.x);
  w[i] = make_double2(p.x, -p.y);
}

__global__ void real_part_k(const double2* __restrict__ r, float* __restrict__ y, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)NTH + threadIdx.x;
  if (i < n) y[i] = (float)(r[i].x / (double)n);
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + NTH - 1) / NTH); }

}  // namespace
}  // namespace csk

using namespace csk;

extern "C" cs_status cs_circulant_apply_static(int64_t n, const double* c, const float* x, float* y,
                                               int transpose, void* stream) {
  if (!c || !x || !y) return CS_ERR_ARG;
  if (n < 64 || n > kStaticMaxN || (n & (n - 1)) != 0) return CS_ERR_UNSUPPORTED;
  // An error the caller left pending on this thread is not this call's: leave
  // it in place (peek does not clear it) and launch nothing.
  if (cudaPeekAtLastError() != cudaSuccess) return CS_ERR_CUDA;
  double2* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return CS_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double2* buf[3] = {base, base + n, base + 2 * n};
  // chat = FFT(c) in buffers 0 / 1
  real_to_complex64_k<<<nblk(n), NTH, 0, s>>>(c, buf[0], n);
  if (cudaGetLastError() != cudaSuccess) return CS_ERR_CUDA;
  double2* chat = nullptr;
  e = launch_fft64_complex(buf[0], buf[1], n, &chat, s);
  if (e != cudaSuccess) return CS_ERR_CUDA;
  double2* f0 = chat == buf[0] ? buf[1] : buf[0];   // the two buffers chat does not occupy
  double2* f1 = buf[2];
  // X = FFT(x)
  float_to_complex64_k<<<nblk(n), NTH, 0, s>>>(x, f0, n);
  if (cudaGetLastError() != cudaSuccess) return CS_ERR_CUDA;
  double2* X = nullptr;
  e = launch_fft64_complex(f0, f1, n, &X, s);
  if (e != cudaSuccess) return CS_ERR_CUDA;
  double2* w = X == f0 ? f1 : f0;
  spectrum_product_k<<<nblk(n), NTH, 0, s>>>(chat, X, w, n, transpose ? 1 : 0);
  if (cudaGetLastError() != cudaSuccess) return CS_ERR_CUDA;
  double2* R = nullptr;
  e = launch_fft64_complex(w, X, n, &R, s);
  if (e != cudaSuccess) return CS_ERR_CUDA;
  real_part_k<<<nblk(n), NTH, 0, s>>>(R, y, n);
  return cudaGetLastError() == cudaSuccess ? CS_OK : CS_ERR_CUDA;
}
