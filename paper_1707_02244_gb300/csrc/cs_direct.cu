// Direct circulant product, one warp per kept row: the paper's own GPU scheme
// (Sec. 5.2, each output of A x formed as an O(n) dot product of x with the
// rotated generating vector).  It is a context comparator for the FFT path,
// not part of any solve.
#include <cuda_runtime.h>

#include "../../include/cs.h"

namespace {

constexpr int DW = 8;   // warps (rows) per CTA

// y_i = sum_j c[(j - rows_i) mod n] x_j   (row rows_i of C, C[i][j] = c[(j - i) mod n])
__global__ void __launch_bounds__(32 * DW) direct_forward_k(const float* __restrict__ c,
                                                          const int32_t* __restrict__ rows, int64_t m,
                                                          int64_t n, const float* __restrict__ x,
                                                          float* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * DW + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= m) return;
  const int64_t r = rows[i];
  if (r < 0 || r >= n) {   // invalid row: no access, NaN result
    if (lane == 0) y[i] = __int_as_float(0x7fc00000);
    return;
  }
  float acc = 0.f;
  // j = lane + 32 q; c index (j - r) mod n: contiguous across the warp
  for (int64_t j = lane; j < n; j += 32) {
    int64_t k = j - r;
    if (k < 0) k += n;
    acc = fmaf(__ldg(c + k), __ldg(x + j), acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) y[i] = acc;
}

}  // namespace

extern "C" cs_status cs_forward_direct(int64_t n, int64_t m, const float* c, const int32_t* rows, const float* x,
                                       float* y, void* stream) {
  if (n < 1 || m < 1 || m > n || !c || !rows || !x || !y) return CS_ERR_ARG;
  const int64_t blocks = (m + DW - 1) / DW;
  if (blocks > 0x7fffffff) return CS_ERR_UNSUPPORTED;
  direct_forward_k<<<(unsigned)blocks, 32 * DW, 0, static_cast<cudaStream_t>(stream)>>>(c, rows, m, n, x, y);
  return cudaGetLastError() == cudaSuccess ? CS_OK : CS_ERR_CUDA;
}
