// Plan-time and bookkeeping kernels: FP64 spectrum of c, twiddle and spectrum
// tables, the row mask of Omega, y scatter / gather, deterministic reductions.
#include "cs_fft.cuh"
#include "cs_internal.h"

namespace csk {

namespace {

constexpr int AUX_NT = 256;

__global__ void set_args_k(CallArgs a, CallArgs* dst) { *dst = a; }

// Deterministic final sum of per-block partials, slot by slot.
__global__ void __launch_bounds__(AUX_NT) finalize_k(const double* __restrict__ partials, int nblk,
                                                     double* __restrict__ stats) {
  __shared__ double red[AUX_NT];
  for (int k = 0; k < NSTAT; ++k) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += AUX_NT) s += partials[b * NSTAT + k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = AUX_NT / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) stats[k] = red[0];
    __syncthreads();
  }
}

// dst[q] = exp(-2 pi i q / M), evaluated in FP64 (exact rational argument)
// and rounded once to fp32.
__global__ void twiddle_k(float2* dst, int count, int64_t M) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  double s, c;
  sincospi(-2.0 * (double)q / (double)M, &s, &c);
  dst[q] = make_float2((float)c, (float)s);
}

// Stage-major twiddle table of a length-L FFT (see stage_twiddle): the
// stage with span Ls and radix R holds w_{Ls R}^(r k) at row(r) Ls + k for
// the rows r it keeps (tw_row_r).
__global__ void stage_tw_k(float2* dst, int lgL, int count) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  int lgLs = 4;
  while (true) {
    const int lgR = (lgL - lgLs) >= 4 ? 4 : (lgL - lgLs);
    const int sz = tw_rows(lgR) << lgLs;
    if (t < sz) {
      const int r = tw_row_r(lgR, t >> lgLs), k = t & ((1 << lgLs) - 1);
      double sn, cs;
      sincospi(-2.0 * (double)(r * k) / (double)(1 << (lgLs + lgR)), &sn, &cs);
      dst[blockIdx.x * blockDim.x + threadIdx.x] = make_float2((float)cs, (float)sn);
      return;
    }
    t -= sz;
    lgLs += lgR;
  }
}

__global__ void c_to_complex_k(const double* __restrict__ c, double2* __restrict__ a, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) a[i] = make_double2(c[i], 0.0);
}

// One radix-2 Stockham stage of the FP64 plan-time FFT (global memory):
// butterfly j pairs a[j] and a[j + n/2]; Ls is the current sub-transform length.
__global__ void fft64_stage_k(const double2* __restrict__ in, double2* __restrict__ out, int64_t n,
                              int64_t Ls) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t h = n >> 1;
  if (j >= h) return;
  const int64_t k = j & (Ls - 1);
  double s, c;
  sincospi(-(double)k / (double)Ls, &s, &c);   // exp(-2 pi i k / (2 Ls))
  const double2 a = in[j], b0 = in[j + h];
  const double2 b = make_double2(b0.x * c - b0.y * s, b0.x * s + b0.y * c);
  const int64_t o = ((j - k) << 1) + k;
  out[o] = make_double2(a.x + b.x, a.y + b.y);
  out[o + Ls] = make_double2(a.x - b.x, a.y - b.y);
}

// The same stage over `batch` transforms of length L with element i of
// transform t at t * bs + i * es (rows: es = 1, bs = L; columns: es = width,
// bs = 1).
__global__ void fft64_strided_stage_k(const double2* __restrict__ in, double2* __restrict__ out, int64_t L,
                                      int64_t Ls, int64_t batch, int64_t es, int64_t bs) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t h = L >> 1;
  if (idx >= h * batch) return;
  const int64_t t = idx / h, j = idx - t * h;
  const int64_t k = j & (Ls - 1);
  double s, c;
  sincospi(-(double)k / (double)Ls, &s, &c);
  const int64_t base = t * bs;
  const double2 a = in[base + j * es], b0 = in[base + (j + h) * es];
  const double2 b = make_double2(b0.x * c - b0.y * s, b0.x * s + b0.y * c);
  const int64_t o = ((j - k) << 1) + k;
  out[base + o * es] = make_double2(a.x + b.x, a.y + b.y);
  out[base + (o + Ls) * es] = make_double2(a.x - b.x, a.y - b.y);
}

// chat_k of a real vector: bins 0 and n/2 are real by construction.
__device__ __forceinline__ double2 chat_at(const double2* chat, int64_t n, int64_t k) {
  double2 v = chat[k];
  if (k == 0 || k == (n >> 1)) v.y = 0.0;
  return v;
}

// Full frequency index of the first element of pair slot t (see the mid pass).
__device__ __forceinline__ int64_t slot_freq(const Geo& g, int64_t t) {
  const int64_t units1 = (int64_t)((g.N2 >> 1) - 1) << g.lgN1;
  if (t < units1) {
    const int64_t u = (t >> g.lgN1) + 1, q = t & (g.N1 - 1);
    return u + ((int64_t)q << g.lgN2);
  }
  const int64_t q = t - units1;
  if (q <= (g.N1 >> 1)) return q << g.lgN2;
  return (g.N2 >> 1) + ((q - (g.N1 >> 1) - 1) << g.lgN2);
}

// Real-FFT geometry (N = n/2), pair (k, N - k), spectrum H = chat (the C^T
// product): P = (H_k + H_{k+N}) / 2N, Q = (H_k - H_{k+N}) / 2N, theta = pi k / N,
//   a = P - Q sin(theta),  a' = conj(P + Q sin(theta)),  b = i Q cos(theta),
// all in FP64, rounded once: tabA = (a, a'), tabB = b.
__global__ void tab_ista_k(const double2* __restrict__ chat, Geo g, int64_t n, float4* __restrict__ tabA,
                           int64_t count) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int64_t k = slot_freq(g, t);
  const double2 a = chat_at(chat, n, k), b = chat_at(chat, n, k + g.N);
  const double s = 0.5 / (double)g.N;
  tabA[t] = make_float4((float)((a.x + b.x) * s), (float)((a.y + b.y) * s), (float)((a.x - b.x) * s),
                        (float)((a.y - b.y) * s));
}

// 2D: bins (k0, k1) with k0 in {0, n0/2} and k1 in {0, n1/2} are real.
__device__ __forceinline__ double2 chat2_at(const double2* chat2, int64_t n0, int64_t n1, int64_t k0, int64_t k1) {
  double2 v = chat2[k0 * n1 + k1];
  if ((k0 == 0 || k0 == (n0 >> 1)) && (k1 == 0 || k1 == (n1 >> 1))) v.y = 0.0;
  return v;
}

// 2D frequency (k2, k1) of pair slot t: rows (u, N2 - u) for units u >= 1;
// unit 0 holds rows 0 and N2/2, each with N1/2 + 1 slots (columns q and
// (N1 - q) mod N1).
__device__ __forceinline__ void slot_freq2d(const Geo& g, int64_t t, int64_t& k2, int64_t& k1) {
  const int64_t units1 = (int64_t)((g.N2 >> 1) - 1) << g.lgN1;
  if (t < units1) {
    k2 = (t >> g.lgN1) + 1;
    k1 = t & (g.N1 - 1);
    return;
  }
  const int64_t q = t - units1;
  if (q <= (g.N1 >> 1)) { k2 = 0; k1 = q; }
  else { k2 = g.N2 >> 1; k1 = q - (g.N1 >> 1) - 1; }
}

// Packed real 2D geometry (N2 = n0 rows, N1 = n1/2 packed columns): as
// tab_ista_k with H_k -> chat2[k2, k1], H_{k+N} -> chat2[k2, k1 + N1] and the
// packing phase exp(-2 pi i k1 / n1).
__global__ void tab_ista2d_k(const double2* __restrict__ chat2, Geo g, int64_t n0, int64_t n1,
                             float4* __restrict__ tabA, int64_t count) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  int64_t k2, k1;
  slot_freq2d(g, t, k2, k1);
  const double2 a = chat2_at(chat2, n0, n1, k2, k1), b = chat2_at(chat2, n0, n1, k2, k1 + g.N1);
  const double s = 0.5 / (double)g.N;
  tabA[t] = make_float4((float)((a.x + b.x) * s), (float)((a.y + b.y) * s), (float)((a.x - b.x) * s),
                        (float)((a.y - b.y) * s));
}

__global__ void tab_admm2d_k(const double2* __restrict__ chat2, Geo g, int64_t n0, int64_t n1,
                             float2* __restrict__ tabc, double* __restrict__ abs2, int64_t count) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  int64_t k2, k1;
  slot_freq2d(g, t, k2, k1);
  const double2 a = chat2_at(chat2, n0, n1, k2, k1);
  tabc[t] = make_float2((float)a.x, (float)a.y);
  abs2[t] = a.x * a.x + a.y * a.y;
}

// Complex-n geometry (N = n): chat_k in fp32 and |chat_k|^2 in FP64.
__global__ void tab_admm_k(const double2* __restrict__ chat, Geo g, int64_t n, float2* __restrict__ tabc,
                           double* __restrict__ abs2, int64_t count) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int64_t k = slot_freq(g, t);
  const double2 a = chat_at(chat, n, k);
  tabc[t] = make_float2((float)a.x, (float)a.y);
  abs2[t] = a.x * a.x + a.y * a.y;
}

// Spectrum of B = (rho C^T C + sigma I)^-1 (Algorithm 3, initial inversion),
// with the 1/n of the inverse FFT folded in; FP64, rounded once.
__global__ void tab_admm_b_k(const double* __restrict__ abs2, int64_t count, int64_t n, double rho,
                             double sigma, float* __restrict__ tabb) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  tabb[t] = (float)(1.0 / ((double)n * (rho * abs2[t] + sigma)));
}

// Tile-order position of natural index p in the column-pass layout of g:
// p = gi G + c + j2 N1  ->  t = gi (G N2) + j2 G + c.
__device__ __forceinline__ int64_t nat_to_tile(const Geo& g, int64_t p) {
  const int64_t j1 = p & (g.N1 - 1), j2 = p >> g.lgN1;
  return ((j1 >> g.lgG) << (g.lgG + g.lgN2)) + (j2 << g.lgG) + (j1 & (g.G - 1));
}
__device__ __forceinline__ int64_t tile_to_nat(const Geo& g, int64_t t) {
  const int64_t gi = t >> (g.lgG + g.lgN2), rem = t & ((int64_t(1) << (g.lgG + g.lgN2)) - 1);
  return (gi << g.lgG) + (rem & (g.G - 1)) + ((rem >> g.lgG) << g.lgN1);
}
// Bit of spatial row r in the tile-ordered row mask: in the real-FFT
// geometry rows 2p and 2p+1 share complex element p.
__device__ __forceinline__ int64_t row_bit(const Geo& g, int packed, int64_t r) {
  return packed ? 2 * nat_to_tile(g, r >> 1) + (r & 1) : nat_to_tile(g, r);
}

__global__ void build_mask_k(const int64_t* __restrict__ rows, int64_t m, int64_t n, Geo g, int packed,
                             uint32_t* mask, int* status) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int64_t r = rows[i];
  if (r < 0 || r >= n) { atomicOr(status, STS_BAD_ROW); return; }
  const int64_t b = row_bit(g, packed, r);
  const uint32_t bit = 1u << (b & 31);
  const uint32_t old = atomicOr(mask + (b >> 5), bit);
  if (old & bit) atomicOr(status, STS_DUP_ROW);
}

template <typename T>
__global__ void to_tile_k(const T* __restrict__ nat, T* __restrict__ tiled, Geo g) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < g.N) tiled[t] = nat[tile_to_nat(g, t)];
}

template <typename T>
__global__ void from_tile_k(const T* __restrict__ tiled, T* __restrict__ nat, Geo g) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < g.N) nat[tile_to_nat(g, t)] = tiled[t];
}

// The same for complex elements of a caller's float vector that starts on a
// 4-byte (not 8-byte) boundary: two 4-byte accesses per element.
__global__ void to_tile_pair_k(const float* __restrict__ nat, float2* __restrict__ tiled, Geo g) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= g.N) return;
  const int64_t p = tile_to_nat(g, t);
  tiled[t] = make_float2(nat[2 * p], nat[2 * p + 1]);
}
__global__ void from_tile_pair_k(const float2* __restrict__ tiled, float* __restrict__ nat, Geo g) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= g.N) return;
  const int64_t p = tile_to_nat(g, t);
  const float2 v = tiled[t];
  nat[2 * p] = v.x;
  nat[2 * p + 1] = v.y;
}

inline bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

// Exclusive prefix count of set bits per 32-bit word, one CTA.
__global__ void __launch_bounds__(1024) prefix_k(const uint32_t* __restrict__ mask, int64_t words,
                                                 uint32_t* __restrict__ prefix) {
  __shared__ uint32_t part[1024];
  const int64_t per = (words + 1023) / 1024;
  const int64_t lo = threadIdx.x * per, hi = min(words, lo + per);
  uint32_t s = 0;
  for (int64_t w = lo; w < hi; ++w) s += __popc(mask[w]);
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int i = 0; i < 1024; ++i) { const uint32_t v = part[i]; part[i] = acc; acc += v; }
  }
  __syncthreads();
  uint32_t acc = part[threadIdx.x];
  for (int64_t w = lo; w < hi; ++w) { prefix[w] = acc; acc += __popc(mask[w]); }
}

// pos[i] = rank of row rows[i] among the kept rows in tile order (index of
// y[i] in the compact tile-ordered y); rows32 = rows as int32.
__global__ void row_pos_k(const int64_t* __restrict__ rows, int64_t m, Geo g, int packed,
                          const uint32_t* __restrict__ mask, const uint32_t* __restrict__ prefix,
                          int32_t* __restrict__ pos, int32_t* __restrict__ rows32) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int64_t r = rows[i];
  const int64_t b = row_bit(g, packed, r);
  const uint32_t w = mask[b >> 5];
  pos[i] = (int32_t)(prefix[b >> 5] + __popc(w & ((1u << (b & 31)) - 1u)));
  if (rows32) rows32[i] = (int32_t)r;
}

__global__ void scatter_y_k(const float* __restrict__ y, const int32_t* __restrict__ pos, int64_t m,
                            float* __restrict__ ys, int* status) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const float v = y[i];
  if (!isfinite(v)) atomicOr(status, STS_NONFINITE);
  ys[pos[i]] = v;
}

__global__ void __launch_bounds__(AUX_NT) sum_scaled_k(const double* __restrict__ v, int count, float scale,
                                                       float* __restrict__ out) {
  __shared__ double red[AUX_NT];
  double s = 0.0;
  for (int b = threadIdx.x; b < count; b += AUX_NT) s += v[b];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = AUX_NT / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = (float)((double)scale * red[0]);
}

__global__ void gather_rows_k(const float* __restrict__ dense, const int32_t* __restrict__ rows32, int64_t m,
                              float* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < m) y[i] = dense[rows32[i]];
}

__global__ void scatter_rows_k(const float* __restrict__ r, const int32_t* __restrict__ rows32, int64_t m,
                               float* __restrict__ dense) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < m) dense[rows32[i]] = r[i];
}

constexpr int NORM_BLOCKS = 256;

__global__ void __launch_bounds__(AUX_NT) norm2_part_k(const float* __restrict__ x, int64_t n,
                                                       double* __restrict__ partials) {
  __shared__ double red[AUX_NT];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)AUX_NT + threadIdx.x; i < n; i += (int64_t)NORM_BLOCKS * AUX_NT) {
    const double v = x[i];
    s += v * v;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = AUX_NT / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void norm2_final_k(const double* __restrict__ partials, double* out) {
  __shared__ double red[NORM_BLOCKS];
  red[threadIdx.x] = partials[threadIdx.x];
  __syncthreads();
  for (int w = NORM_BLOCKS / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// Fixed start vector for the power iteration: a 32-bit integer hash of the
// index mapped to [-1, 1).
__global__ void power_init_k(float* u, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t h = (uint32_t)i * 2654435761u + 0x9e3779b9u;
  h ^= h >> 16; h *= 0x85ebca6bu; h ^= h >> 13; h *= 0xc2b2ae35u; h ^= h >> 16;
  u[i] = (float)((double)h * (2.0 / 4294967296.0) - 1.0);
}

inline unsigned blocks_for(int64_t count) { return (unsigned)((count + AUX_NT - 1) / AUX_NT); }

}  // namespace

cudaError_t launch_set_args(const CallArgs& a, CallArgs* dst, cudaStream_t s) {
  set_args_k<<<1, 1, 0, s>>>(a, dst);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const double* partials, int nblk, double* stats, cudaStream_t s) {
  finalize_k<<<1, AUX_NT, 0, s>>>(partials, nblk, stats);
  return cudaGetLastError();
}

cudaError_t launch_twiddle(float2* dst, int count, int64_t M, cudaStream_t s) {
  twiddle_k<<<blocks_for(count), AUX_NT, 0, s>>>(dst, count, M);
  return cudaGetLastError();
}

cudaError_t launch_fft64(const double* c, double2* a, double2* b, int64_t n, double2** out,
                         cudaStream_t s) {
  c_to_complex_k<<<blocks_for(n), AUX_NT, 0, s>>>(c, a, n);
  double2* in = a;
  double2* o = b;
  for (int64_t Ls = 1; Ls < n; Ls <<= 1) {
    fft64_stage_k<<<blocks_for(n >> 1), AUX_NT, 0, s>>>(in, o, n, Ls);
    double2* t = in; in = o; o = t;
  }
  *out = in;
  return cudaGetLastError();
}

cudaError_t launch_fft64_2d(const double* c2, double2* a, double2* b, int64_t n0, int64_t n1, double2** out,
                            cudaStream_t s) {
  const int64_t n = n0 * n1;
  c_to_complex_k<<<blocks_for(n), AUX_NT, 0, s>>>(c2, a, n);
  double2* in = a;
  double2* o = b;
  for (int64_t Ls = 1; Ls < n1; Ls <<= 1) {   // rows
    fft64_strided_stage_k<<<blocks_for(n >> 1), AUX_NT, 0, s>>>(in, o, n1, Ls, n0, 1, n1);
    double2* t = in; in = o; o = t;
  }
  for (int64_t Ls = 1; Ls < n0; Ls <<= 1) {   // columns
    fft64_strided_stage_k<<<blocks_for(n >> 1), AUX_NT, 0, s>>>(in, o, n0, Ls, n1, n1, 1);
    double2* t = in; in = o; o = t;
  }
  *out = in;
  return cudaGetLastError();
}

cudaError_t launch_tab_ista2d(const double2* chat2, const Geo& g, int64_t n0, int64_t n1, float4* tabA,
                              cudaStream_t s) {
  const int64_t cnt = tab_count(g);
  tab_ista2d_k<<<blocks_for(cnt), AUX_NT, 0, s>>>(chat2, g, n0, n1, tabA, cnt);
  return cudaGetLastError();
}

cudaError_t launch_tab_admm2d(const double2* chat2, const Geo& g, int64_t n0, int64_t n1, float2* tabc,
                              double* abs2, cudaStream_t s) {
  const int64_t cnt = tab_count(g);
  tab_admm2d_k<<<blocks_for(cnt), AUX_NT, 0, s>>>(chat2, g, n0, n1, tabc, abs2, cnt);
  return cudaGetLastError();
}

cudaError_t launch_fft64_complex(double2* a, double2* b, int64_t n, double2** out, cudaStream_t s) {
  double2* in = a;
  double2* o = b;
  for (int64_t Ls = 1; Ls < n; Ls <<= 1) {
    fft64_stage_k<<<blocks_for(n >> 1), AUX_NT, 0, s>>>(in, o, n, Ls);
    double2* t = in; in = o; o = t;
  }
  *out = in;
  return cudaGetLastError();
}


cudaError_t launch_tab_ista(const double2* chat, const Geo& g, int64_t n, float4* tabA, cudaStream_t s) {
  const int64_t cnt = tab_count(g);
  tab_ista_k<<<blocks_for(cnt), AUX_NT, 0, s>>>(chat, g, n, tabA, cnt);
  return cudaGetLastError();
}

cudaError_t launch_stage_tw(float2* dst, int lgL, int count, cudaStream_t s) {
  if (count > 0) stage_tw_k<<<blocks_for(count), AUX_NT, 0, s>>>(dst, lgL, count);
  return cudaGetLastError();
}

cudaError_t launch_tab_admm(const double2* chat, const Geo& g, int64_t n, float2* tabc, double* abs2,
                            cudaStream_t s) {
  const int64_t cnt = tab_count(g);
  tab_admm_k<<<blocks_for(cnt), AUX_NT, 0, s>>>(chat, g, n, tabc, abs2, cnt);
  return cudaGetLastError();
}

cudaError_t launch_tab_admm_b(const double* abs2, int count, int64_t n, double rho, double sigma,
                              float* tabb, cudaStream_t s) {
  tab_admm_b_k<<<blocks_for(count), AUX_NT, 0, s>>>(abs2, count, n, rho, sigma, tabb);
  return cudaGetLastError();
}

cudaError_t launch_build_mask(const int64_t* rows, int64_t m, int64_t n, const Geo& g, int packed,
                              uint32_t* mask, int* status, cudaStream_t s) {
  build_mask_k<<<blocks_for(m), AUX_NT, 0, s>>>(rows, m, n, g, packed, mask, status);
  return cudaGetLastError();
}

cudaError_t launch_to_tile(const void* nat, void* tiled, const Geo& g, int complex_elems, cudaStream_t s) {
  if (complex_elems && !aligned8(nat))
    to_tile_pair_k<<<blocks_for(g.N), AUX_NT, 0, s>>>((const float*)nat, (float2*)tiled, g);
  else if (complex_elems)
    to_tile_k<float2><<<blocks_for(g.N), AUX_NT, 0, s>>>((const float2*)nat, (float2*)tiled, g);
  else
    to_tile_k<float><<<blocks_for(g.N), AUX_NT, 0, s>>>((const float*)nat, (float*)tiled, g);
  return cudaGetLastError();
}

cudaError_t launch_from_tile(const void* tiled, void* nat, const Geo& g, int complex_elems, cudaStream_t s) {
  if (complex_elems && !aligned8(nat))
    from_tile_pair_k<<<blocks_for(g.N), AUX_NT, 0, s>>>((const float2*)tiled, (float*)nat, g);
  else if (complex_elems)
    from_tile_k<float2><<<blocks_for(g.N), AUX_NT, 0, s>>>((const float2*)tiled, (float2*)nat, g);
  else
    from_tile_k<float><<<blocks_for(g.N), AUX_NT, 0, s>>>((const float*)tiled, (float*)nat, g);
  return cudaGetLastError();
}

// ---- grouped element-wise kernels (blockIdx.y: the plan, grid-stride in x)

__global__ void group_scatter_y_k(const GroupDesc* __restrict__ d, const float* __restrict__ y, int geo,
                                  int* status) {
  const GroupDesc& g = d[blockIdx.y];
  const int32_t* pos = geo ? g.pos_a : g.pos_i;
  float* ys = geo ? g.ys_a : g.ys_i;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < g.m; r += (int64_t)gridDim.x * blockDim.x) {
    const float v = y[g.moff + r];
    if (!isfinite(v)) atomicOr(status, STS_NONFINITE);
    ys[pos[r]] = v;
  }
}

template <bool IN>
__global__ void group_ista_k(const GroupDesc* __restrict__ d, float* x) {
  const GroupDesc& g = d[blockIdx.y];
  float* xn = x + g.noff;   // 4-byte aligned only: the concatenation may hold odd-length instances
  float2* xt = reinterpret_cast<float2*>(g.xi_t);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < g.gi.N; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = tile_to_nat(g.gi, t);
    if (IN) {
      xt[t] = make_float2(xn[2 * p], xn[2 * p + 1]);
    } else {
      const float2 v = xt[t];
      xn[2 * p] = v.x;
      xn[2 * p + 1] = v.y;
    }
  }
}

__global__ void group_admm_zero_k(const GroupDesc* __restrict__ d) {
  const GroupDesc& g = d[blockIdx.y];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < g.ga.N; t += (int64_t)gridDim.x * blockDim.x) {
    g.av[t] = 0.f;
    g.az[t] = 0.f;
    g.amu[t] = 0.f;
    g.anu[t] = 0.f;
  }
}

__global__ void group_admm_out_k(const GroupDesc* __restrict__ d, float* z) {
  const GroupDesc& g = d[blockIdx.y];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < g.ga.N; t += (int64_t)gridDim.x * blockDim.x)
    z[g.noff + tile_to_nat(g.ga, t)] = g.az[t];
}

constexpr unsigned GROUP_GX = 32;   // CTAs per plan in the grouped element-wise kernels

cudaError_t launch_group_scatter_y(const GroupDesc* d, int count, const float* y, int geo, int* status,
                                   cudaStream_t s) {
  if (count < 1) return cudaSuccess;
  group_scatter_y_k<<<dim3(GROUP_GX, count), AUX_NT, 0, s>>>(d, y, geo, status);
  return cudaGetLastError();
}

cudaError_t launch_group_ista_in(const GroupDesc* d, int count, const float* x, cudaStream_t s) {
  if (count < 1) return cudaSuccess;
  group_ista_k<true><<<dim3(GROUP_GX, count), AUX_NT, 0, s>>>(d, const_cast<float*>(x));
  return cudaGetLastError();
}

cudaError_t launch_group_ista_out(const GroupDesc* d, int count, float* x, cudaStream_t s) {
  if (count < 1) return cudaSuccess;
  group_ista_k<false><<<dim3(GROUP_GX, count), AUX_NT, 0, s>>>(d, x);
  return cudaGetLastError();
}

cudaError_t launch_group_admm_zero(const GroupDesc* d, int count, cudaStream_t s) {
  if (count < 1) return cudaSuccess;
  group_admm_zero_k<<<dim3(GROUP_GX, count), AUX_NT, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_group_admm_out(const GroupDesc* d, int count, float* z, cudaStream_t s) {
  if (count < 1) return cudaSuccess;
  group_admm_out_k<<<dim3(GROUP_GX, count), AUX_NT, 0, s>>>(d, z);
  return cudaGetLastError();
}

cudaError_t launch_prefix(const uint32_t* mask, int64_t words, uint32_t* prefix, cudaStream_t s) {
  prefix_k<<<1, 1024, 0, s>>>(mask, words, prefix);
  return cudaGetLastError();
}

cudaError_t launch_row_pos(const int64_t* rows, int64_t m, const Geo& g, int packed, const uint32_t* mask,
                           const uint32_t* prefix, int32_t* pos, int32_t* rows32, cudaStream_t s) {
  row_pos_k<<<blocks_for(m), AUX_NT, 0, s>>>(rows, m, g, packed, mask, prefix, pos, rows32);
  return cudaGetLastError();
}

cudaError_t launch_scatter_y(const float* y, const int32_t* pos, int64_t m, float* ys, int* status,
                             cudaStream_t s) {
  scatter_y_k<<<blocks_for(m), AUX_NT, 0, s>>>(y, pos, m, ys, status);
  return cudaGetLastError();
}

cudaError_t launch_sum_scaled(const double* v, int count, float scale, float* out, cudaStream_t s) {
  sum_scaled_k<<<1, AUX_NT, 0, s>>>(v, count, scale, out);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(const float* dense, const int32_t* rows32, int64_t m, float* y,
                               cudaStream_t s) {
  gather_rows_k<<<blocks_for(m), AUX_NT, 0, s>>>(dense, rows32, m, y);
  return cudaGetLastError();
}

cudaError_t launch_scatter_rows(const float* r, const int32_t* rows32, int64_t m, float* dense,
                                cudaStream_t s) {
  scatter_rows_k<<<blocks_for(m), AUX_NT, 0, s>>>(r, rows32, m, dense);
  return cudaGetLastError();
}

cudaError_t launch_norm2(const float* x, int64_t n, double* partials, double* out, cudaStream_t s) {
  norm2_part_k<<<NORM_BLOCKS, AUX_NT, 0, s>>>(x, n, partials);
  norm2_final_k<<<1, NORM_BLOCKS, 0, s>>>(partials, out);
  return cudaGetLastError();
}

cudaError_t launch_power_init(float* u, int64_t n, cudaStream_t s) {
  power_init_k<<<blocks_for(n), AUX_NT, 0, s>>>(u, n);
  return cudaGetLastError();
}

}  // namespace csk
