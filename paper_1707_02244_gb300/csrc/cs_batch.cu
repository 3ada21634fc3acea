// Batched solver: many independent instances A_i = P_i C(c_i) of uneven size.
// Every instance with n <= CS_BATCH_MAX_N is solved by one CTA that keeps its
// iterate in shared memory for all iterations (no global exchange at all: the
// whole FFT of the instance fits in the CTA); CTAs are ordered largest
// instance first, one launch per power-of-two size class.  Larger instances
// have their own plan's buffers and tables but are iterated together: each
// pass of an iteration is one grouped launch over the tiles of all of them
// (col_kernel_multi / mid_kernel_multi), so a whole solve of every large
// instance is one captured CUDA graph on the batch's stream, ordered by the
// kernel boundaries alone.  Instances whose n is 7-smooth but not a power of
// two go to the mixed-radix solver of cs_smooth.cu (one persistent launch per
// solve over all of them).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/cs.h"
#include "cs_fft.cuh"
#include "cs_internal.h"

namespace csk {
namespace {

constexpr int LG_TW = 13;       // master twiddle table exp(-2 pi i q / 8192)
constexpr int BI_LG_MIN = 5, BI_LG_MAX = 12;   // ISTA: packed length N = n/2 = 2^LG
constexpr int BA_LG_MIN = 6, BA_LG_MAX = 13;   // ADMM: complex length n = 2^LG
constexpr int NSIDE_MAX = 4;    // side streams of the size-class launches (within CUDA's default 8 queues)

struct BatchDesc {
  int n, lgn, m;
  int pad0;
  int64_t noff;   // offset of x / z / state in the concatenated n-vectors
  int64_t moff;   // offset of y in the concatenated m-vectors
  int64_t woff;   // offset of the row-mask words
  int64_t itab;   // ISTA table offset (n/4 + 1 entries)
  int64_t atab;   // ADMM table offset (n/2 + 1 entries)
};

struct BatchScalars {   // per call
  float thr, tau, rho, sigma, tau1, tau2, d_on, d_off;
};

__device__ __forceinline__ float soft(float u, float g) { return u > g ? u - g : (u < -g ? u + g : 0.f); }

// Packed real-FFT spectrum operator of one instance (as in the mid pass,
// with the pair (k, N - k) of a single vector).
template <bool ADJ>
__device__ __forceinline__ void pair_real(const float4 t, float2 be, float2& za, float2& zb) {
  float2 al = make_float2(t.x, t.y), al2 = make_float2(t.z, t.w);
  float2 be2 = make_float2(-be.x, be.y);
  if (!ADJ) {
    al = cconj(al);
    al2 = cconj(al2);
    const float2 tb = be;
    be = make_float2(-tb.x, tb.y);
    be2 = tb;
  }
  const float2 a2 = za, b2 = zb;
  za = cadd(cmul(al, a2), cmul(be, cconj(b2)));
  zb = cadd(cmul(al2, b2), cmul(be2, cconj(a2)));
}

// One FFT of the instance's vector (length 2^LG, one CTA of 2^LG / 16
// threads) in shared memory; the shape is fixed at compile time so every
// address of a stage is a base plus an immediate.
template <int DIR, int LG>
__device__ __forceinline__ void fft_vec(float2* S, const float2* __restrict__ tw) {
  constexpr int L = 1 << LG;
  const StaticLayout<LG, 0, false> lay;
  tile_fft<DIR, L, L / EPT>(S, lay, tw, LG_TW);
}

template <bool ADJ, int N, int NT>
__device__ __forceinline__ void pair_pass(float2* S, const float4* __restrict__ tA, const float2* __restrict__ tB) {
  for (int k = threadIdx.x; k <= (N >> 1); k += NT) {
    const int kp = (N - k) & (N - 1);
    float2 za = S[pad(k)], zb = S[pad(kp)];
    pair_real<ADJ>(__ldg(tA + k), __ldg(tB + k), za, zb);
    S[pad(kp)] = zb;   // self-pairs keep the k-side value
    S[pad(k)] = za;
  }
  __syncthreads();
}

// One CTA solves instance order[blockIdx.x] (n = 2^(LG+1)) for `iters` ISTA
// iterations (Algorithm 1, threshold tau * lambda):
//   x <- eta(x + tau C^T M (y~ - C x)).
template <int LG>
__global__ void __launch_bounds__((1 << LG) / EPT) batch_ista_k(
    const BatchDesc* __restrict__ descs, const BatchScalars* __restrict__ sc, const int* __restrict__ order,
    const float4* __restrict__ tA, const float2* __restrict__ tB, const uint32_t* __restrict__ mask,
    const uint32_t* __restrict__ prefix, const float* __restrict__ ys, const float2* __restrict__ tw,
    float* __restrict__ x, int iters) {
  constexpr int N = 1 << LG, NT = N / EPT;
  extern __shared__ float2 sm[];
  float2* S = sm;
  float2* X = sm + smem_slots(N);
  const int id = order[blockIdx.x];
  const BatchDesc d = descs[id];
  const BatchScalars s = sc[id];
  float* xg = x + d.noff;   // 4-byte aligned only: the concatenation may hold odd-length instances
  const uint32_t* mk = mask + d.woff;
  const uint32_t* pf = prefix + d.woff;
  const float* yv = ys + d.moff;
  const float4* tAi = tA + d.itab;
  const float2* tBi = tB + d.itab;
  for (int p = threadIdx.x; p < N; p += NT) {
    const float2 v = make_float2(xg[2 * p], xg[2 * p + 1]);
    X[p] = v;
    S[pad(p)] = v;
  }
  __syncthreads();
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
    fft_vec<-1, LG>(S, tw);
    pair_pass<false, N, NT>(S, tAi, tBi);
    fft_vec<+1, LG>(S, tw);
    // r~ = M (y~ - C x) on rows 2p, 2p+1
    for (int p = threadIdx.x; p < N; p += NT) {
      const uint32_t w = mk[p >> 4];
      const int b = (2 * p) & 31;
      const int i0 = (int)pf[p >> 4] + __popc(w & ((1u << b) - 1u));
      const uint32_t mm = (w >> b) & 3u;
      const float2 v = S[pad(p)];
      S[pad(p)] = make_float2((mm & 1u) ? yv[i0] - v.x : 0.f, (mm & 2u) ? yv[i0 + (int)(mm & 1u)] - v.y : 0.f);
    }
    __syncthreads();
    fft_vec<-1, LG>(S, tw);
    pair_pass<true, N, NT>(S, tAi, tBi);
    fft_vec<+1, LG>(S, tw);
    for (int p = threadIdx.x; p < N; p += NT) {
      const float2 g = S[pad(p)], xo = X[p];
      const float2 xn = make_float2(soft(fmaf(s.tau, g.x, xo.x), s.thr), soft(fmaf(s.tau, g.y, xo.y), s.thr));
      X[p] = xn;
      S[pad(p)] = xn;
    }
    __syncthreads();
  }
  for (int p = threadIdx.x; p < N; p += NT) {
    xg[2 * p] = X[p].x;
    xg[2 * p + 1] = X[p].y;
  }
}

// One CTA solves instance order[blockIdx.x] (n = 2^LG) for `iters`
// iterations of Algorithm 3 from the zero state.  The complex-n FFT of
// (v + mu) + i (z - nu) lives in shared memory; mu and nu in global memory
// (the instance's slice).
template <int LG>
__global__ void __launch_bounds__((1 << LG) / EPT) batch_admm_k(
    const BatchDesc* __restrict__ descs, const BatchScalars* __restrict__ sc, const int* __restrict__ order,
    const float2* __restrict__ tc, const float* __restrict__ tb, const uint32_t* __restrict__ mask,
    const uint32_t* __restrict__ prefix, const float* __restrict__ ys, const float2* __restrict__ tw,
    float* __restrict__ z, float* __restrict__ mu, float* __restrict__ nu, int iters) {
  constexpr int n = 1 << LG, NT = n / EPT;
  extern __shared__ float2 sm[];
  float2* S = sm;
  const int id = order[blockIdx.x];
  const BatchDesc d = descs[id];
  const BatchScalars s = sc[id];
  float* zi = z + d.noff;
  float* mui = mu + d.noff;
  float* nui = nu + d.noff;
  const uint32_t* mk = mask + d.woff;
  const uint32_t* pf = prefix + d.woff;
  const float* yv = ys + d.moff;
  const float2* tci = tc + d.atab;
  const float* tbi = tb + d.atab;
  for (int p = threadIdx.x; p < n; p += NT) {
    mui[p] = 0.f;
    nui[p] = 0.f;
    S[pad(p)] = make_float2(0.f, 0.f);
  }
  __syncthreads();
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
    fft_vec<-1, LG>(S, tw);
    // x-update spectrum (Algorithm 3) for every pair (k, n - k):
    //   V = (Z_k + conj Z_{n-k}) / 2, W = (Z_k - conj Z_{n-k}) / 2i,
    //   X = bhat (rho chat V + sigma W) / n, then X + i conj(chat) X
    for (int k = threadIdx.x; k <= (n >> 1); k += NT) {
      const int kp = (n - k) & (n - 1);
      const float2 za = S[pad(k)], zb = S[pad(kp)];
      const float2 ch = __ldg(tci + k);
      const float bb = __ldg(tbi + k);
      const float2 V = make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y - zb.y));
      const float2 Wk = make_float2(0.5f * (za.y + zb.y), -0.5f * (za.x - zb.x));
      const float2 cv = cmul(ch, V);
      const float2 X = make_float2(bb * fmaf(s.rho, cv.x, s.sigma * Wk.x), bb * fmaf(s.rho, cv.y, s.sigma * Wk.y));
      const float2 Pc = cmulc(X, ch);
      S[pad(kp)] = make_float2(X.x + Pc.y, Pc.x - X.y);
      S[pad(k)] = make_float2(X.x - Pc.y, X.y + Pc.x);
    }
    __syncthreads();
    fft_vec<+1, LG>(S, tw);
    const bool last = it == iters - 1;
    for (int p = threadIdx.x; p < n; p += NT) {
      const uint32_t w = mk[p >> 5];
      const int b = p & 31;
      const bool on = (w >> b) & 1u;
      const float yvv = on ? yv[pf[p >> 5] + __popc(w & ((1u << b) - 1u))] : 0.f;
      const float2 xc = S[pad(p)];
      const float xx = xc.x, cx = xc.y;
      const float m0 = mui[p], n0 = nui[p];
      const float vv = (on ? s.d_on : s.d_off) * fmaf(s.rho, cx - m0, yvv);
      const float zz = soft(xx + n0, s.thr);
      const float m2 = fmaf(s.tau1, vv - cx, m0);
      const float n2 = fmaf(s.tau2, xx - zz, n0);
      mui[p] = m2;
      nui[p] = n2;
      if (last) zi[p] = zz;
      S[pad(p)] = make_float2(vv + m2, zz - n2);
    }
    __syncthreads();
  }
}

template <int LG>
size_t ista_smem() { return sizeof(float2) * (smem_slots(1 << LG) + (1 << LG)); }
template <int LG>
size_t admm_smem() { return sizeof(float2) * smem_slots(1 << LG); }

// Per size class: the kernel instantiation and its launch shape.
struct ClassKernel {
  const void* fn;
  unsigned nt;
  size_t smem;
};

template <int LG>
ClassKernel ista_kernel() { return {reinterpret_cast<const void*>(&batch_ista_k<LG>), (1u << LG) / EPT, ista_smem<LG>()}; }
template <int LG>
ClassKernel admm_kernel() { return {reinterpret_cast<const void*>(&batch_admm_k<LG>), (1u << LG) / EPT, admm_smem<LG>()}; }

ClassKernel ista_class(int lg) {
  switch (lg) {
    case 5: return ista_kernel<5>();
    case 6: return ista_kernel<6>();
    case 7: return ista_kernel<7>();
    case 8: return ista_kernel<8>();
    case 9: return ista_kernel<9>();
    case 10: return ista_kernel<10>();
    case 11: return ista_kernel<11>();
    default: return ista_kernel<12>();
  }
}

ClassKernel admm_class(int lg) {
  switch (lg) {
    case 6: return admm_kernel<6>();
    case 7: return admm_kernel<7>();
    case 8: return admm_kernel<8>();
    case 9: return admm_kernel<9>();
    case 10: return admm_kernel<10>();
    case 11: return admm_kernel<11>();
    case 12: return admm_kernel<12>();
    default: return admm_kernel<13>();
  }
}

// ---------------------------------------------------------------- plan time

__global__ void tab_ista1_k(const double2* __restrict__ chat, int64_t n, float4* __restrict__ tA,
                            float2* __restrict__ tB) {
  // single-vector packed geometry: N = n/2, pairs (k, N - k) for k in [0, N/2]
  const int64_t N = n >> 1;
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k > (N >> 1)) return;
  double2 a = chat[k], b = chat[k + N];
  if (k == 0) { a.y = 0.0; b.y = 0.0; }
  const double s = 0.5 / (double)N;
  const double Px = (a.x + b.x) * s, Py = (a.y + b.y) * s, Qx = (a.x - b.x) * s, Qy = (a.y - b.y) * s;
  double sn, cs;
  sincospi((double)k / (double)N, &sn, &cs);
  tA[k] = make_float4((float)(Px - Qx * sn), (float)(Py - Qy * sn), (float)(Px + Qx * sn), (float)(-(Py + Qy * sn)));
  tB[k] = make_float2((float)(-Qy * cs), (float)(Qx * cs));
}

__global__ void tab_admm1_k(const double2* __restrict__ chat, int64_t n, float2* __restrict__ tc,
                            double* __restrict__ abs2) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k > (n >> 1)) return;
  double2 a = chat[k];
  if (k == 0 || k == (n >> 1)) a.y = 0.0;
  tc[k] = make_float2((float)a.x, (float)a.y);
  abs2[k] = a.x * a.x + a.y * a.y;
}

__global__ void tab_admm1_b_k(const double* __restrict__ abs2, int64_t count, const int* __restrict__ inst,
                              const BatchDesc* __restrict__ descs, const double* __restrict__ rho,
                              const double* __restrict__ sigma, float* __restrict__ tb) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int i = inst[t];
  tb[t] = (float)(1.0 / ((double)descs[i].n * (rho[i] * abs2[t] + sigma[i])));
}

__global__ void batch_mask_k(const int64_t* __restrict__ rows, int64_t m, int64_t n, uint32_t* mask,
                             int* status) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int64_t r = rows[i];
  if (r < 0 || r >= n) { atomicOr(status, STS_BAD_ROW); return; }
  const uint32_t bit = 1u << (r & 31);
  if (atomicOr(mask + (r >> 5), bit) & bit) atomicOr(status, STS_DUP_ROW);
}

__global__ void batch_pos_k(const int64_t* __restrict__ rows, int64_t m, const uint32_t* __restrict__ mask,
                            const uint32_t* __restrict__ prefix, int64_t moff, int32_t* __restrict__ pos) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int64_t r = rows[i];
  const uint32_t w = mask[r >> 5];
  pos[i] = (int32_t)(moff + prefix[r >> 5] + __popc(w & ((1u << (r & 31)) - 1u)));
}

// pos < 0 marks measurements of instances solved by their own plan
__global__ void batch_scatter_k(const float* __restrict__ y, const int32_t* __restrict__ pos, int64_t count,
                                float* __restrict__ ys, int* status) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int32_t q = pos[i];
  if (q < 0) return;
  const float v = y[i];
  if (!isfinite(v)) atomicOr(status, STS_NONFINITE);
  ys[q] = v;
}

inline unsigned nb256(int64_t c) { return (unsigned)((c + 255) / 256); }

}  // namespace
}  // namespace csk

using namespace csk;

struct cs_batch_s {
  int count = 0;
  cudaStream_t stream = nullptr;
  std::vector<int64_t> n, m, noff, moff;
  std::vector<int> small;           // instances solved by the single-CTA kernels, largest first
  std::vector<int> large;           // instances solved by their own plan
  std::vector<int> smooth_ids;      // 7-smooth, not power-of-two n: the mixed-radix solver
  SmoothSet* smooth = nullptr;
  std::vector<cs_plan_t> plans;     // per large instance
  // grouped launches over the large instances (in the order of `large`)
  struct Group {
    int count = 0;
    std::vector<GroupDesc> hdesc;
    GroupDesc* desc = nullptr;
    KParams *kps_i = nullptr, *kps_a0 = nullptr, *kps_a1 = nullptr;
    CallArgs* ca = nullptr;
    int2 *map_col_i = nullptr, *map_mid_i = nullptr, *map_col_a = nullptr, *map_mid_a = nullptr;
    int n_col_i = 0, n_mid_i = 0, n_col_a = 0, n_mid_a = 0;
    cudaStream_t cap = nullptr;
    std::map<uint64_t, cudaGraphExec_t> graphs;
  } grp;
  struct Class {
    int lgn, start, count, side;    // instances order[start, start + count) have n = 2^lgn
  };
  std::vector<Class> classes;
  int nside = NSIDE_MAX;
  cudaStream_t side[NSIDE_MAX] = {};
  cudaEvent_t side_done[NSIDE_MAX] = {};
  cudaEvent_t fork = nullptr;
  BatchDesc* descs = nullptr;
  BatchScalars* sc = nullptr;
  int* order = nullptr;
  float4* tA = nullptr;
  float2* tB = nullptr;
  float2* tc = nullptr;
  double* abs2 = nullptr;
  float* tb = nullptr;
  int* tb_inst = nullptr;           // instance of every ADMM table entry
  double* drho = nullptr;
  double* dsigma = nullptr;
  uint32_t* mask = nullptr;
  uint32_t* prefix = nullptr;
  int32_t* pos = nullptr;
  float* ys = nullptr;
  float2* tw = nullptr;
  float *amu = nullptr, *anu = nullptr;
  int* status = nullptr;
  int64_t ntot = 0, mtot = 0, atab_tot = 0;
  std::vector<double> host_rho, host_sigma;
};

namespace {

void batch_free(cs_batch_s* b) {
  if (!b) return;
  for (cs_plan_t p : b->plans)
    if (p) cs_plan_destroy(p);
  smooth_free(b->smooth);
  void* bufs[] = {b->descs, b->sc,   b->order,  b->tA,  b->tB, b->tc, b->abs2, b->tb,  b->tb_inst,
                  b->drho,  b->dsigma, b->mask, b->prefix, b->pos, b->ys, b->tw, b->amu, b->anu, b->status};
  for (void* q : bufs)
    if (q) cudaFree(q);
  for (int k = 0; k < NSIDE_MAX; ++k) {
    if (b->side[k]) cudaStreamDestroy(b->side[k]);
    if (b->side_done[k]) cudaEventDestroy(b->side_done[k]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  auto& G = b->grp;
  for (auto& kv : G.graphs) cudaGraphExecDestroy(kv.second);
  void* gb[] = {G.desc, G.kps_i, G.kps_a0, G.kps_a1, G.ca, G.map_col_i, G.map_mid_i, G.map_col_a, G.map_mid_a};
  for (void* q : gb)
    if (q) cudaFree(q);
  if (G.cap) cudaStreamDestroy(G.cap);
  delete b;
}

template <typename T>
cudaError_t balloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), (count ? count : 1) * sizeof(T) + 256);
}

cs_status cstat(cudaError_t e) {
  return e == cudaSuccess ? CS_OK : (e == cudaErrorMemoryAllocation ? CS_ERR_NOMEM : CS_ERR_CUDA);
}

bool pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

int ilog2(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l;
}

// Side streams wait for the work already on the batch's stream ...
cudaError_t fork_sides(cs_batch_s* b) {
  cudaError_t e = cudaEventRecord(b->fork, b->stream);
  for (int k = 0; k < b->nside && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->side[k], b->fork, 0);
  return e;
}

// ... and the batch's stream waits for all of theirs.
cudaError_t join_sides(cs_batch_s* b) {
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < b->nside && e == cudaSuccess; ++k) {
    e = cudaEventRecord(b->side_done[k], b->side[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->side_done[k], 0);
  }
  return e;
}

// Run `enqueue` on the batch's stream as a cached CUDA graph under `key`.
template <class F>
cudaError_t run_group_graph(cs_batch_s* b, uint64_t key, F&& enqueue) {
  auto& G = b->grp;
  auto it = G.graphs.find(key);
  if (it == G.graphs.end()) {
    cudaError_t e = cudaStreamBeginCapture(G.cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t e2 = enqueue(G.cap);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(G.cap, &graph);
    if (e2 != cudaSuccess || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return e2 != cudaSuccess ? e2 : e;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    it = G.graphs.emplace(key, exec).first;
  }
  return cudaGraphLaunch(it->second, b->stream);
}

// T iterations of Algorithm 1 on every large instance: per iteration four
// grouped passes (C x, residual, C^T r, update), each over the tiles of all
// of them.
cudaError_t enqueue_group_ista(cs_batch_s* b, int T, cudaStream_t s) {
  auto& G = b->grp;
  cudaError_t e = launch_col_multi(COL_LOAD, G.kps_i, G.map_col_i, G.n_col_i, s);
  for (int t = 0; t < T && e == cudaSuccess; ++t) {
    e = launch_mid_multi(MID_FWD, G.kps_i, G.map_mid_i, G.n_mid_i, s);
    if (e == cudaSuccess) e = launch_col_multi(COL_RESIDUAL, G.kps_i, G.map_col_i, G.n_col_i, s);
    if (e == cudaSuccess) e = launch_mid_multi(MID_ADJ, G.kps_i, G.map_mid_i, G.n_mid_i, s);
    if (e == cudaSuccess)
      e = launch_col_multi(t + 1 < T ? COL_ISTA : COL_ISTA_LAST, G.kps_i, G.map_col_i, G.n_col_i, s);
  }
  return e;
}

// T iterations of Algorithm 3 on every large instance: per iteration the
// grouped x-update (mid pass) and elementwise steps (column pass); the last
// one writes z.
cudaError_t enqueue_group_admm(cs_batch_s* b, int T, cudaStream_t s) {
  auto& G = b->grp;
  cudaError_t e = launch_col_multi(COL_ADMM_INIT, G.kps_a0, G.map_col_a, G.n_col_a, s);
  for (int t = 0; t < T && e == cudaSuccess; ++t) {
    e = launch_mid_multi(MID_ADMM, G.kps_a0, G.map_mid_a, G.n_mid_a, s);
    if (e == cudaSuccess) {
      const bool last = t + 1 == T;
      e = launch_col_multi(last ? COL_ADMM_LAST : COL_ADMM, last ? G.kps_a1 : G.kps_a0,
                           G.map_col_a, G.n_col_a, s);
    }
  }
  return e;
}

}  // namespace

extern "C" {

cs_status cs_batch_plan(cs_batch_t* out, int count, const int64_t* n, const int64_t* m, const int64_t* rows,
                        const double* c, void* stream) {
  if (!out || count < 1 || !n || !m || !rows || !c) return CS_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    const bool p2 = pow2(n[i]) && n[i] >= 64 && n[i] <= (int64_t(1) << 21);
    if (!p2 && !smooth_size(n[i])) return CS_ERR_UNSUPPORTED;
    if (m[i] < 1 || m[i] > n[i]) return CS_ERR_ARG;
  }
  cs_batch_s* b = new (std::nothrow) cs_batch_s();
  if (!b) return CS_ERR_NOMEM;
  b->count = count;
  b->stream = static_cast<cudaStream_t>(stream);

  cudaStream_t s = b->stream;
  b->n.assign(n, n + count);
  b->m.assign(m, m + count);
  b->noff.resize(count);
  b->moff.resize(count);
  std::vector<BatchDesc> hd(count);
  int64_t no = 0, mo = 0, wo = 0, it = 0, at = 0;
  for (int i = 0; i < count; ++i) {
    b->noff[i] = no;
    b->moff[i] = mo;
    BatchDesc& d = hd[i];
    d.n = (int)n[i];
    d.lgn = ilog2(n[i]);
    d.m = (int)m[i];
    d.pad0 = 0;
    d.noff = no;
    d.moff = mo;
    d.woff = wo;
    d.itab = it;
    d.atab = at;
    no += n[i];
    mo += m[i];
    if (!pow2(n[i])) {
      b->smooth_ids.push_back(i);
    } else if (n[i] <= CS_BATCH_MAX_N) {
      b->small.push_back(i);
      wo += n[i] / 32;
      it += n[i] / 4 + 1;
      at += n[i] / 2 + 1;
    } else {
      b->large.push_back(i);
    }
  }
  b->ntot = no;
  b->mtot = mo;
  b->atab_tot = at;
  std::stable_sort(b->small.begin(), b->small.end(), [&](int a, int c2) { return n[a] > n[c2]; });
  std::stable_sort(b->large.begin(), b->large.end(), [&](int a, int c2) { return n[a] > n[c2]; });
  // The size-class launches of the small instances go to the side streams
  // longest first, each to the stream with the least work so far (cost ~ n
  // per iteration; a class runs its instances side by side, about 2 * 152 at
  // a time); the grouped launches of the large instances run on the batch's
  // stream.
  for (size_t j = 0; j < b->small.size();) {
    const int lg = hd[b->small[j]].lgn;
    size_t e = j;
    while (e < b->small.size() && hd[b->small[e]].lgn == lg) ++e;
    b->classes.push_back({lg, (int)j, (int)(e - j), 0});
    j = e;
  }
  {
    struct Item { double cost; int kind, idx; };
    std::vector<Item> items;
    for (size_t j = 0; j < b->classes.size(); ++j) {
      const auto& cl = b->classes[j];
      items.push_back({(double)(int64_t(1) << cl.lgn) * (double)((cl.count + 303) / 304), 0, (int)j});
    }
    std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& c2) { return a.cost > c2.cost; });
    double load[NSIDE_MAX] = {};
    for (const Item& itm : items) {
      const int k = (int)(std::min_element(load, load + b->nside) - load);
      load[k] += itm.cost;
      b->classes[itm.idx].side = k;
    }
  }
  auto fail = [&](cs_status e) {
    batch_free(b);
    return e;
  };
#define CS_B_TRY(expr)                          \
  do {                                          \
    cs_status e_ = cstat(expr);                 \
    if (e_ != CS_OK) return fail(e_);           \
  } while (0)
  for (int k = 0; k < b->nside; ++k) {
    CS_B_TRY(cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking));
    CS_B_TRY(cudaEventCreateWithFlags(&b->side_done[k], cudaEventDisableTiming));
  }
  CS_B_TRY(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  // large instances: their own plans (buffers, tables, masks) on the batch's
  // stream, and the parameters of the grouped launches over all of them
  for (size_t j = 0; j < b->large.size(); ++j) {
    const int i = b->large[j];
    cs_plan_t p = nullptr;
    const cs_status st = cs_plan(&p, n[i], m[i], rows + b->moff[i], c + b->noff[i], s);
    if (st != CS_OK) return fail(st);
    b->plans.push_back(p);
  }
  if (!b->large.empty()) {
    auto& G = b->grp;
    G.count = (int)b->large.size();
    CS_B_TRY(cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking));
    CS_B_TRY(balloc(&G.desc, G.count));
    CS_B_TRY(balloc(&G.kps_i, G.count));
    CS_B_TRY(balloc(&G.kps_a0, G.count));
    CS_B_TRY(balloc(&G.kps_a1, G.count));
    CS_B_TRY(balloc(&G.ca, G.count));
    std::vector<KParams> ki(G.count), ka0(G.count), ka1(G.count);
    std::vector<int2> mci, mmi, mca, mma;
    for (int j = 0; j < G.count; ++j) {
      const int i = b->large[j];
      const PlanView v = plan_view(b->plans[j]);
      GroupDesc d = v.desc;
      d.noff = b->noff[i];
      d.moff = b->moff[i];
      G.hdesc.push_back(d);
      ki[j] = v.kp_i;
      ka0[j] = v.kp_a;
      ki[j].ca = ka0[j].ca = G.ca + j;
      ka1[j] = ka0[j];
      ka1[j].flags = FL_WRITE_STATE;
      for (int t = 0; t < d.gi.col_ctas; ++t) mci.push_back(make_int2(j, t));
      for (int t = 0; t < d.gi.mid_ctas; ++t) mmi.push_back(make_int2(j, t));
      for (int t = 0; t < d.ga.col_ctas; ++t) mca.push_back(make_int2(j, t));
      for (int t = 0; t < d.ga.mid_ctas; ++t) mma.push_back(make_int2(j, t));
      // grouped launches take 4096-value tiles and run-time shapes only
      if (d.gi.tile != 4096 || d.ga.tile != 4096 || d.gi.col_tile != 4096 || d.ga.col_tile != 4096)
        return fail(CS_ERR_UNSUPPORTED);
    }
    G.n_col_i = (int)mci.size();
    G.n_mid_i = (int)mmi.size();
    G.n_col_a = (int)mca.size();
    G.n_mid_a = (int)mma.size();
    CS_B_TRY(balloc(&G.map_col_i, mci.size()));
    CS_B_TRY(balloc(&G.map_mid_i, mmi.size()));
    CS_B_TRY(balloc(&G.map_col_a, mca.size()));
    CS_B_TRY(balloc(&G.map_mid_a, mma.size()));
    CS_B_TRY(cudaMemcpyAsync(G.desc, G.hdesc.data(), G.count * sizeof(GroupDesc), cudaMemcpyHostToDevice, s));
    CS_B_TRY(cudaMemcpyAsync(G.kps_i, ki.data(), G.count * sizeof(KParams), cudaMemcpyHostToDevice, s));
    CS_B_TRY(cudaMemcpyAsync(G.kps_a0, ka0.data(), G.count * sizeof(KParams), cudaMemcpyHostToDevice, s));
    CS_B_TRY(cudaMemcpyAsync(G.kps_a1, ka1.data(), G.count * sizeof(KParams), cudaMemcpyHostToDevice, s));
    CS_B_TRY(cudaMemcpyAsync(G.map_col_i, mci.data(), mci.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    CS_B_TRY(cudaMemcpyAsync(G.map_mid_i, mmi.data(), mmi.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    CS_B_TRY(cudaMemcpyAsync(G.map_col_a, mca.data(), mca.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    CS_B_TRY(cudaMemcpyAsync(G.map_mid_a, mma.data(), mma.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    CS_B_TRY(cudaStreamSynchronize(s));
  }
  if (!b->small.empty()) {
    for (int lg = BI_LG_MIN; lg <= BI_LG_MAX; ++lg) {
      const ClassKernel k = ista_class(lg);
      CS_B_TRY(cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem));
    }
    for (int lg = BA_LG_MIN; lg <= BA_LG_MAX; ++lg) {
      const ClassKernel k = admm_class(lg);
      CS_B_TRY(cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem));
    }
    CS_B_TRY(balloc(&b->descs, count));
    CS_B_TRY(balloc(&b->sc, count));
    CS_B_TRY(balloc(&b->order, b->small.size()));
    CS_B_TRY(balloc(&b->tA, it));
    CS_B_TRY(balloc(&b->tB, it));
    CS_B_TRY(balloc(&b->tc, at));
    CS_B_TRY(balloc(&b->abs2, at));
    CS_B_TRY(balloc(&b->tb, at));
    CS_B_TRY(balloc(&b->tb_inst, at));
    CS_B_TRY(balloc(&b->drho, count));
    CS_B_TRY(balloc(&b->dsigma, count));
    CS_B_TRY(balloc(&b->mask, wo));
    CS_B_TRY(balloc(&b->prefix, wo));
    CS_B_TRY(balloc(&b->pos, mo));
    CS_B_TRY(balloc(&b->ys, mo));
    CS_B_TRY(balloc(&b->tw, 1 << LG_TW));
    CS_B_TRY(balloc(&b->amu, no));
    CS_B_TRY(balloc(&b->anu, no));
    CS_B_TRY(balloc(&b->status, 1));
    CS_B_TRY(cudaMemsetAsync(b->status, 0, sizeof(int), s));
    CS_B_TRY(cudaMemsetAsync(b->mask, 0, (wo ? wo : 1) * sizeof(uint32_t), s));
    CS_B_TRY(cudaMemsetAsync(b->pos, 0xff, (mo ? mo : 1) * sizeof(int32_t), s));   // -1: not a small instance
    CS_B_TRY(cudaMemcpyAsync(b->descs, hd.data(), count * sizeof(BatchDesc), cudaMemcpyHostToDevice, s));
    CS_B_TRY(cudaMemcpyAsync(b->order, b->small.data(), b->small.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    CS_B_TRY(launch_twiddle(b->tw, 1 << LG_TW, 1 << LG_TW, s));
    std::vector<int> inst(at);
    int64_t nmax = 0, mmax = 0;
    for (int i : b->small) {
      nmax = std::max(nmax, n[i]);
      mmax = std::max(mmax, m[i]);
      std::fill(inst.begin() + hd[i].atab, inst.begin() + hd[i].atab + n[i] / 2 + 1, i);
    }
    CS_B_TRY(cudaMemcpyAsync(b->tb_inst, inst.data(), at * sizeof(int), cudaMemcpyHostToDevice, s));
    double* dc = nullptr;
    double2 *fa = nullptr, *fb = nullptr;
    int64_t* drows = nullptr;
    CS_B_TRY(balloc(&dc, nmax));
    CS_B_TRY(balloc(&fa, nmax));
    CS_B_TRY(balloc(&fb, nmax));
    CS_B_TRY(balloc(&drows, mmax));
    cudaError_t e = cudaSuccess;
    for (int i : b->small) {
      const BatchDesc& d = hd[i];
      if (e == cudaSuccess) e = cudaMemcpyAsync(dc, c + d.noff, n[i] * sizeof(double), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(drows, rows + d.moff, m[i] * sizeof(int64_t), cudaMemcpyHostToDevice, s);
      double2* chat = nullptr;
      if (e == cudaSuccess) e = launch_fft64(dc, fa, fb, n[i], &chat, s);
      if (e == cudaSuccess) {
        tab_ista1_k<<<nb256(n[i] / 4 + 1), 256, 0, s>>>(chat, n[i], b->tA + d.itab, b->tB + d.itab);
        tab_admm1_k<<<nb256(n[i] / 2 + 1), 256, 0, s>>>(chat, n[i], b->tc + d.atab, b->abs2 + d.atab);
        batch_mask_k<<<nb256(m[i]), 256, 0, s>>>(drows, m[i], n[i], b->mask + d.woff, b->status);
        e = launch_prefix(b->mask + d.woff, n[i] / 32, b->prefix + d.woff, s);
      }
      if (e == cudaSuccess) {
        batch_pos_k<<<nb256(m[i]), 256, 0, s>>>(drows, m[i], b->mask + d.woff, b->prefix + d.woff, d.moff,
                                                 b->pos + d.moff);
        e = cudaGetLastError();
      }
      // the staging buffers are reused by the next instance: keep the order
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    cudaFree(dc);
    cudaFree(fa);
    cudaFree(fb);
    cudaFree(drows);
    CS_B_TRY(e);
    int hs = 0;
    CS_B_TRY(cudaMemcpy(&hs, b->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (hs & (STS_BAD_ROW | STS_DUP_ROW)) return fail(CS_ERR_ARG);
    b->host_rho.assign(count, -1.0);
    b->host_sigma.assign(count, -1.0);
  }
  if (!b->status) {
    CS_B_TRY(balloc(&b->status, 1));
    CS_B_TRY(cudaMemsetAsync(b->status, 0, sizeof(int), s));
  }
  if (!b->smooth_ids.empty()) {
    const cs_status st = (cs_status)smooth_plan(&b->smooth, b->smooth_ids.data(), (int)b->smooth_ids.size(), n, m,
                                                b->noff.data(), b->moff.data(), rows, c, b->status, s);
    if (st != CS_OK) return fail(st);
  }
  CS_B_TRY(cudaStreamSynchronize(s));
  for (int k = 0; k < b->nside; ++k) CS_B_TRY(cudaStreamSynchronize(b->side[k]));
#undef CS_B_TRY
  *out = b;
  return CS_OK;
}

cs_status cs_batch_destroy(cs_batch_t b) {
  if (!b) return CS_ERR_ARG;
  cudaStreamSynchronize(b->stream);
  for (int k = 0; k < b->nside; ++k)
    if (b->side[k]) cudaStreamSynchronize(b->side[k]);
  batch_free(b);
  return CS_OK;
}

cs_status cs_batch_ista(cs_batch_t b, const float* y, const float* lambda, const float* tau, int iters, float* x) {
  if (!b || !y || !lambda || !tau || !x || iters < 0) return CS_ERR_ARG;
  for (int i = 0; i < b->count; ++i)
    if (!(lambda[i] >= 0.f) || !(tau[i] > 0.f) || !std::isfinite(lambda[i]) || !std::isfinite(tau[i])) return CS_ERR_ARG;
  cudaStream_t s = b->stream;
  if (!b->small.empty() && iters > 0) {
    std::vector<BatchScalars> h(b->count);
    for (int i = 0; i < b->count; ++i) {
      h[i] = BatchScalars{};
      h[i].thr = (float)((double)tau[i] * (double)lambda[i]);
      h[i].tau = tau[i];
    }
    const cs_status st = cstat(cudaMemcpyAsync(b->sc, h.data(), b->count * sizeof(BatchScalars),
                                               cudaMemcpyHostToDevice, s));
    if (st != CS_OK) return st;
    batch_scatter_k<<<nb256(b->mtot), 256, 0, s>>>(y, b->pos, b->mtot, b->ys, b->status);
  }
  cs_status st = cstat(fork_sides(b));
  if (!b->large.empty() && st == CS_OK) {
    auto& G = b->grp;
    std::vector<CallArgs> h(G.count);
    for (int j = 0; j < G.count; ++j) {
      const int i = b->large[j];
      h[j] = CallArgs{};
      h[j].src = x + b->noff[i];   // COL_LOAD transforms x(0) in natural order
      h[j].x = G.hdesc[j].xi_t;    // the iterate lives in tile order during the solve
      h[j].thr = (float)((double)tau[i] * (double)lambda[i]);
      h[j].tau = tau[i];
    }
    st = cstat(cudaMemcpyAsync(G.ca, h.data(), G.count * sizeof(CallArgs), cudaMemcpyHostToDevice, s));
    if (st == CS_OK) st = cstat(launch_group_scatter_y(G.desc, G.count, y, 0, b->status, s));
    if (st == CS_OK && iters > 0) {
      st = cstat(launch_group_ista_in(G.desc, G.count, x, s));
      if (st == CS_OK)
        st = cstat(run_group_graph(b, (uint64_t(1) << 40) | (uint32_t)iters,
                                   [&](cudaStream_t cs) { return enqueue_group_ista(b, iters, cs); }));
      if (st == CS_OK) st = cstat(launch_group_ista_out(G.desc, G.count, x, s));
    }
  }
  if (iters > 0) {
    for (const auto& cl : b->classes) {
      if (st != CS_OK) break;
      const ClassKernel k = ista_class(cl.lgn - 1);
      const int* ord = b->order + cl.start;
      void* args[] = {&b->descs, &b->sc, (void*)&ord, &b->tA, &b->tB, &b->mask, &b->prefix, &b->ys, &b->tw,
                      (void*)&x, (void*)&iters};
      st = cstat(cudaLaunchKernel(k.fn, dim3((unsigned)cl.count), dim3(k.nt), args, k.smem, b->side[cl.side]));
    }
  }
  const cs_status sj = cstat(join_sides(b));
  if (st == CS_OK && sj == CS_OK && b->smooth) st = cstat(smooth_ista(b->smooth, y, lambda, tau, iters, x, s));
  return st != CS_OK ? st : sj;
}

cs_status cs_batch_admm(cs_batch_t b, const float* y, const float* lambda, const float* rho, int iters, float* z) {
  if (!b || !y || !lambda || !rho || !z || iters < 0) return CS_ERR_ARG;
  for (int i = 0; i < b->count; ++i)
    if (!(lambda[i] >= 0.f) || !(rho[i] > 0.f) || !std::isfinite(lambda[i]) || !std::isfinite(rho[i])) return CS_ERR_ARG;
  cudaStream_t s = b->stream;
  cs_status st = CS_OK;
  if (!b->small.empty() && iters == 0) {
    for (int i : b->small) {
      st = cstat(cudaMemsetAsync(z + b->noff[i], 0, b->n[i] * sizeof(float), s));
      if (st != CS_OK) return st;
    }
  }
  if (!b->small.empty() && iters > 0) {
    // sigma = rho, tau1 = tau2 = 1 (as cs_admm); B's spectrum re-tabulated when rho changes
    bool changed = false;
    std::vector<BatchScalars> h(b->count);
    for (int i = 0; i < b->count; ++i) {
      const double r = rho[i];
      if (r != b->host_rho[i]) changed = true;
      b->host_rho[i] = r;
      b->host_sigma[i] = r;
      h[i] = BatchScalars{};
      h[i].thr = (float)((double)lambda[i] / r);
      h[i].rho = (float)r;
      h[i].sigma = (float)r;
      h[i].tau1 = 1.f;
      h[i].tau2 = 1.f;
      h[i].d_on = (float)(1.0 / (1.0 + r));
      h[i].d_off = (float)(1.0 / r);
    }
    st = cstat(cudaMemcpyAsync(b->sc, h.data(), b->count * sizeof(BatchScalars), cudaMemcpyHostToDevice, s));
    if (st != CS_OK) return st;
    if (changed) {
      st = cstat(cudaMemcpyAsync(b->drho, b->host_rho.data(), b->count * sizeof(double), cudaMemcpyHostToDevice, s));
      if (st == CS_OK)
        st = cstat(cudaMemcpyAsync(b->dsigma, b->host_sigma.data(), b->count * sizeof(double),
                                   cudaMemcpyHostToDevice, s));
      if (st != CS_OK) return st;
      tab_admm1_b_k<<<nb256(b->atab_tot), 256, 0, s>>>(b->abs2, b->atab_tot, b->tb_inst, b->descs, b->drho,
                                                        b->dsigma, b->tb);
    }
    batch_scatter_k<<<nb256(b->mtot), 256, 0, s>>>(y, b->pos, b->mtot, b->ys, b->status);
  }
  st = cstat(fork_sides(b));
  if (!b->large.empty() && st == CS_OK) {
    // sigma = rho, tau1 = tau2 = 1 (as cs_admm), zero start
    auto& G = b->grp;
    std::vector<CallArgs> h(G.count);
    for (int j = 0; j < G.count && st == CS_OK; ++j) {
      const int i = b->large[j];
      const double r = rho[i];
      st = cstat(plan_admm_table(b->plans[j], r, r, s));
      h[j] = CallArgs{};
      h[j].z = G.hdesc[j].az;
      h[j].mu = G.hdesc[j].amu;
      h[j].nu = G.hdesc[j].anu;
      h[j].v = G.hdesc[j].av;
      h[j].thr = (float)((double)lambda[i] / r);
      h[j].rho = (float)r;
      h[j].sigma = (float)r;
      h[j].tau1 = 1.f;
      h[j].tau2 = 1.f;
      h[j].d_on = (float)(1.0 / (1.0 + r));
      h[j].d_off = (float)(1.0 / r);
    }
    if (st == CS_OK) st = cstat(cudaMemcpyAsync(G.ca, h.data(), G.count * sizeof(CallArgs), cudaMemcpyHostToDevice, s));
    if (st == CS_OK) st = cstat(launch_group_admm_zero(G.desc, G.count, s));
    if (st == CS_OK) st = cstat(launch_group_scatter_y(G.desc, G.count, y, 1, b->status, s));
    if (st == CS_OK && iters > 0)
      st = cstat(run_group_graph(b, (uint64_t(2) << 40) | (uint32_t)iters,
                                 [&](cudaStream_t cs) { return enqueue_group_admm(b, iters, cs); }));
    if (st == CS_OK) st = cstat(launch_group_admm_out(G.desc, G.count, z, s));
  }
  if (iters > 0) {
    for (const auto& cl : b->classes) {
      if (st != CS_OK) break;
      const ClassKernel k = admm_class(cl.lgn);
      const int* ord = b->order + cl.start;
      void* args[] = {&b->descs, &b->sc, (void*)&ord, &b->tc, &b->tb, &b->mask, &b->prefix, &b->ys, &b->tw,
                      (void*)&z, &b->amu, &b->anu, (void*)&iters};
      st = cstat(cudaLaunchKernel(k.fn, dim3((unsigned)cl.count), dim3(k.nt), args, k.smem, b->side[cl.side]));
    }
  }
  const cs_status sj = cstat(join_sides(b));
  if (st == CS_OK && sj == CS_OK && b->smooth) st = cstat(smooth_admm(b->smooth, y, lambda, rho, iters, z, s));
  return st != CS_OK ? st : sj;
}

cs_status cs_batch_status_sync(cs_batch_t b) {
  if (!b) return CS_ERR_ARG;
  cs_status st = cstat(cudaStreamSynchronize(b->stream));
  if (st != CS_OK) return st;
  for (cs_plan_t p : b->plans) {
    const cs_status ps = cs_status_sync(p);
    if (ps != CS_OK) return ps;
  }
  if (b->status) {
    int hs = 0;
    st = cstat(cudaMemcpy(&hs, b->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != CS_OK) return st;
    st = cstat(cudaMemset(b->status, 0, sizeof(int)));   // reported once, as cs_status_sync
    if (st != CS_OK) return st;
    if (hs & STS_TIMEOUT) return CS_ERR_TIMEOUT;
    if (hs & STS_NONFINITE) return CS_ERR_NONFINITE;
  }
  return CS_OK;
}

}  // extern "C"
