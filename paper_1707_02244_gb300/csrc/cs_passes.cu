// Fused FFT passes of the ISTA / ADMM iterations (fp32, sm_103a).
//
// Every circulant product is a convolution (Sec. 4.2: circulant matrices are
// diagonalised by the DFT).  A length-N complex FFT is split four-step into an
// N2 x N1 array: the column pass runs the length-N2 FFTs, the mid pass the
// length-N1 FFTs plus the inter-pass twiddle.  A convolution is therefore
//   column pass (forward)  ->  mid pass (forward, spectrum op, inverse)
//   ->  column pass (inverse)
// and the elementwise work of the method (residual on the kept rows,
// soft threshold, the ADMM updates) is fused into the column pass between the
// inverse FFT of one product and the forward FFT of the next.
//
// Real-FFT geometry (ISTA, products with C and C^T): a real n-vector is
// packed as n/2 complex values (x_2p + i x_2p+1); the mid pass combines the
// spectra at k and N-k so that the packed spectrum is multiplied by the
// circulant's real-signal spectrum without ever being unpacked.
// Complex-n geometry (ADMM): (v + mu) + i (z - nu) is one complex FFT whose
// k / N-k pairs give both real spectra; the x-update solve with
// B = (rho C^T C + sigma I)^-1 is a spectrum multiply (Sec. 4.3), and
// x + i C x comes back from one inverse FFT.
#include "cs_fft.cuh"
#include "cs_internal.h"

namespace csk {

namespace {

__device__ __forceinline__ float soft(float u, float g) {
  // Eq. 4: sgn(u)(|u| - g) for |u| > g, else 0
  return u > g ? u - g : (u < -g ? u + g : 0.f);
}

struct Acc {
  float v[NSTAT];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < NSTAT; ++i) v[i] = 0.f;
  }
};

// Block reduction of the per-thread accumulators into partials[block].
// Deterministic: fixed shuffle tree, fixed warp order.  SLOTS is a bit mask.
template <int SLOTS>
__device__ void block_stats(const Acc& a, double* partials) {
  __shared__ double red[NT / 32][NSTAT];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NSTAT; ++k) {
    if (!((SLOTS >> k) & 1)) continue;
    double d = (double)a.v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
    if (lane == 0) red[wid][k] = d;
  }
  __syncthreads();
  if (threadIdx.x < NSTAT && ((SLOTS >> threadIdx.x) & 1)) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w][threadIdx.x];
    partials[blockIdx.x * NSTAT + threadIdx.x] = s;
  }
}

// Row-of-Omega test and compact y index for spatial row i.
struct RowSel {
  const uint32_t* __restrict__ mask;
  const uint32_t* __restrict__ prefix;
  __device__ __forceinline__ bool get(int i, int& idx) const {
    const uint32_t w = __ldg(mask + (i >> 5));
    const int b = i & 31;
    idx = (int)__ldg(prefix + (i >> 5)) + __popc(w & ((1u << b) - 1u));
    return (w >> b) & 1u;
  }
};

__device__ __forceinline__ float2 ld2(const float* p, int i) {
  return __ldg(reinterpret_cast<const float2*>(p) + i);
}

// ---------------------------------------------------------------- epilogues
// apply(v, p, acc): v is the inverse-FFT output at complex index p (when the
// kind reads the exchange buffer); returns the forward-FFT input at p.

template <int KIND> struct Epi;

template <> struct Epi<COL_LOAD> {
  static constexpr bool kRead = false, kFwd = true;
  __device__ static float2 apply(const KParams& kp, const CallArgs& a, float2, int p, Acc&) {
    return ld2(a.src, p);
  }
};

template <> struct Epi<COL_LOAD_SCALED> {
  static constexpr bool kRead = false, kFwd = true;
  __device__ static float2 apply(const KParams& kp, const CallArgs& a, float2, int p, Acc&) {
    const float s = (float)rsqrt(kp.pp.stats[ST_X2]);
    float2 u = cscale(ld2(a.src, p), s);
    reinterpret_cast<float2*>(a.aux)[p] = u;
    return u;
  }
};

template <> struct Epi<COL_STORE> {
  static constexpr bool kRead = true, kFwd = false;
  __device__ static float2 apply(const KParams&, const CallArgs& a, float2 v, int p, Acc&) {
    reinterpret_cast<float2*>(a.dst)[p] = v;
    return v;
  }
};

template <> struct Epi<COL_MASK> {
  static constexpr bool kRead = true, kFwd = true;
  __device__ static float2 apply(const KParams& kp, const CallArgs&, float2 v, int p, Acc&) {
    RowSel rs{kp.pp.mask, kp.pp.prefix};
    int i0, i1;
    const bool m0 = rs.get(2 * p, i0), m1 = rs.get(2 * p + 1, i1);
    return make_float2(m0 ? v.x : 0.f, m1 ? v.y : 0.f);
  }
};

// r~ = M (P^T y - C x): residual of Algorithm 1 on the kept rows, zero off
// them, so that the next product gives A^T r = C^T P^T r.
template <> struct Epi<COL_RESIDUAL> {
  static constexpr bool kRead = true, kFwd = true;
  __device__ static float2 apply(const KParams& kp, const CallArgs&, float2 v, int p, Acc& acc) {
    RowSel rs{kp.pp.mask, kp.pp.prefix};
    int i0, i1;
    const bool m0 = rs.get(2 * p, i0), m1 = rs.get(2 * p + 1, i1);
    const float r0 = m0 ? __ldg(kp.pp.ys + i0) - v.x : 0.f;
    const float r1 = m1 ? __ldg(kp.pp.ys + i1) - v.y : 0.f;
    acc.v[ST_R2] = fmaf(r0, r0, fmaf(r1, r1, acc.v[ST_R2]));
    return make_float2(r0, r1);
  }
};

// x(t) = eta_{tau lambda}[x(t-1) + tau A^T r(t)]  (Algorithm 1, Eq. 4)
template <bool FWD> struct EpiIsta {
  static constexpr bool kRead = true, kFwd = FWD;
  __device__ static float2 apply(const KParams& kp, const CallArgs& a, float2 g, int p, Acc& acc) {
    float2* x = reinterpret_cast<float2*>(a.x);
    const float2 xo = x[p];
    float2 xn;
    xn.x = soft(fmaf(a.tau, g.x, xo.x), a.thr);
    xn.y = soft(fmaf(a.tau, g.y, xo.y), a.thr);
    x[p] = xn;
    if (kp.flags & FL_STATS) {
      const float d0 = xn.x - xo.x, d1 = xn.y - xo.y;
      acc.v[ST_DX2] = fmaf(d0, d0, fmaf(d1, d1, acc.v[ST_DX2]));
      acc.v[ST_X2] = fmaf(xn.x, xn.x, fmaf(xn.y, xn.y, acc.v[ST_X2]));
      acc.v[ST_L1] += fabsf(xo.x) + fabsf(xo.y);
      if (a.xtrue) {
        const float2 t = ld2(a.xtrue, p);
        const float e0 = xn.x - t.x, e1 = xn.y - t.y;
        acc.v[ST_ERR2] = fmaf(e0, e0, fmaf(e1, e1, acc.v[ST_ERR2]));
      }
      if (!isfinite(xn.x) || !isfinite(xn.y)) acc.v[ST_NONFIN] += 1.f;
    }
    return xn;
  }
};
template <> struct Epi<COL_ISTA> : EpiIsta<true> {};
template <> struct Epi<COL_ISTA_LAST> : EpiIsta<false> {};

template <> struct Epi<COL_POWER_OUT> {
  static constexpr bool kRead = true, kFwd = false;
  __device__ static float2 apply(const KParams&, const CallArgs& a, float2 w, int p, Acc& acc) {
    const float2 u = ld2(a.aux, p);
    reinterpret_cast<float2*>(a.dst)[p] = w;
    acc.v[ST_X2] = fmaf(w.x, w.x, fmaf(w.y, w.y, acc.v[ST_X2]));
    acc.v[ST_DX2] = fmaf(u.x, w.x, fmaf(u.y, w.y, acc.v[ST_DX2]));
    return w;
  }
};

// Complex-n geometry: p is the spatial index itself.
template <> struct Epi<COL_ADMM_INIT> {
  static constexpr bool kRead = false, kFwd = true;
  __device__ static float2 apply(const KParams&, const CallArgs& a, float2, int p, Acc&) {
    return make_float2(a.v[p], a.z[p] - a.nu[p]);
  }
};

// Algorithm 3, after the x-update: v = D(rho C x - rho mu + P^T y),
// z = eta_{lambda/sigma}(x + nu), mu += tau1 (v - C x), nu += tau2 (x - z),
// v <- v + mu; the next x-update reads (v) + i (z - nu).
template <bool FWD> struct EpiAdmm {
  static constexpr bool kRead = true, kFwd = FWD;
  __device__ static float2 apply(const KParams& kp, const CallArgs& a, float2 xc, int p, Acc& acc) {
    RowSel rs{kp.pp.mask, kp.pp.prefix};
    int iy;
    const bool on = rs.get(p, iy);
    const float yv = on ? __ldg(kp.pp.ys + iy) : 0.f;
    const float x = xc.x, cx = xc.y;
    const float mu = a.mu[p], nu = a.nu[p];
    const float d = on ? a.d_on : a.d_off;
    const float v = d * fmaf(a.rho, cx - mu, yv);
    const float z = soft(x + nu, a.thr);
    const float mu2 = fmaf(a.tau1, v - cx, mu);
    const float nu2 = fmaf(a.tau2, x - z, nu);
    const float vf = v + mu2;
    a.mu[p] = mu2;
    a.nu[p] = nu2;
    if (kp.flags & FL_WRITE_STATE) {
      a.z[p] = z;
      a.v[p] = vf;
      if (a.x) a.x[p] = x;
    }
    if (kp.flags & FL_STATS) {
      if (a.xtrue) {
        const float e = z - __ldg(a.xtrue + p);
        acc.v[ST_ERR2] = fmaf(e, e, acc.v[ST_ERR2]);
      }
      const float pr = x - z;
      acc.v[ST_DX2] = fmaf(pr, pr, acc.v[ST_DX2]);
      acc.v[ST_X2] = fmaf(z, z, acc.v[ST_X2]);
      acc.v[ST_L1] += fabsf(z);
      const float r = on ? yv - cx : 0.f;
      acc.v[ST_R2] = fmaf(r, r, acc.v[ST_R2]);
      if (!isfinite(z) || !isfinite(vf)) acc.v[ST_NONFIN] += 1.f;
    }
    return make_float2(vf, z - nu2);
  }
};
template <> struct Epi<COL_ADMM> : EpiAdmm<true> {};
template <> struct Epi<COL_ADMM_LAST> : EpiAdmm<false> {};

// ---------------------------------------------------------------- column pass

template <int KIND>
__global__ void __launch_bounds__(NT) col_kernel(const KParams kp) {
  using E = Epi<KIND>;
  extern __shared__ float2 sm[];
  const Geo& g = kp.geo;
  const CallArgs a = *kp.ca;
  const int G = g.G, lgG = g.lgG;
  const int col0 = blockIdx.x << lgG;
  const int tot = G << g.lgN2;
  const VecLayout lay{g.lgN2, lgG, true};
  float2* __restrict__ W = kp.pp.W;

  if (E::kRead) {
    for (int e = 2 * threadIdx.x; e < tot; e += 2 * NT) {
      const int j2 = e >> lgG, c = e & (G - 1);
      const float4 v = __ldcg(reinterpret_cast<const float4*>(W + col0 + c + ((size_t)j2 << g.lgN1)));
      sm[pad(e)] = make_float2(v.x, v.y);
      sm[pad(e + 1)] = make_float2(v.z, v.w);
    }
    __syncthreads();
    tile_fft<+1>(sm, lay, g.tw2, g.lgN2);
  }

  Acc acc;
  acc.zero();
  for (int e = threadIdx.x; e < tot; e += NT) {
    const int j2 = e >> lgG, c = e & (G - 1);
    const int p = col0 + c + (j2 << g.lgN1);
    const float2 v = E::kRead ? sm[pad(e)] : make_float2(0.f, 0.f);
    sm[pad(e)] = E::apply(kp, a, v, p, acc);
  }
  if (kp.flags & FL_STATS) {
    constexpr int kSlots =
        KIND == COL_RESIDUAL ? (1 << ST_R2)
        : KIND == COL_POWER_OUT ? ((1 << ST_DX2) | (1 << ST_X2))
        : (KIND == COL_ISTA || KIND == COL_ISTA_LAST)
            ? ((1 << ST_ERR2) | (1 << ST_DX2) | (1 << ST_X2) | (1 << ST_L1) | (1 << ST_NONFIN))
        : (KIND == COL_ADMM || KIND == COL_ADMM_LAST) ? ((1 << ST_ERR2) | (1 << ST_DX2) | (1 << ST_X2) |
                                                         (1 << ST_L1) | (1 << ST_R2) | (1 << ST_NONFIN))
        : 0;
    if (kSlots) block_stats<kSlots>(acc, kp.pp.partials);
  }
  if (E::kFwd) {
    __syncthreads();
    tile_fft<-1>(sm, lay, g.tw2, g.lgN2);
    for (int e = 2 * threadIdx.x; e < tot; e += 2 * NT) {
      const int j2 = e >> lgG, c = e & (G - 1);
      const float2 lo = sm[pad(e)], hi = sm[pad(e + 1)];
      __stcg(reinterpret_cast<float4*>(W + col0 + c + ((size_t)j2 << g.lgN1)),
             make_float4(lo.x, lo.y, hi.x, hi.y));
    }
  }
}

// ---------------------------------------------------------------- mid pass

// w_N^(j1 k2) from the two-level table: w_N^p = w_N^(p mod N1) * w_N2^(p div N1)
__device__ __forceinline__ float2 tw4(const Geo& g, int p) {
  return cmul(__ldg(g.twl + (p & (g.N1 - 1))), __ldg(g.tw2 + (p >> g.lgN1)));
}

__device__ __forceinline__ int slot_row(const Geo& g, int u, int second) {
  if (u == 0) return second ? (g.N2 >> 1) : 0;
  return second ? g.N2 - u : u;
}

// Real-FFT spectrum operator (products with C and C^T on the packed vector).
// For the pair (k, N - k) of the packed spectrum Z, with H the real-signal
// spectrum of the product (H = chat for C^T, conj(chat) for C) and
// theta = 2 pi k / (2N):
//   Z'_k   = a  Z_k   + b  conj(Z_{N-k})
//   Z'_N-k = a' Z_N-k + b' conj(Z_k)
//   a = P - Q sin, b = i Q cos, a' = conj(P) + conj(Q) sin, b' = -conj(b),
//   P = (H_k + H_{k+N}) / 2N, Q = (H_k - H_{k+N}) / 2N.
// The table stores P, Q for H = chat; H = conj(chat) conjugates a, a' and
// swaps b -> -conj(b), b' -> b.
template <bool ADJ>
__device__ __forceinline__ void op_real(const Geo& g, const PlanPtrs& pp, int tidx, int k2, int k1,
                                        float2& za, float2& zb) {
  const float4 t = __ldg(pp.tab_ista + tidx);
  const float2 P = make_float2(t.x, t.y), Q = make_float2(t.z, t.w);
  const float2 e = cmul(__ldg(g.twr + k2), __ldg(g.tw1 + k1));   // exp(-i theta)
  const float cs = e.x, sn = -e.y;
  float2 al = make_float2(fmaf(-Q.x, sn, P.x), fmaf(-Q.y, sn, P.y));
  float2 be = make_float2(-Q.y * cs, Q.x * cs);
  float2 al2 = make_float2(fmaf(Q.x, sn, P.x), -fmaf(Q.y, sn, P.y));
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

// Complex-n ADMM operator for the pair (k, N - k) of Z = FFT((v) + i (z - nu)):
//   V = (Z_k + conj Z_{N-k}) / 2,  Wk = (Z_k - conj Z_{N-k}) / 2i
//   X = bhat (rho chat V + sigma Wk) / N            (x-update, Algorithm 3)
//   Pc = conj(chat) X                                 (spectrum of C x)
//   Z'_k = X + i Pc,  Z'_{N-k} = conj(X) + i conj(Pc)
__device__ __forceinline__ void op_admm(const PlanPtrs& pp, const CallArgs& a, int tidx,
                                        float2& za, float2& zb) {
  const float2 ch = __ldg(pp.tab_admm_c + tidx);
  const float bb = __ldg(pp.tab_admm_b + tidx);
  const float2 V = make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y - zb.y));
  const float2 Wk = make_float2(0.5f * (za.y + zb.y), -0.5f * (za.x - zb.x));
  const float2 cv = cmul(ch, V);
  const float2 X = make_float2(bb * fmaf(a.rho, cv.x, a.sigma * Wk.x),
                               bb * fmaf(a.rho, cv.y, a.sigma * Wk.y));
  const float2 Pc = cmulc(X, ch);
  za = make_float2(X.x - Pc.y, X.y + Pc.x);
  zb = make_float2(X.x + Pc.y, Pc.x - X.y);
}

template <int KIND>
__global__ void __launch_bounds__(NT) mid_kernel(const KParams kp) {
  extern __shared__ float2 sm[];
  const Geo& g = kp.geo;
  const int lgU = g.lgU, U = g.U;
  const int u0 = blockIdx.x << lgU;
  const int N1 = g.N1, lgN1 = g.lgN1;
  const int tot = (2 * U) << lgN1;
  const VecLayout lay{lgN1, lgU + 1, false};
  float2* __restrict__ W = kp.pp.W;

  // load 2U rows, applying the forward four-step twiddle w_N^(j1 k2)
  for (int e = 2 * threadIdx.x; e < tot; e += 2 * NT) {
    const int slot = e >> lgN1, j1 = e & (N1 - 1);
    const int k2 = slot_row(g, u0 + (slot >> 1), slot & 1);
    const float4 v = __ldcg(reinterpret_cast<const float4*>(W + ((size_t)k2 << lgN1) + j1));
    sm[pad(e)] = cmul(make_float2(v.x, v.y), tw4(g, j1 * k2));
    sm[pad(e + 1)] = cmul(make_float2(v.z, v.w), tw4(g, (j1 + 1) * k2));
  }
  __syncthreads();
  tile_fft<-1>(sm, lay, g.tw1, g.lgN1 + 1);

  // spectrum operator over all (k, N-k) pairs held by this CTA
  const CallArgs a = *kp.ca;
  const int nslots = (U << lgN1) + (u0 == 0 ? 1 : 0);
  const int base_u1 = ((g.N2 >> 1) - 1) << lgN1;   // table offset of unit 0
  for (int t = threadIdx.x; t < nslots; t += NT) {
    int ul, q;
    if (t < (U << lgN1)) { ul = t >> lgN1; q = t & (N1 - 1); }
    else { ul = 0; q = N1; }
    const int u = u0 + ul;
    int ea, eb, k2, k1, tidx;
    if (u > 0) {
      k2 = u; k1 = q;
      ea = ((2 * ul) << lgN1) + q;
      eb = ((2 * ul + 1) << lgN1) + (N1 - 1 - q);
      tidx = ((u - 1) << lgN1) + q;
    } else if (q <= (N1 >> 1)) {
      k2 = 0; k1 = q;
      ea = ((2 * ul) << lgN1) + q;
      eb = ((2 * ul) << lgN1) + ((N1 - q) & (N1 - 1));
      tidx = base_u1 + q;
    } else {
      const int qq = q - (N1 >> 1) - 1;
      k2 = g.N2 >> 1; k1 = qq;
      ea = ((2 * ul + 1) << lgN1) + qq;
      eb = ((2 * ul + 1) << lgN1) + (N1 - 1 - qq);
      tidx = base_u1 + q;
    }
    float2 za = sm[pad(ea)], zb = sm[pad(eb)];
    if (KIND == MID_ADMM) op_admm(kp.pp, a, tidx, za, zb);
    else op_real<KIND == MID_ADJ>(g, kp.pp, tidx, k2, k1, za, zb);
    sm[pad(eb)] = zb;   // self-pairs (ea == eb) keep the k-side value
    sm[pad(ea)] = za;
  }
  __syncthreads();
  tile_fft<+1>(sm, lay, g.tw1, g.lgN1 + 1);

  // store with the inverse twiddle conj(w_N^(j1 k2))
  for (int e = 2 * threadIdx.x; e < tot; e += 2 * NT) {
    const int slot = e >> lgN1, j1 = e & (N1 - 1);
    const int k2 = slot_row(g, u0 + (slot >> 1), slot & 1);
    const float2 lo = cmulc(sm[pad(e)], tw4(g, j1 * k2));
    const float2 hi = cmulc(sm[pad(e + 1)], tw4(g, (j1 + 1) * k2));
    __stcg(reinterpret_cast<float4*>(W + ((size_t)k2 << lgN1) + j1), make_float4(lo.x, lo.y, hi.x, hi.y));
  }
}

template <typename K>
cudaError_t launch_k(K kern, int grid, const KParams& kp, cudaStream_t s) {
  kern<<<grid, NT, pass_smem_bytes(), s>>>(kp);
  return cudaGetLastError();
}

template <typename K>
cudaError_t set_smem(K kern) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pass_smem_bytes());
}

}  // namespace

size_t pass_smem_bytes() { return sizeof(float2) * (size_t)smem_slots(TILE); }

// Opt every pass kernel into the shared memory it needs (once per device).
cudaError_t init_pass_kernels() {
  cudaError_t e = cudaSuccess;
#define CS_SET(k) if (e == cudaSuccess) e = set_smem(k)
  CS_SET(col_kernel<COL_LOAD>); CS_SET(col_kernel<COL_LOAD_SCALED>); CS_SET(col_kernel<COL_STORE>);
  CS_SET(col_kernel<COL_MASK>); CS_SET(col_kernel<COL_RESIDUAL>); CS_SET(col_kernel<COL_ISTA>);
  CS_SET(col_kernel<COL_ISTA_LAST>); CS_SET(col_kernel<COL_POWER_OUT>);
  CS_SET(col_kernel<COL_ADMM_INIT>); CS_SET(col_kernel<COL_ADMM>); CS_SET(col_kernel<COL_ADMM_LAST>);
  CS_SET(mid_kernel<MID_FWD>); CS_SET(mid_kernel<MID_ADJ>); CS_SET(mid_kernel<MID_ADMM>);
#undef CS_SET
  return e;
}

cudaError_t launch_col(ColKind kind, const KParams& kp, cudaStream_t s) {
  const int grid = kp.geo.col_ctas;
  switch (kind) {
    case COL_LOAD: return launch_k(col_kernel<COL_LOAD>, grid, kp, s);
    case COL_LOAD_SCALED: return launch_k(col_kernel<COL_LOAD_SCALED>, grid, kp, s);
    case COL_STORE: return launch_k(col_kernel<COL_STORE>, grid, kp, s);
    case COL_MASK: return launch_k(col_kernel<COL_MASK>, grid, kp, s);
    case COL_RESIDUAL: return launch_k(col_kernel<COL_RESIDUAL>, grid, kp, s);
    case COL_ISTA: return launch_k(col_kernel<COL_ISTA>, grid, kp, s);
    case COL_ISTA_LAST: return launch_k(col_kernel<COL_ISTA_LAST>, grid, kp, s);
    case COL_POWER_OUT: return launch_k(col_kernel<COL_POWER_OUT>, grid, kp, s);
    case COL_ADMM_INIT: return launch_k(col_kernel<COL_ADMM_INIT>, grid, kp, s);
    case COL_ADMM: return launch_k(col_kernel<COL_ADMM>, grid, kp, s);
    case COL_ADMM_LAST: return launch_k(col_kernel<COL_ADMM_LAST>, grid, kp, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_mid(MidKind kind, const KParams& kp, cudaStream_t s) {
  const int grid = kp.geo.mid_ctas;
  switch (kind) {
    case MID_FWD: return launch_k(mid_kernel<MID_FWD>, grid, kp, s);
    case MID_ADJ: return launch_k(mid_kernel<MID_ADJ>, grid, kp, s);
    case MID_ADMM: return launch_k(mid_kernel<MID_ADMM>, grid, kp, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace csk
