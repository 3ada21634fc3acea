// Fused FFT passes of the ISTA / ADMM iterations (fp32, sm_103a): shared
// pieces of the column pass (cs_col.cu) and the mid pass (cs_mid.cu).
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
#pragma once

#include <type_traits>

#include "cs_fft.cuh"
#include "cs_internal.h"

namespace csk {

namespace {

__device__ __forceinline__ float sgnf(float v) { return v > 0.f ? 1.f : (v < 0.f ? -1.f : 0.f); }

__device__ __forceinline__ float soft(float u, float g) {
  // Eq. 4: sgn(u)(|u| - g) for |u| > g, else 0
  return u > g ? u - g : (u < -g ? u + g : 0.f);
}

constexpr int NACC = ST_NONFIN + 1;   // accumulated statistic slots

struct Acc {
  float v[NACC];
  // the CTA's tile of the row mask and its prefix counts, copied to shared
  // memory (indexed by global word minus wbase)
  const uint32_t* smask;
  const uint32_t* spref;
  int wbase;
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < NACC; ++i) v[i] = 0.f;
  }
};

// Block reduction of the per-thread accumulators into partials[block].
// Deterministic: fixed shuffle tree, fixed warp order.  SLOTS is a bit mask.
template <int SLOTS, int NT>
__device__ void block_stats(const Acc& a, double* partials, int blk) {
  __shared__ double red[NT / 32][NSTAT];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NACC; ++k) {
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
    partials[blk * NSTAT + threadIdx.x] = s;
  }
}

// Row-of-Omega test and compact y index for the row with mask bit i (tile
// order), from the CTA's copy of its mask words in shared memory.
struct RowSel {
  const uint32_t* mask;     // shared: words wbase ..
  const uint32_t* prefix;
  int wbase;
  __device__ __forceinline__ bool get(int i, int& idx) const {
    const uint32_t w = mask[(i >> 5) - wbase];
    const int b = i & 31;
    idx = (int)prefix[(i >> 5) - wbase] + __popc(w & ((1u << b) - 1u));
    return (w >> b) & 1u;
  }
  // bits 2p and 2p+1 (same word): returns the two bits, idx of bit 2p
  __device__ __forceinline__ uint32_t get2(int p, int& idx) const {
    const uint32_t w = mask[(p >> 4) - wbase];
    const int b = (2 * p) & 31;
    idx = (int)prefix[(p >> 4) - wbase] + __popc(w & ((1u << b) - 1u));
    return (w >> b) & 3u;
  }
};

// Which epilogues look up the row mask, and how many mask bits one element
// of the tile holds (2 in the packed real-FFT geometry, 1 in complex-n).
template <int KIND> struct UsesMask {
  static constexpr int kBits = (KIND == COL_RESIDUAL || KIND == COL_MASK || KIND == COL_RES_SAVE ||
                                KIND == COL_GRAD_MASK) ? 2
                              : (KIND == COL_ADMM || KIND == COL_ADMM_LAST || KIND == COL_ADMM_SEG ||
                                 KIND == COL_ADMM_REV) ? 1 : 0;
};

// Block sum of one per-thread value, added to dst[blk] (one slot per tile,
// so repeated launches accumulate without atomics; fixed order).
template <int NT>
__device__ void block_accum(float v, double* dst, int blk) {
  __shared__ double red[NT / 32];
  double d = (double)v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w];
    dst[blk] += s;
  }
}

// Complex element i (floats 2i, 2i + 1) of a float vector that may start at
// any 4-byte boundary (a caller's slice of a concatenation of odd-length
// vectors): one 8-byte access when the vector is 8-byte aligned, two 4-byte
// ones otherwise; the test is the same for every thread of a launch.
__device__ __forceinline__ float2 ld2(const float* p, int i) {
  if ((reinterpret_cast<uintptr_t>(p) & 7u) == 0) return __ldg(reinterpret_cast<const float2*>(p) + i);
  return make_float2(__ldg(p + 2 * i), __ldg(p + 2 * i + 1));
}
__device__ __forceinline__ void st2(float* p, int i, float2 v) {
  if ((reinterpret_cast<uintptr_t>(p) & 7u) == 0) {
    reinterpret_cast<float2*>(p)[i] = v;
  } else {
    p[2 * i] = v.x;
    p[2 * i + 1] = v.y;
  }
}

// ---------------------------------------------------------------- epilogues
// apply(v, p, t, acc): v is the inverse-FFT output at complex index p (when the
// kind reads the exchange buffer); returns the forward-FFT input at p.

// Index conventions.  p is the natural index (complex p of the packed vector
// in the real-FFT geometry, the spatial index in the complex-n geometry);
// API-facing buffers (src, dst, aux) use it.  t is the tile-order index of
// the column pass: t = g (G N2) + j2 G + c for p = g G + c + j2 N1.  The
// solver state (x; v, z, mu, nu), the ground truth copy, the row mask and the
// compact y all live in tile order, so each column CTA touches one contiguous
// block of every one of them.
template <int KIND> struct Epi;

template <> struct Epi<COL_LOAD> {
  static constexpr bool kRead = false, kFwd = true;
  __device__ static float2 apply(const KParams& kp, const CallArgs& a, float2, int p, int t, Acc&) {
    return ld2(a.src, p);
  }
};

template <> struct Epi<COL_LOAD_SCALED> {
  static constexpr bool kRead = false, kFwd = true;
  __device__ static float2 apply(const KParams& kp, const CallArgs& a, float2, int p, int t, Acc&) {
    const float s = (float)rsqrt(kp.pp.stats[ST_X2]);
    float2 u = cscale(ld2(a.src, p), s);
    st2(a.aux, p, u);
    return u;
  }
};

template <> struct Epi<COL_STORE> {
  static constexpr bool kRead = true, kFwd = false;
  __device__ static float2 apply(const KParams&, const CallArgs& a, float2 v, int p, int t, Acc&) {
    st2(a.dst, p, v);
    return v;
  }
};

template <> struct Epi<COL_MASK> {
  static constexpr bool kRead = true, kFwd = true;
  __device__ static float2 apply(const KParams& kp, const CallArgs&, float2 v, int p, int t, Acc& acc) {
    RowSel rs{acc.smask, acc.spref, acc.wbase};
    int i0;
    const uint32_t mm = rs.get2(t, i0);
    return make_float2((mm & 1u) ? v.x : 0.f, (mm & 2u) ? v.y : 0.f);
  }
};

// r~ = M (P^T y - C x): residual of Algorithm 1 on the kept rows, zero off
// them, so that the next product gives A^T r = C^T P^T r.
template <> struct Epi<COL_RESIDUAL> {
  static constexpr bool kRead = true, kFwd = true;
  __device__ static float2 apply(const KParams& kp, const CallArgs&, float2 v, int p, int t, Acc& acc) {
    RowSel rs{acc.smask, acc.spref, acc.wbase};
    int i0;
    const uint32_t mm = rs.get2(t, i0);
    const float r0 = (mm & 1u) ? __ldg(kp.pp.ys + i0) - v.x : 0.f;
    const float r1 = (mm & 2u) ? __ldg(kp.pp.ys + i0 + (int)(mm & 1u)) - v.y : 0.f;
    acc.v[ST_R2] = fmaf(r0, r0, fmaf(r1, r1, acc.v[ST_R2]));
    return make_float2(r0, r1);
  }
};

// x(t) = eta_{tau lambda}[x(t-1) + tau A^T r(t)]  (Algorithm 1, Eq. 4)
// Every element of x is read once, by the thread that then overwrites it, and
// by no other thread: the read can take the read-only path, which lets the
// loads of a thread's elements issue together instead of waiting behind the
// stores to x (that might otherwise alias them).
template <bool FWD> struct EpiIsta {
  static constexpr bool kRead = true, kFwd = FWD;
  __device__ static float2 apply(const KParams& kp, const CallArgs& a, float2 g, int p, int t, Acc& acc) {
    float2* x = reinterpret_cast<float2*>(a.x);
    const float2 xo = __ldg(x + t);
    float2 xn;
    xn.x = soft(fmaf(a.tau, g.x, xo.x), a.thr);
    xn.y = soft(fmaf(a.tau, g.y, xo.y), a.thr);
    x[t] = xn;
    if (kp.flags & FL_STATS) {
      const float d0 = xn.x - xo.x, d1 = xn.y - xo.y;
      acc.v[ST_DX2] = fmaf(d0, d0, fmaf(d1, d1, acc.v[ST_DX2]));
      acc.v[ST_X2] = fmaf(xn.x, xn.x, fmaf(xn.y, xn.y, acc.v[ST_X2]));
      acc.v[ST_L1] += fabsf(xo.x) + fabsf(xo.y);
      if (a.xtrue) {
        const float2 xs = ld2(a.xtrue, t);
        const float e0 = xn.x - xs.x, e1 = xn.y - xs.y;
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
  __device__ static float2 apply(const KParams&, const CallArgs& a, float2 w, int p, int t, Acc& acc) {
    const float2 u = ld2(a.aux, p);
    st2(a.dst, p, w);
    acc.v[ST_X2] = fmaf(w.x, w.x, fmaf(w.y, w.y, acc.v[ST_X2]));
    acc.v[ST_DX2] = fmaf(u.x, w.x, fmaf(u.y, w.y, acc.v[ST_DX2]));
    return w;
  }
};

// Complex-n geometry: p is the spatial index itself.
template <> struct Epi<COL_ADMM_INIT> {
  static constexpr bool kRead = false, kFwd = true;
  __device__ static float2 apply(const KParams&, const CallArgs& a, float2, int p, int t, Acc&) {
    return make_float2(__ldg(a.v + t), __ldg(a.z + t) - __ldg(a.nu + t));
  }
};

// Algorithm 3, after the x-update: v = D(rho C x - rho mu + P^T y),
// z = eta_{lambda/sigma}(x + nu), mu += tau1 (v - C x), nu += tau2 (x - z),
// v <- v + mu; the next x-update reads (v) + i (z - nu).
template <bool FWD, bool SEG = false> struct EpiAdmm {
  static constexpr bool kRead = true, kFwd = FWD;
  __device__ static float2 apply(const KParams& kp, const CallArgs& a, float2 xc, int p, int t, Acc& acc) {
    RowSel rs{acc.smask, acc.spref, acc.wbase};
    int iy;
    const bool on = rs.get(t, iy);
    const float yv = on ? __ldg(kp.pp.ys + iy) : 0.f;
    const float x = xc.x, cx = xc.y;
    // read-once / write-once per element by its own thread: read-only path (as EpiIsta)
    const float mu = __ldg(a.mu + t), nu = __ldg(a.nu + t);
    const float d = on ? a.d_on : a.d_off;
    const float v = d * fmaf(a.rho, cx - mu, yv);
    const float z = soft(x + nu, a.thr);
    if constexpr (SEG) a.aux[t] = x + nu;   // the soft threshold's input, for the reverse pass
    const float mu2 = fmaf(a.tau1, v - cx, mu);
    const float nu2 = fmaf(a.tau2, x - z, nu);
    const float vf = v + mu2;
    a.mu[t] = mu2;
    a.nu[t] = nu2;
    if (kp.flags & FL_WRITE_STATE) {
      a.z[t] = z;
      a.v[t] = vf;
      if (a.x) a.x[t] = x;
    }
    if (kp.flags & FL_STATS) {
      if (a.xtrue) {
        const float e = z - __ldg(a.xtrue + t);
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
template <> struct Epi<COL_ADMM_SEG> : EpiAdmm<true, true> {};

template <> struct Epi<COL_STORE_RE> {
  static constexpr bool kRead = true, kFwd = false;
  __device__ static float2 apply(const KParams&, const CallArgs& a, float2 v, int p, int t, Acc&) {
    a.dst[p] = v.x;
    return v;
  }
};

// ------------------------------------------------ unrolled-ADMM gradient
// Reverse mode of one Algorithm 3 iteration (state (v, z, mu, nu) -> (v2,
// z1, mu1, nu1), see the forward epilogue above).  The inverse FFT brings
// b' = B x' and C b' of the later iteration, which give the adjoints of the
// new state: v2' = rho C b', z1' = sigma b' (+ dL/dz(T) at the last
// iteration), mu1' (kept in mu) and nu1' = (kept in nu) - sigma b'.  Then
//   mu1' += v2',  v1' = v2' + tau1 mu1',  p' = -tau1 mu1',  x' = tau2 nu1',
//   z1' -= tau2 nu1',  s' = z1' on {|s| > lam/sigma},  x' += s',  nu' = nu1' + s',
//   a' = D v1',  p' += rho a',  mu' = mu1' - rho a',  y' += P a',
// with dL/dlam += -sum sign(s) s' / sigma (per-CTA partials; the host applies
// 1/sigma).  mu' and nu' (without its -sigma b' term, added by the earlier
// iteration's pass) go back to mu and nu; p' + i x' is transformed for the
// mid pass, which forms x' + C^T p' and b' = B(...) there.  CallArgs: mu, nu
// the adjoint state, aux = s of this iteration, v = dL/dy (compact rows, tile
// order), src = dL/dz(T) and xtrue = dL/dx(T) at the last iteration only.
template <> struct Epi<COL_ADMM_REV> {
  static constexpr bool kRead = true, kFwd = true;
  __device__ static float2 apply(const KParams&, const CallArgs& a, float2 bc, int p, int t, Acc& acc) {
    RowSel rs{acc.smask, acc.spref, acc.wbase};
    int iy;
    const bool on = rs.get(t, iy);
    const float b = bc.x, cb = bc.y;
    const float vb = a.rho * cb;
    float zb = a.sigma * b;
    if (a.src) zb += __ldg(a.src + t);
    float mub = a.mu[t] + vb;
    float nub = fmaf(-a.sigma, b, a.nu[t]);
    const float v1b = fmaf(a.tau1, mub, vb);
    float pb = -a.tau1 * mub;
    float xb = a.tau2 * nub;
    if (a.xtrue) xb += __ldg(a.xtrue + t);
    zb = fmaf(-a.tau2, nub, zb);
    const float sv = __ldg(a.aux + t);
    const float sb = fabsf(sv) > a.thr ? zb : 0.f;
    acc.v[0] -= sgnf(sv) * sb;
    xb += sb;
    nub += sb;
    const float ab = (on ? a.d_on : a.d_off) * v1b;
    pb = fmaf(a.rho, ab, pb);
    mub = fmaf(-a.rho, ab, mub);
    if (on) a.v[iy] += ab;   // each compact row belongs to one element: plain read-modify-write
    a.mu[t] = mub;
    a.nu[t] = nub;
    return make_float2(pb, xb);
  }
};

// ------------------------------------------------ unrolled-ISTA gradient
// Reverse mode of T steps x(t+1) = eta_theta(u(t)), u(t) = x(t) + tau C^T r(t),
// r(t) = M (P^T y - C x(t)).  With g = dL/dx(t+1) and w = g on the support
// of x(t+1) (the support of the soft threshold's derivative: x(t+1) != 0
// exactly when |u(t)| > theta, and then sign u(t) = sign x(t+1)):
//   dL/dx(t) = w - tau C^T M C w,  dL/dtheta += -sum sign(x(t+1)) w,
//   dL/dy += tau P C w,  dL/dc_k += tau sum_i (r_i w_{i+k} - q_i x(t)_{i+k})
// with q = M C w.  CallArgs of one step: x = x(t), z = x(t+1), v = r(t),
// mu = w, nu = q, dst = g, aux = dL/dy (compact, tile order of the rows); all
// n-vectors packed float2 in tile order.

template <> struct Epi<COL_LOADT> {
  static constexpr bool kRead = false, kFwd = true;
  __device__ static float2 apply(const KParams&, const CallArgs& a, float2, int p, int t, Acc&) {
    return ld2(a.x, t);
  }
};

template <> struct Epi<COL_RES_SAVE> {
  static constexpr bool kRead = true, kFwd = true;
  __device__ static float2 apply(const KParams& kp, const CallArgs& a, float2 v, int p, int t, Acc& acc) {
    RowSel rs{acc.smask, acc.spref, acc.wbase};
    int i0;
    const uint32_t mm = rs.get2(t, i0);
    const float r0 = (mm & 1u) ? __ldg(kp.pp.ys + i0) - v.x : 0.f;
    const float r1 = (mm & 2u) ? __ldg(kp.pp.ys + i0 + (int)(mm & 1u)) - v.y : 0.f;
    const float2 r = make_float2(r0, r1);
    st2(a.v, t, r);
    return r;
  }
};

template <> struct Epi<COL_ISTA_SEG> {
  static constexpr bool kRead = true, kFwd = true;
  __device__ static float2 apply(const KParams&, const CallArgs& a, float2 g, int p, int t, Acc&) {
    const float2 xo = ld2(a.x, t);
    const float2 xn = make_float2(soft(fmaf(a.tau, g.x, xo.x), a.thr), soft(fmaf(a.tau, g.y, xo.y), a.thr));
    st2(a.z, t, xn);
    return xn;
  }
};


template <> struct Epi<COL_GRAD_W> {
  static constexpr bool kRead = false, kFwd = true;
  __device__ static float2 apply(const KParams&, const CallArgs& a, float2, int p, int t, Acc& acc) {
    const float2 g = ld2(a.dst, t), xn = ld2(a.z, t);
    const float2 w = make_float2(xn.x != 0.f ? g.x : 0.f, xn.y != 0.f ? g.y : 0.f);
    acc.v[0] -= sgnf(xn.x) * w.x + sgnf(xn.y) * w.y;
    st2(a.mu, t, w);
    return w;
  }
};

template <> struct Epi<COL_GRAD_MASK> {
  static constexpr bool kRead = true, kFwd = true;
  __device__ static float2 apply(const KParams&, const CallArgs& a, float2 v, int p, int t, Acc& acc) {
    RowSel rs{acc.smask, acc.spref, acc.wbase};
    int i0;
    const uint32_t mm = rs.get2(t, i0);
    // each compact row index belongs to one element: plain read-modify-write
    if (mm & 1u) a.aux[i0] = fmaf(a.tau, v.x, a.aux[i0]);
    if (mm & 2u) a.aux[i0 + (int)(mm & 1u)] = fmaf(a.tau, v.y, a.aux[i0 + (int)(mm & 1u)]);
    const float2 q = make_float2((mm & 1u) ? v.x : 0.f, (mm & 2u) ? v.y : 0.f);
    st2(a.nu, t, q);
    return q;
  }
};

template <> struct Epi<COL_GRAD_G> {
  static constexpr bool kRead = true, kFwd = false;
  __device__ static float2 apply(const KParams&, const CallArgs& a, float2 v, int p, int t, Acc&) {
    const float2 w = ld2(a.mu, t);
    const float2 g = make_float2(fmaf(-a.tau, v.x, w.x), fmaf(-a.tau, v.y, w.y));
    st2(a.dst, t, g);
    return g;
  }
};

// (r, w) -> (W, W2); with FL_PAIR2 (q, x(t)) -> (W, W2)
template <> struct Epi<COL_LOAD2> {
  static constexpr bool kRead = false, kFwd = true;
  __device__ static float2 apply(const KParams& kp, const CallArgs& a, float2, int p, int t, Acc&) {
    return ld2((kp.flags & FL_PAIR2) ? a.nu : a.v, t);
  }
  __device__ static float2 apply2(const KParams& kp, const CallArgs& a, int t) {
    return ld2((kp.flags & FL_PAIR2) ? a.x : a.mu, t);
  }
};

template <int TILE> struct Cfg {
  static constexpr int NT = TILE / EPT;                 // threads per CTA
  static constexpr int MINB = 65536 / (64 * NT);        // mid pass: CTAs per SM at <= 64 registers
  static constexpr int NLD = TILE / (2 * NT);           // float4 loads per thread per tile
};

// Programmatic dependent launch: every pass kernel lets the next kernel in the
// stream start launching as soon as all of its own CTAs are running
// (pdl_trigger at entry), and waits for the previous kernel to finish
// (pdl_wait) only before its first read of data produced upstream; what it
// does before that reads plan constants only.  Outside a programmatic launch
// both are no-ops.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename K>
cudaError_t launch_k(K kern, int grid, int tile, const KParams& kp, cudaStream_t s, int smem_mult = 1) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(tile / EPT);
  cfg.dynamicSmemBytes = smem_mult * pass_smem_bytes(tile);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, kp);
}

// Opt a kernel into its dynamic shared memory and ask for a carveout just
// large enough for `ctas` resident CTAs, leaving the rest of the unified
// L1 / shared array to L1 (where the twiddle tables live).
template <typename K>
cudaError_t set_smem(K kern, int tile, int ctas, int smem_mult = 1) {
  const size_t dyn = smem_mult * pass_smem_bytes(tile);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  const size_t per_cta = dyn + fa.sharedSizeBytes + 1024;
  int pct = (int)((per_cta * ctas * 100 + 228 * 1024 - 1) / (228 * 1024));
  if (pct > 100) pct = 100;
  return cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

}  // namespace
}  // namespace csk
