// Mid pass of the fused FFT iteration: forward length-N1 FFTs along the rows
// of the N2 x N1 exchange array (with the four-step twiddle), the spectrum
// operator over every (k, N - k) pair, and the inverse FFTs.
#include "cs_passes.cuh"

namespace csk {

namespace {

// ---------------------------------------------------------------- mid pass

// w_N^(j1 k2) from the two-level table: w_N^p = w_N^(p mod N1) * w_N2^(p div N1)
__device__ __forceinline__ float2 tw4(const Geo& g, int p) {
  return cmul(__ldg(g.twl + (p & (g.N1 - 1))), __ldg(g.tw2 + (p >> g.lgN1)));
}

__device__ __forceinline__ int slot_row(const Geo& g, int u, int second) {
  if (u == 0) return second ? (g.N2 >> 1) : 0;
  return second ? g.N2 - u : u;
}

// Global source / sink of the first forward and last inverse FFT stages of
// the static shapes: row `vec` of the tile is row slot_row(u0 + vec/2,
// vec & 1) of the N2 x N1 exchange array.
struct MidIO {
  static constexpr bool kGlobal = true;
  float2* W;
  int u0, lgN1, N2;
  __device__ __forceinline__ float2* at(int vec, int idx) const {
    const int u = u0 + (vec >> 1);
    const int k2 = u == 0 ? ((vec & 1) ? (N2 >> 1) : 0) : ((vec & 1) ? N2 - u : u);
    return W + ((size_t)k2 << lgN1) + idx;
  }
  __device__ __forceinline__ float2 load(int vec, int idx) const { return __ldcg(at(vec, idx)); }
  __device__ __forceinline__ void store(int vec, int idx, float2 v) const { __stcg(at(vec, idx), v); }
};

// Four-step twiddle as FFT hooks: w_N^(j1 k2) on the values the first
// forward stage loads, its conjugate on the values the last inverse stage
// produces (k2 = the tile row's index in the N2 x N1 array).  With
// j1 = j + r L/R:  w_N^(j1 k2) = w_N^(j k2) * w_N^(r (L/R) k2); the second
// factor comes from a per-CTA table rt[row][r] in shared memory.
constexpr int MID_MAX_ROWS = 64;   // 2U <= min(N2, TILE/N1) <= 64 rows, as N2 <= N1

// Static shapes: w_N^(j1 k2) = lo[j1 mod 16] * hi[j1 div 16], two per-row
// tables of 16 and N1/16 entries (both exact FP64-rounded values).  With
// j1 = j + r L/R and L/R >= 16, lo depends on the thread only and hi is read
// at (j div 16) + r (L/R)/16.
template <bool PRE>
struct MidTwHookS {
  static constexpr bool kPre = PRE, kPost = !PRE;
  const float2* lo;   // [rows][16]
  const float2* hi;   // [rows][N1/16]
  int lgN1;
  float2 wl;
  __device__ __forceinline__ void begin(int vec, int j) { wl = lo[vec * 16 + (j & 15)]; }
  __device__ __forceinline__ float2 tw(int vec, int j, int r, int lgLR) const {
    return cmul(wl, hi[(vec << (lgN1 - 4)) + (j >> 4) + (r << (lgLR - 4))]);
  }
  __device__ __forceinline__ float2 pre(int vec, int j, int r, int lgLR, float2 v) const {
    return cmul(v, tw(vec, j, r, lgLR));
  }
  __device__ __forceinline__ float2 post(int vec, int j, int r, int lgLR, float2 v) {
    return cmulc(v, tw(vec, j, r, lgLR));
  }
};

template <bool PRE>
struct MidTwHook {
  static constexpr bool kPre = PRE, kPost = !PRE;
  const Geo& g;
  int u0;
  const float2* rt;   // [2U][16]
  float2 wj;
  __device__ __forceinline__ void begin(int vec, int j) {
    wj = tw4(g, j * slot_row(g, u0 + (vec >> 1), vec & 1));
  }
  __device__ __forceinline__ float2 pre(int vec, int, int r, int, float2 v) const {
    return cmul(v, cmul(wj, rt[vec * 16 + r]));
  }
  __device__ __forceinline__ float2 post(int vec, int, int r, int, float2 v) {
    return cmulc(v, cmul(wj, rt[vec * 16 + r]));
  }
};
// Real-FFT spectrum operator (products with C and C^T on the packed vector).
// For the pair (k, N - k) of the packed spectrum Z, with H the real-signal
// spectrum of the product (H = chat for C^T, conj(chat) for C):
//   Z'_k   = a  Z_k   + b  conj(Z_{N-k})
//   Z'_N-k = a' Z_N-k + b' conj(Z_k),   b' = -conj(b)
// with, for H = chat, P = (H_k + H_{k+N})/2N, Q = (H_k - H_{k+N})/2N (the
// table, FP64-rounded once) and the packing phase w = exp(-i theta),
// theta = 2 pi k / 2N:  a = P - Q sin(theta), a' = conj(P + Q sin(theta)),
// b = i Q cos(theta).  H = conj(chat) conjugates a and a' and maps
// b -> -conj(b).  w = w_2N^k is the product of two small tables (1D:
// twr[k2] tw1[k1]; 2D, where the phase is that of the packed axis only:
// tw1[k1]).
template <bool ADJ>
__device__ __forceinline__ void op_real(const PlanPtrs& pp, int tidx, float2 w, float2& za, float2& zb) {
  const float4 t = __ldg(pp.tab_ista + tidx);
  const float2 P = make_float2(t.x, t.y), Q = make_float2(t.z, t.w);
  // sin(theta) = -w.y, cos(theta) = w.x
  float2 al = make_float2(fmaf(w.y, Q.x, P.x), fmaf(w.y, Q.y, P.y));
  float2 al2 = make_float2(fmaf(-w.y, Q.x, P.x), -fmaf(-w.y, Q.y, P.y));
  float2 be = make_float2(-w.x * Q.y, w.x * Q.x);
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
__device__ __forceinline__ void op_admm(const PlanPtrs& pp, float rho, float sigma, int tidx,
                                        float2& za, float2& zb) {
  const float2 ch = __ldg(pp.tab_admm_c + tidx);
  const float bb = __ldg(pp.tab_admm_b + tidx);
  const float2 V = make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y - zb.y));
  const float2 Wk = make_float2(0.5f * (za.y + zb.y), -0.5f * (za.x - zb.x));
  const float2 cv = cmul(ch, V);
  const float2 X = make_float2(bb * fmaf(rho, cv.x, sigma * Wk.x),
                               bb * fmaf(rho, cv.y, sigma * Wk.y));
  const float2 Pc = cmulc(X, ch);
  za = make_float2(X.x - Pc.y, X.y + Pc.x);
  zb = make_float2(X.x + Pc.y, Pc.x - X.y);
}

// SHAPE 0: any geometry; SHAPE s > 0 fixes (log2 N1, log2 U) at compile time
// for the geometries of N = 2^20 (1024 x 1024, U = 2), 2^21 (2048 x 1024,
// U = 1) and 2^22 (4096 x 1024, U = 1).
// SHAPE 4..6: the same for a 2D DFT (no four-step twiddle; see Geo::twod):
// 4 any geometry, 5 and 6 fix (log2 N1, log2 U) = (11, 0) and (12, 0), the
// packed and the complex geometry of a 4096 x 4096 image.
template <int SHAPE> struct MidShape;
template <> struct MidShape<0> {
  using Lay = DynLayout;
  static constexpr bool kTwoD = false;
  __device__ static Lay lay(const Geo& g) { return Lay{g.lgN1, g.lgU + 1, false}; }
  __device__ static int lgN1(const Geo& g) { return g.lgN1; }
  __device__ static int lgU(const Geo& g) { return g.lgU; }
};
template <int LGN1, int LGU, bool TWOD = false> struct MidShapeS {
  using Lay = StaticLayout<LGN1, LGU + 1, false>;
  static constexpr bool kTwoD = TWOD;
  __device__ static Lay lay(const Geo&) { return Lay{}; }
  __device__ static constexpr int lgN1(const Geo&) { return LGN1; }
  __device__ static constexpr int lgU(const Geo&) { return LGU; }
};
template <> struct MidShape<1> : MidShapeS<10, 1> {};
template <> struct MidShape<2> : MidShapeS<11, 0> {};
template <> struct MidShape<3> : MidShapeS<12, 0> {};
template <> struct MidShape<4> : MidShape<0> { static constexpr bool kTwoD = true; };
template <> struct MidShape<5> : MidShapeS<11, 0, true> {};
template <> struct MidShape<6> : MidShapeS<12, 0, true> {};

// The mid pass of tile `blk` (row-pair units blk U .. blk U + U - 1).
template <int KIND, int TILE, int SHAPE>
__device__ __forceinline__ void mid_body(const KParams& kp, const int blk) {
  constexpr int NT = Cfg<TILE>::NT;
  constexpr int NLD = Cfg<TILE>::NLD;
  using S = MidShape<SHAPE>;
  extern __shared__ float2 sm[];
  pdl_trigger();
  const Geo& g = kp.geo;
  const int lgU = S::lgU(g), U = 1 << lgU;
  const int u0 = blk << lgU;
  const int lgN1 = S::lgN1(g), N1 = 1 << lgN1;
  const int tot = (2 * U) << lgN1;
  const auto lay = S::lay(g);
  float2* __restrict__ W = kp.pp.W;
  constexpr bool TWS = S::Lay::kStatic;   // static shape: twiddles in shared memory
  constexpr bool TWOD = S::kTwoD;         // 2D DFT: no four-step twiddle hooks
  constexpr int LGN1S = TWS ? S::lgN1(Geo{}) : 4;
  constexpr int ROWS = TWS ? (2 << S::lgU(Geo{})) : MID_MAX_ROWS;
  constexpr int TW_N = TWS ? stage_tw_count(LGN1S) : 2;
  __shared__ __align__(16) float2 tws[TW_N];
  // static shapes: per-row lo[16] and hi[N1/16]; dynamic: rt (see MidTwHook)
  constexpr int LOHI = (TWS && !TWOD) ? ROWS * (16 + (1 << (LGN1S - 4))) : 2;
  __shared__ float2 lohi[LOHI];
  __shared__ float2 rt[2][(TWS || TWOD) ? 2 : MID_MAX_ROWS * 16];
  if (TWS) copy_table<NT>(tws, g.tws1, TW_N);
  if constexpr (TWOD) {
  } else if (TWS) {
    constexpr int HI = 1 << (LGN1S - 4);
    for (int t = threadIdx.x; t < ROWS * (16 + HI); t += NT) {
      const bool is_lo = t < ROWS * 16;
      const int tt = is_lo ? t : t - ROWS * 16;
      const int vec = is_lo ? (tt >> 4) : (tt >> (LGN1S - 4));
      const int q = is_lo ? (tt & 15) : (tt & (HI - 1)) << 4;
      const int k2 = slot_row(g, u0 + (vec >> 1), vec & 1);
      lohi[t] = tw4(g, (q * k2) & (g.N - 1));
    }
  } else {
    // rt[0][row][r] = w_N^(r (L/R) k2) for R the radix of the first stage (the
    // forward pre-hook), rt[1] for the radix of the last stage (inverse post-hook)
    const int lgRf = lgN1 >= 4 ? 4 : lgN1;
    const int lgRl = (lgN1 & 3) ? (lgN1 & 3) : 4;
    for (int t = threadIdx.x; t < 2 * 2 * U * 16; t += NT) {
      const int which = t / (2 * U * 16);
      const int tt = t - which * (2 * U * 16);
      const int vec = tt >> 4, r = tt & 15;
      const int lgR = which ? lgRl : lgRf;
      const int k2 = slot_row(g, u0 + (vec >> 1), vec & 1);
      rt[which][tt] = r < (1 << lgR) ? tw4(g, ((r << (lgN1 - lgR)) * k2) & (g.N - 1)) : make_float2(1.f, 0.f);
    }
  }
  pdl_wait();   // the twiddle tables above are plan constants; W is not
  const float a_rho = kp.ca->rho, a_sigma = kp.ca->sigma;   // ADMM only
  auto load_tile = [&](float2* dst, const float2* __restrict__ src) {
    float4 buf[NLD];
#pragma unroll
    for (int i = 0; i < NLD; ++i) {
      const int e = 2 * (threadIdx.x + i * NT);
      if (e < tot) {
        const int slot = e >> lgN1, j1 = e & (N1 - 1);
        const int k2 = slot_row(g, u0 + (slot >> 1), slot & 1);
        buf[i] = __ldcg(reinterpret_cast<const float4*>(src + ((size_t)k2 << lgN1) + j1));
      }
    }
#pragma unroll
    for (int i = 0; i < NLD; ++i) {
      const int e = 2 * (threadIdx.x + i * NT);
      if (e < tot) {
        dst[pad(e)] = make_float2(buf[i].x, buf[i].y);
        dst[pad(e + 1)] = make_float2(buf[i].z, buf[i].w);
      }
    }
    __syncthreads();
  };
  // static shapes: the first forward stage reads the rows from W itself
  // (after a barrier: its hook reads the twiddle tables written above)
  auto fwd_rows_from_global = [&]() {
    if constexpr (TWS) {
      __syncthreads();
      const MidIO io{W, u0, lgN1, g.N2};
      if constexpr (TWOD) {
        NoHook nh;
        tile_fft<-1, TILE, NT, true>(sm, lay, tws, lgN1, nh, io, SmemIO{});
      } else {
        MidTwHookS<true> h{lohi, lohi + ROWS * 16, LGN1S, make_float2(1.f, 0.f)};
        tile_fft<-1, TILE, NT, true>(sm, lay, tws, lgN1, h, io, SmemIO{});
      }
    }
  };
  auto fwd_rows = [&](float2* buf) {
    if constexpr (TWOD) {
      if constexpr (TWS) tile_fft<-1, TILE, NT, true>(buf, lay, tws, lgN1);
      else tile_fft<-1, TILE, NT, false>(buf, lay, g.tw1h, lgN1);
    } else if constexpr (TWS) {
      MidTwHookS<true> h{lohi, lohi + ROWS * 16, LGN1S, make_float2(1.f, 0.f)};
      tile_fft<-1, TILE, NT, true>(buf, lay, tws, lgN1, h);
    } else {
      MidTwHook<true> h{g, u0, rt[0], make_float2(1.f, 0.f)};
      tile_fft<-1, TILE, NT, false>(buf, lay, g.tw1, lgN1 + 1, h);
    }
  };
  // Pair slot t of this CTA: elements ea (frequency k = k2 + N2 k1) and eb
  // (frequency N - k) of the tile, table index tidx.
  const int nslots = (U << lgN1) + (u0 == 0 ? (TWOD ? 2 : 1) : 0);
  const int base_u1 = ((g.N2 >> 1) - 1) << lgN1;   // table offset of unit 0
  auto slot_at = [&](int t, int& ea, int& eb, int& k2, int& k1, int& tidx) {
    int ul, q;
    if (t < (U << lgN1)) { ul = t >> lgN1; q = t & (N1 - 1); }
    else { ul = 0; q = N1 + (t - (U << lgN1)); }
    const int u = u0 + ul;
    if constexpr (TWOD) {
      // 2D partner of (k2, k1): (-k2, -k1); unit 0: rows 0 and N2/2, each
      // with N1/2 + 1 slots q -> (q, (N1 - q) mod N1)
      if (u > 0) {
        k2 = u; k1 = q;
        ea = ((2 * ul) << lgN1) + q;
        eb = ((2 * ul + 1) << lgN1) + ((N1 - q) & (N1 - 1));
        tidx = ((u - 1) << lgN1) + q;
      } else {
        const bool hi = q > (N1 >> 1);
        const int qq = hi ? q - (N1 >> 1) - 1 : q;
        k2 = hi ? (g.N2 >> 1) : 0; k1 = qq;
        ea = ((2 * ul + (hi ? 1 : 0)) << lgN1) + qq;
        eb = ((2 * ul + (hi ? 1 : 0)) << lgN1) + ((N1 - qq) & (N1 - 1));
        tidx = base_u1 + q;
      }
      return;
    }
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
  };

  if constexpr (KIND == MID_CORR) {
    // Spectra of two packed real vectors a (W) and b (W2).  From the pair
    // (Z_k, Z_{N-k}) of a packed spectrum: E = (Z_k + conj Z_{N-k}) / 2,
    // O = (Z_k - conj Z_{N-k}) / 2i, and the length-2N real spectrum is
    // a^_k = E + w O, a^_{k+N} = E - w O, w = exp(-2 pi i k / 2N).
    float2* sm2 = sm + smem_slots(TILE);
    load_tile(sm, W);
    fwd_rows(sm);
    load_tile(sm2, kp.pp.W2);
    fwd_rows(sm2);
    const float sgn = (kp.flags & FL_PAIR2) ? -1.f : 1.f;
    for (int t = threadIdx.x; t < nslots; t += NT) {
      int ea, eb, k2, k1, tidx;
      slot_at(t, ea, eb, k2, k1, tidx);
      const float2 w = cmul(__ldg(g.twr + k2), __ldg(g.tw1 + k1));
      float2 sa[2], sb[2];
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        const float2* bufv = v ? sm2 : sm;
        const float2 za = bufv[pad(ea)], zb = bufv[pad(eb)];
        const float2 E = make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y - zb.y));
        const float2 O = make_float2(0.5f * (za.y + zb.y), -0.5f * (za.x - zb.x));
        const float2 wo = cmul(w, O);
        float2* dst = v ? sb : sa;
        dst[0] = cadd(E, wo);
        dst[1] = csub(E, wo);
      }
      const float2 p0 = cmulc(sb[0], sa[0]), p1 = cmulc(sb[1], sa[1]);   // conj(a^) b^
      float4 acc = kp.pp.gacc[tidx];
      acc.x = fmaf(sgn, p0.x, acc.x);
      acc.y = fmaf(sgn, p0.y, acc.y);
      acc.z = fmaf(sgn, p1.x, acc.z);
      acc.w = fmaf(sgn, p1.y, acc.w);
      kp.pp.gacc[tidx] = acc;
    }
    return;
  } else if constexpr (KIND == MID_ADMM_REV) {
    // Reverse of the x-update of one Algorithm 3 iteration.  W holds the
    // column transform of p' + i x', W2 that of the iteration's forward pair
    // v + i (z - nu).  Per pair slot, with the k-side spectra P', X'l, V0, Wf
    // of the four real vectors: Xs = bhat (rho chat V0 + sigma Wf) and
    // Bs = bhat (chat P' + X'l) are the spectra of x and b' = B (C^T p' + x')
    // divided by N (bhat holds 1/N).  The spectrum of this iteration's dL/dc
    // divided by N,
    //   A = conj(P') Xs + rho conj(V0) Bs - 2 rho N chat Re(conj(Xs) Bs),
    // is added to gacc_a (DFT of sum_i a_i b_{i+k} = conj(a^) b^; the B-term
    // pairs C x with b' and C b' with x, whose sum is real times chat), and
    // Bs + i conj(chat) Bs goes back for the inverse: b' + i C b'.
    float2* sm2 = sm + smem_slots(TILE);
    load_tile(sm, W);
    fwd_rows(sm);
    load_tile(sm2, kp.pp.W2);
    fwd_rows(sm2);
    const float rho = kp.ca->rho, sigma = kp.ca->sigma;
    const float nN = (float)g.N;
    for (int t = threadIdx.x; t < nslots; t += NT) {
      int ea, eb, k2, k1, tidx;
      slot_at(t, ea, eb, k2, k1, tidx);
      const float2 za = sm[pad(ea)], zb = sm[pad(eb)];
      const float2 fa = sm2[pad(ea)], fb = sm2[pad(eb)];
      const float2 Pb = make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y - zb.y));
      const float2 Xl = make_float2(0.5f * (za.y + zb.y), -0.5f * (za.x - zb.x));
      const float2 V0 = make_float2(0.5f * (fa.x + fb.x), 0.5f * (fa.y - fb.y));
      const float2 Wf = make_float2(0.5f * (fa.y + fb.y), -0.5f * (fa.x - fb.x));
      const float2 ch = __ldg(kp.pp.tab_admm_c + tidx);
      const float bb = __ldg(kp.pp.tab_admm_b + tidx);
      const float2 cv = cmul(ch, V0);
      const float2 Xs = make_float2(bb * fmaf(rho, cv.x, sigma * Wf.x), bb * fmaf(rho, cv.y, sigma * Wf.y));
      const float2 cp = cmul(ch, Pb);
      const float2 Bs = make_float2(bb * (cp.x + Xl.x), bb * (cp.y + Xl.y));
      const float2 t1 = cmulc(Xs, Pb);
      const float2 t2 = cmulc(Bs, V0);
      const float sc = -2.f * rho * nN * fmaf(Xs.x, Bs.x, Xs.y * Bs.y);
      const float2 acc = kp.pp.gacc_a[tidx];
      kp.pp.gacc_a[tidx] = make_float2(acc.x + fmaf(rho, t2.x, fmaf(sc, ch.x, t1.x)),
                                       acc.y + fmaf(rho, t2.y, fmaf(sc, ch.y, t1.y)));
      const float2 Pc = cmulc(Bs, ch);
      sm[pad(eb)] = make_float2(Bs.x + Pc.y, Pc.x - Bs.y);   // self-pairs keep the k-side value
      sm[pad(ea)] = make_float2(Bs.x - Pc.y, Bs.y + Pc.x);
    }
    __syncthreads();
  } else if constexpr (KIND == MID_ADMM_FROM_ACC) {
    // dL/dc = the inverse transform of the accumulated Hermitian spectrum
    for (int t = threadIdx.x; t < nslots; t += NT) {
      int ea, eb, k2, k1, tidx;
      slot_at(t, ea, eb, k2, k1, tidx);
      const float2 A = kp.pp.gacc_a[tidx];
      sm[pad(eb)] = cconj(A);
      sm[pad(ea)] = A;
    }
    __syncthreads();
  } else if constexpr (KIND == MID_FROM_ACC) {
    // The packed spectrum of the real vector d whose length-2N spectrum is
    // gacc (D_k, D_{k+N} per slot), times tau / N for the unnormalised
    // inverse:  E' = (D_k + D_{k+N}) / 2,  O' = conj(w) (D_k - D_{k+N}) / 2,
    // Z'_k = E' + i O',  Z'_{N-k} = conj(E') + i conj(O').
    const float sc = kp.ca->tau / (float)g.N;
    for (int t = threadIdx.x; t < nslots; t += NT) {
      int ea, eb, k2, k1, tidx;
      slot_at(t, ea, eb, k2, k1, tidx);
      const float2 w = cmul(__ldg(g.twr + k2), __ldg(g.tw1 + k1));
      const float4 d = kp.pp.gacc[tidx];
      const float2 d0 = make_float2(d.x, d.y), d1 = make_float2(d.z, d.w);
      const float2 E = cscale(cadd(d0, d1), 0.5f);
      const float2 O = cscale(cmulc(csub(d0, d1), w), 0.5f);
      const float2 za = make_float2(E.x - O.y, E.y + O.x);
      const float2 zb = make_float2(E.x + O.y, O.x - E.y);
      sm[pad(eb)] = cscale(zb, sc);   // self-pairs (ea == eb): both sides agree
      sm[pad(ea)] = cscale(za, sc);
    }
    __syncthreads();
  } else {
    if constexpr (TWS) {
      fwd_rows_from_global();
    } else {
      load_tile(sm, W);
      fwd_rows(sm);
    }
    // spectrum operator over all (k, N-k) pairs held by this CTA (unrolled so
    // that the table loads of several slots are in flight together)
#pragma unroll 8
    for (int t = threadIdx.x; t < nslots; t += NT) {
      int ea, eb, k2, k1, tidx;
      slot_at(t, ea, eb, k2, k1, tidx);
      float2 za = sm[pad(ea)], zb = sm[pad(eb)];
      if (KIND == MID_ADMM) {
        op_admm(kp.pp, a_rho, a_sigma, tidx, za, zb);
      } else {
        const float2 w = TWOD ? __ldg(g.tw1 + k1) : cmul(__ldg(g.twr + k2), __ldg(g.tw1 + k1));
        op_real<KIND == MID_ADJ>(kp.pp, tidx, w, za, zb);
      }
      sm[pad(eb)] = zb;   // self-pairs (ea == eb) keep the k-side value
      sm[pad(ea)] = za;
    }
    __syncthreads();
  }
  if constexpr (TWS) {
    // static shapes: the last inverse stage writes the rows to W itself
    const MidIO io{W, u0, lgN1, g.N2};
    if constexpr (TWOD) {
      NoHook nh;
      tile_fft<+1, TILE, NT, true>(sm, lay, tws, lgN1, nh, SmemIO{}, io);
    } else {
      MidTwHookS<false> h{lohi, lohi + ROWS * 16, LGN1S, make_float2(1.f, 0.f)};
      tile_fft<+1, TILE, NT, true>(sm, lay, tws, lgN1, h, SmemIO{}, io);
    }
    return;
  } else {
    if constexpr (TWOD) {
      tile_fft<+1, TILE, NT, false>(sm, lay, g.tw1h, lgN1);
    } else {
      MidTwHook<false> h{g, u0, rt[1], make_float2(1.f, 0.f)};
      tile_fft<+1, TILE, NT, false>(sm, lay, g.tw1, lgN1 + 1, h);
    }
  }

#pragma unroll
  for (int i = 0; i < NLD; ++i) {
    const int e = 2 * (threadIdx.x + i * NT);
    if (e < tot) {
      const int slot = e >> lgN1, j1 = e & (N1 - 1);
      const int k2 = slot_row(g, u0 + (slot >> 1), slot & 1);
      const float2 lo = sm[pad(e)], hi = sm[pad(e + 1)];
      __stcg(reinterpret_cast<float4*>(W + ((size_t)k2 << lgN1) + j1), make_float4(lo.x, lo.y, hi.x, hi.y));
    }
  }
}

template <int KIND, int TILE, int SHAPE>
__global__ void __launch_bounds__(Cfg<TILE>::NT, Cfg<TILE>::MINB) mid_kernel(const KParams kp) {
  mid_body<KIND, TILE, SHAPE>(kp, blockIdx.x);
}

// Grouped launch over many plans (batched solves): CTA b runs tile
// map[b].y of plan map[b].x (4096-value tiles, run-time shapes).
template <int KIND>
__global__ void __launch_bounds__(Cfg<4096>::NT, Cfg<4096>::MINB)
    mid_kernel_multi(const KParams* __restrict__ kps, const int2* __restrict__ map) {
  static_assert(sizeof(KParams) % 4 == 0 && sizeof(KParams) / 4 <= Cfg<4096>::NT, "KParams copy");
  __shared__ KParams skp;
  const int2 it = map[blockIdx.x];
  if (threadIdx.x < sizeof(KParams) / 4)
    reinterpret_cast<int*>(&skp)[threadIdx.x] = reinterpret_cast<const int*>(kps + it.x)[threadIdx.x];
  __syncthreads();
  mid_body<KIND, 4096, 0>(skp, it.y);
}

}  // namespace

#define CS_MID_KINDS(X, T, S)                                                                    \
  X(MID_FWD, T, S) X(MID_ADJ, T, S) X(MID_ADMM, T, S) X(MID_CORR, T, S) X(MID_FROM_ACC, T, S)       \
  X(MID_ADMM_REV, T, S) X(MID_ADMM_FROM_ACC, T, S)
#define CS_MID_KINDS_2D(X, T, S) X(MID_FWD, T, S) X(MID_ADJ, T, S) X(MID_ADMM, T, S)

// MID_CORR and MID_ADMM_REV hold two tiles in shared memory
constexpr int mid_smem_mult(int kind) { return (kind == MID_CORR || kind == MID_ADMM_REV) ? 2 : 1; }

cudaError_t init_mid_kernels() {
  cudaError_t e = cudaSuccess;
#define CS_SET_MID(k, T, S) \
  if (e == cudaSuccess) e = set_smem(mid_kernel<k, T, S>, T, Cfg<T>::MINB, mid_smem_mult(k));
  CS_MID_KINDS(CS_SET_MID, 4096, 0)
  CS_MID_KINDS(CS_SET_MID, 8192, 0)
  CS_MID_KINDS(CS_SET_MID, 4096, 1)
  CS_MID_KINDS(CS_SET_MID, 4096, 2)
  CS_MID_KINDS(CS_SET_MID, 8192, 3)
  CS_MID_KINDS_2D(CS_SET_MID, 4096, 4)
  CS_MID_KINDS_2D(CS_SET_MID, 8192, 4)
  CS_MID_KINDS_2D(CS_SET_MID, 4096, 5)
  CS_MID_KINDS_2D(CS_SET_MID, 8192, 6)
#undef CS_SET_MID
  return e;
}

cudaError_t launch_mid(MidKind kind, const KParams& kp, cudaStream_t s) {
  const Geo& g = kp.geo;
  const int grid = g.mid_ctas;
#define CS_L_MID(k, T, S) case k: return launch_k(mid_kernel<k, T, S>, grid, T, kp, s, mid_smem_mult(k));
  if (g.twod) {
    if (g.lgN1 == 11 && g.lgU == 0 && g.tile == 4096) {
      switch (kind) { CS_MID_KINDS_2D(CS_L_MID, 4096, 5) default: break; }
    } else if (g.lgN1 == 12 && g.lgU == 0 && g.tile == 8192) {
      switch (kind) { CS_MID_KINDS_2D(CS_L_MID, 8192, 6) default: break; }
    } else if (g.tile == 4096) {
      switch (kind) { CS_MID_KINDS_2D(CS_L_MID, 4096, 4) default: break; }
    } else {
      switch (kind) { CS_MID_KINDS_2D(CS_L_MID, 8192, 4) default: break; }
    }
    return cudaErrorInvalidValue;
  }
  int shape = 0;
  if (g.lgN1 == 10 && g.lgU == 1 && g.tile == 4096) shape = 1;
  if (g.lgN1 == 11 && g.lgU == 0 && g.tile == 4096) shape = 2;
  if (g.lgN1 == 12 && g.lgU == 0 && g.tile == 8192) shape = 3;
  switch (shape) {
    case 1: switch (kind) { CS_MID_KINDS(CS_L_MID, 4096, 1) } break;
    case 2: switch (kind) { CS_MID_KINDS(CS_L_MID, 4096, 2) } break;
    case 3: switch (kind) { CS_MID_KINDS(CS_L_MID, 8192, 3) } break;
    default:
      if (g.tile == 4096) { switch (kind) { CS_MID_KINDS(CS_L_MID, 4096, 0) } }
      else { switch (kind) { CS_MID_KINDS(CS_L_MID, 8192, 0) } }
  }
#undef CS_L_MID
  return cudaErrorInvalidValue;
}

#define CS_MID_KINDS_MULTI(X) X(MID_FWD) X(MID_ADJ) X(MID_ADMM)

cudaError_t init_mid_multi_kernels() {
  cudaError_t e = cudaSuccess;
#define CS_SET_MIDM(k) \
  if (e == cudaSuccess) e = set_smem(mid_kernel_multi<k>, 4096, Cfg<4096>::MINB);
  CS_MID_KINDS_MULTI(CS_SET_MIDM)
#undef CS_SET_MIDM
  return e;
}

cudaError_t launch_mid_multi(MidKind kind, const KParams* kps, const int2* map, int nctas, cudaStream_t s) {
  if (nctas < 1) return cudaSuccess;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(nctas);
  cfg.blockDim = dim3(Cfg<4096>::NT);
  cfg.dynamicSmemBytes = pass_smem_bytes(4096);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  switch (kind) {
    case MID_FWD: return cudaLaunchKernelEx(&cfg, mid_kernel_multi<MID_FWD>, kps, map);
    case MID_ADJ: return cudaLaunchKernelEx(&cfg, mid_kernel_multi<MID_ADJ>, kps, map);
    case MID_ADMM: return cudaLaunchKernelEx(&cfg, mid_kernel_multi<MID_ADMM>, kps, map);
    default: break;
  }
  return cudaErrorInvalidValue;
}

cudaError_t init_pass_kernels() {
  cudaError_t e = init_col_kernels();
  if (e == cudaSuccess) e = init_mid_kernels();
  if (e == cudaSuccess) e = init_col_multi_kernels();
  return e == cudaSuccess ? init_mid_multi_kernels() : e;
}

size_t pass_smem_bytes(int tile) { return sizeof(float2) * (size_t)smem_slots(tile); }

}  // namespace csk
