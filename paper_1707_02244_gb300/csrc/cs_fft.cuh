// Shared-memory Stockham FFT building blocks (fp32, sm_103a).
//
// A CTA holds TILE complex values in shared memory, arranged as `nvec`
// vectors of length L (a power of two).  One Stockham stage of radix R reads
// R values per butterfly at stride L/R, twiddles them, applies an in-register
// DFT_R and writes them back in auto-sorted order, so no bit reversal is ever
// needed.  Stages use radix 16 while log2(L) allows it and one radix-2/4/8
// stage for the remainder.  Every thread owns EPT = 16 values per stage
// (TILE = 16 * NT), which keeps a stage within 64 registers.
//
// Shared-memory index of linear element e is e + (e >> 4): one pad slot per
// 16 complex values keeps the stride-16 writes of the first stage free of
// bank conflicts.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace csk {

constexpr int EPT = 16;   // complex values per thread per stage

__host__ __device__ constexpr int smem_slots(int tile) { return tile + (tile >> 4); }

__device__ __forceinline__ int pad(int e) { return e + (e >> 4); }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by DIR*i  (DIR = -1 forward, +1 inverse)
template <int DIR>
__device__ __forceinline__ float2 mul_diri(float2 a) {
  return DIR > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// cos / sin of 2*pi*j/16, exact decimal expansions of the constants
__device__ __forceinline__ float cos16(int j) {
  constexpr float c1 = 0.92387953251128674f, r = 0.70710678118654752f, s1 = 0.38268343236508978f;
  switch (j & 15) {
    case 0: return 1.f;   case 1: return c1;   case 2: return r;    case 3: return s1;
    case 4: return 0.f;   case 5: return -s1;  case 6: return -r;   case 7: return -c1;
    case 8: return -1.f;  case 9: return -c1;  case 10: return -r;  case 11: return -s1;
    case 12: return 0.f;  case 13: return s1;  case 14: return r;   default: return c1;
  }
}
__device__ __forceinline__ float sin16(int j) { return cos16(j - 4); }

// a * exp(DIR * 2 pi i j / 16); j is a compile-time constant after unrolling
template <int DIR>
__device__ __forceinline__ float2 rot16(float2 a, int j) {
  j &= 15;
  if (j == 0) return a;
  if (j == 4) return mul_diri<DIR>(a);
  if (j == 8) return make_float2(-a.x, -a.y);
  if (j == 12) return mul_diri<-DIR>(a);
  return cmul(a, make_float2(cos16(j), DIR * sin16(j)));
}

// In-register DFT of length R in {2,4,8,16}: X_k = sum_r a_r exp(DIR 2 pi i r k / R).
// Computed in place; X_k ends in register slot out_slot<R>(k).
template <int R> __device__ __forceinline__ constexpr int out_slot(int k) {
  // R = 4 * Q (Q = R/4) for R >= 8: X[k1 + 4 k2] lands in a[Q k1 + k2]
  return R <= 4 ? k : (R / 4) * (k % 4) + k / 4;
}

template <int DIR>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 s02 = cadd(a0, a2), d02 = csub(a0, a2);
  const float2 s13 = cadd(a1, a3), d13 = mul_diri<DIR>(csub(a1, a3));
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, d13);
  a3 = csub(d02, d13);
}

template <int R, int DIR>
__device__ __forceinline__ void dft(float2* a) {
  if (R == 2) {
    const float2 t = a[1];
    a[1] = csub(a[0], t);
    a[0] = cadd(a[0], t);
  } else if (R == 4) {
    dft4<DIR>(a[0], a[1], a[2], a[3]);
  } else {
    // R = 4 * Q: n = Q n1 + n2, k = k1 + 4 k2
    constexpr int Q = R / 4;
#pragma unroll
    for (int n2 = 0; n2 < Q; ++n2) dft4<DIR>(a[n2], a[Q + n2], a[2 * Q + n2], a[3 * Q + n2]);
    // now a[Q k1 + n2] holds the length-4 transform; twiddle by w_R^(n2 k1)
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1)
#pragma unroll
      for (int n2 = 1; n2 < Q; ++n2) a[Q * k1 + n2] = rot16<DIR>(a[Q * k1 + n2], n2 * k1 * (16 / R));
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      if (Q == 2) {
        const float2 t = a[Q * k1 + 1];
        a[Q * k1 + 1] = csub(a[Q * k1], t);
        a[Q * k1] = cadd(a[Q * k1], t);
      } else {
        dft4<DIR>(a[Q * k1], a[Q * k1 + 1], a[Q * k1 + 2], a[Q * k1 + 3]);
      }
    }
  }
}

// Geometry of the vectors held in shared memory.
//   rows layout (vec_fast = false): element (vec, idx) at vec*L + idx
//   cols layout (vec_fast = true):  element (vec, idx) at idx*nvec + vec
// DynLayout carries the shape at run time; StaticLayout fixes it at compile
// time for the hot sizes, so every shared-memory address of a stage folds to
// a base register plus an immediate offset.
struct DynLayout {
  static constexpr bool kStatic = false;
  int lgL;      // log2 vector length
  int lgnv;     // log2 number of vectors
  bool vec_fast;
  __device__ __forceinline__ int LG() const { return lgL; }
  __device__ __forceinline__ int NV() const { return lgnv; }
  __device__ __forceinline__ bool VF() const { return vec_fast; }
  __device__ __forceinline__ int at(int vec, int idx) const {
    return vec_fast ? ((idx << lgnv) + vec) : ((vec << lgL) + idx);
  }
};

template <int LGL, int LGNV, bool VEC_FAST>
struct StaticLayout {
  static constexpr bool kStatic = true;
  static constexpr int kLgL = LGL, kLgNv = LGNV;
  __device__ __forceinline__ constexpr int LG() const { return LGL; }
  __device__ __forceinline__ constexpr int NV() const { return LGNV; }
  __device__ __forceinline__ constexpr bool VF() const { return VEC_FAST; }
  __device__ __forceinline__ int at(int vec, int idx) const {
    return VEC_FAST ? ((idx << LGNV) + vec) : ((vec << LGL) + idx);
  }
  // Padded index split: pad(at(vec, idx)) = padV(vec) + padP(idx), and
  // padP(a + b) = padP(a) + padP(b) whenever b (or a) times the element
  // stride is a multiple of 16 -- so a stage's 16 reads / writes are one base
  // plus compile-time offsets.  (Cols: vec < 2^LGNV <= 16 never carries.)
  __device__ __forceinline__ static constexpr int padP(int idx) {
    return VEC_FAST ? ((idx << LGNV) + ((idx << LGNV) >> 4)) : (idx + (idx >> 4));
  }
  __device__ __forceinline__ static constexpr int padV(int vec) {
    return VEC_FAST ? vec : vec * ((1 << LGL) + (1 << (LGL - 4)));
  }
};

// Element hooks: `pre` runs on the values a first stage loads (before its
// DFT), `post` on the values a last stage produces (before they are stored).
// In both cases the element's index within its vector (natural order) is
// j + r * (L / R): butterfly j, slot r.
struct NoHook {
  static constexpr bool kPre = false, kPost = false;
  __device__ __forceinline__ void begin(int, int) {}
  __device__ __forceinline__ float2 pre(int, int, int, int, float2 v) const { return v; }
  __device__ __forceinline__ float2 post(int, int, int, int, float2 v) { return v; }
};

// Where a stage takes its inputs from and puts its outputs.  SmemIO (the
// default) is the padded tile in shared memory.  A pass kernel may give the
// first stage of an FFT a source in global memory (load(vec, idx)) and the
// last stage a sink in global memory (store(vec, idx, v)), so that the tile
// is never staged through shared memory on its way in or out: one shared
// round trip and one barrier less at each end.
struct SmemIO {
  static constexpr bool kGlobal = false;
  __device__ __forceinline__ float2 load(int, int) const { return make_float2(0.f, 0.f); }
  __device__ __forceinline__ void store(int, int, float2) const {}
};

// Stage-major twiddle tables keep, for a stage of span Ls and radix R, the
// rows r of w_{Ls R}^(r k) (k < Ls) that stage_twiddle reads: r = 1, 2, 3, 4,
// 8, 12 for radix 16, r = 1 .. 4 for radix 8, r = 1 .. R-1 for radix 4 and 2.
// Row `row` of a stage holds r = tw_row_r(lgR, row).
__host__ __device__ constexpr int tw_rows(int lgR) { return lgR == 4 ? 6 : lgR == 3 ? 4 : lgR == 2 ? 3 : 1; }
__host__ __device__ constexpr int tw_row_r(int lgR, int row) { return lgR == 4 && row >= 4 ? 4 * (row - 2) : row + 1; }
__host__ __device__ constexpr int tw_row_of(int lgR, int r) { return lgR == 4 && r >= 8 ? r / 4 + 2 : r - 1; }

// Multiply the R inputs of a butterfly by w^(r k), r = 1 .. R-1, from the
// stage's block tw[row(r) Ls + k] = w^(r k) of the table in shared memory.
// Radix 16 reads r = 1, 2, 3, 4, 8, 12 and forms the other nine as
// w^((r1 + 4 r2) k) = w^(r1 k) w^(4 r2 k); radix 8 reads r = 1 .. 4 and forms
// r = 5 .. 7 as w^(4k) w^((r - 4) k).  Every table value is an FP64 result
// rounded once, so each twiddle is at most one product away from it; the
// shared-memory reads drop from 15 to 6 (radix 16) and from 7 to 4 (radix 8).
template <int R, int DIR>
__device__ __forceinline__ void stage_twiddle(float2* v, const float2* __restrict__ tw, int Ls, int k) {
  constexpr int lgR = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4;
  auto get = [&](int r) {
    float2 w = tw[tw_row_of(lgR, r) * Ls + k];
    if (DIR > 0) w.y = -w.y;
    return w;
  };
  if constexpr (R == 16) {
    const float2 w1 = get(1), w2 = get(2), w3 = get(3);
    const float2 w4 = get(4), w8 = get(8), w12 = get(12);
    v[1] = cmul(v[1], w1);
    v[2] = cmul(v[2], w2);
    v[3] = cmul(v[3], w3);
    v[4] = cmul(v[4], w4);
    v[5] = cmul(v[5], cmul(w4, w1));
    v[6] = cmul(v[6], cmul(w4, w2));
    v[7] = cmul(v[7], cmul(w4, w3));
    v[8] = cmul(v[8], w8);
    v[9] = cmul(v[9], cmul(w8, w1));
    v[10] = cmul(v[10], cmul(w8, w2));
    v[11] = cmul(v[11], cmul(w8, w3));
    v[12] = cmul(v[12], w12);
    v[13] = cmul(v[13], cmul(w12, w1));
    v[14] = cmul(v[14], cmul(w12, w2));
    v[15] = cmul(v[15], cmul(w12, w3));
  } else if constexpr (R == 8) {
    const float2 w1 = get(1), w2 = get(2), w3 = get(3), w4 = get(4);
    v[1] = cmul(v[1], w1);
    v[2] = cmul(v[2], w2);
    v[3] = cmul(v[3], w3);
    v[4] = cmul(v[4], w4);
    v[5] = cmul(v[5], cmul(w4, w1));
    v[6] = cmul(v[6], cmul(w4, w2));
    v[7] = cmul(v[7], cmul(w4, w3));
  } else {
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = cmul(v[r], get(r));
  }
}

// One Stockham stage of radix R over all vectors of the tile.
//   Ls   product of the radices of the stages already done
//   tw   without TWS: table tw[q] = exp(-2 pi i q / Lt), Lt = 1 << lgLt >= L,
//        in global memory (read-only path).  With TWS: this stage's block of
//        the stage-major table in shared memory, tw[(r-1) Ls + k] =
//        w_{Ls R}^(r k), so the reads of a butterfly use immediate offsets
//        and neighbouring threads read neighbouring words.
//   in   source of the stage's inputs (first stage only; SmemIO = the tile)
//   out  sink of its outputs (last stage only; SmemIO = the tile)
// A stage whose source is the tile waits at a barrier after reading it (the
// tile is then overwritten); one whose sink is the tile ends with a barrier.
// A stage with a global source must only follow a barrier after any earlier
// use of the tile, and one with a global sink leaves the tile free for reuse
// only after the caller's next barrier.
template <int R, int DIR, int TILE, int NT, bool TWS, class LAY, class H, class IN = SmemIO, class OUT = SmemIO>
__device__ __forceinline__ void stockham_stage(float2* s, const LAY& lay, int lgLs,
                                               const float2* __restrict__ tw, int lgLt, H& hook,
                                               const IN& in = IN{}, const OUT& out = OUT{}) {
  constexpr int BPT = TILE / (R * NT);   // butterflies per thread
  constexpr int lgR = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4;
  const int lgL = lay.LG();
  const int lgnv = lay.NV();
  const int lgLR = lgL - lgR;                    // log2(L/R)
  const int nb = 1 << (lgnv + lgLR);             // butterflies in the tile
  const int Ls = 1 << lgLs;
  const int lgstep = lgLt - lgLs - lgR;          // w_{Ls R}^(r k) = tw[(r k) << lgstep]
  const bool first = lgLs == 0;
  const bool last = lgLs + lgR == lgL;
  float2 v[BPT][R];
  int vecs[BPT], js[BPT];
#pragma unroll
  for (int i = 0; i < BPT; ++i) {
    const int b = threadIdx.x + i * NT;
    if (lay.VF()) { vecs[i] = b & ((1 << lgnv) - 1); js[i] = b >> lgnv; }
    else { vecs[i] = b >> lgLR; js[i] = b & ((1 << lgLR) - 1); }
    if (b < nb) {
      if constexpr (IN::kGlobal) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[i][r] = in.load(vecs[i], js[i] + (r << lgLR));
      } else if constexpr (LAY::kStatic) {
        const float2* lb = s + LAY::padV(vecs[i]) + LAY::padP(js[i]);
#pragma unroll
        for (int r = 0; r < R; ++r) v[i][r] = lb[LAY::padP(r << lgLR)];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[i][r] = s[pad(lay.at(vecs[i], js[i] + (r << lgLR)))];
      }
    }
  }
  if constexpr (!IN::kGlobal) __syncthreads();
#pragma unroll
  for (int i = 0; i < BPT; ++i) {
    const int b = threadIdx.x + i * NT;
    if (b < nb) {
      const int j = js[i];
      const int k = j & (Ls - 1);
      if (H::kPre && first) {
        hook.begin(vecs[i], j);
#pragma unroll
        for (int r = 0; r < R; ++r) v[i][r] = hook.pre(vecs[i], j, r, lgLR, v[i][r]);
      }
      if (!first) {
        if constexpr (TWS) {
          stage_twiddle<R, DIR>(v[i], tw, Ls, k);
        } else {
          const int kk = k << lgstep;   // w_{Ls R}^(r k) = tw[r * kk]
#pragma unroll
          for (int r = 1; r < R; ++r) {
            float2 w = __ldg(tw + r * kk);
            if (DIR > 0) w.y = -w.y;
            v[i][r] = cmul(v[i][r], w);
          }
        }
      }
      dft<R, DIR>(v[i]);
      const int base = ((j - k) << lgR) + k;   // in the last stage base == j, Ls == L/R
      if (H::kPost && last && !(H::kPre && first)) hook.begin(vecs[i], j);
      // static layouts: Ls * stride is a multiple of 16 past the first stage,
      // and in the first stage base = 16 j is (radix 16), so the split holds
      float2* sb = s;
      if constexpr (LAY::kStatic) sb = s + LAY::padV(vecs[i]) + LAY::padP(base);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float2 o = v[i][out_slot<R>(r)];
        if (H::kPost && last) o = hook.post(vecs[i], j, r, lgLR, o);
        if constexpr (OUT::kGlobal) out.store(vecs[i], base + r * Ls, o);
        else if constexpr (LAY::kStatic) sb[LAY::padP(r * Ls)] = o;
        else s[pad(lay.at(vecs[i], base + r * Ls))] = o;
      }
    }
  }
  if constexpr (!OUT::kGlobal) __syncthreads();
}

// Full FFT of every vector in the tile (natural order in and out).  Forward
// (DIR = -1): X_k = sum_j x_j exp(-2 pi i jk/L); inverse (DIR = +1) uses
// exp(+2 pi i jk/L) without the 1/L factor.  The first stage reads from `in`
// and the last writes to `out` (both the tile unless a pass gives global
// ones; only static layouts take global ones).
template <int DIR, int TILE, int NT, bool TWS = false, class LAY, class H, class IN = SmemIO, class OUT = SmemIO>
__device__ __forceinline__ void tile_fft(float2* s, const LAY& lay, const float2* __restrict__ tw, int lgLt,
                                         H& hook, const IN& in = IN{}, const OUT& out = OUT{}) {
  if constexpr (LAY::kStatic) {
    constexpr int LGL = LAY::kLgL;
    constexpr int N16 = LGL / 4;      // radix-16 stages
    constexpr int rem = LGL % 4;      // radix of the closing stage: 2^rem (none when 0)
    constexpr int NST = N16 + (rem ? 1 : 0);
    static_assert(NST >= 2, "a global source and sink need distinct first and last stages");
    // with TWS, stage st (span 16^st) reads block st-1 of the stage-major table
    int off = 0;
#pragma unroll
    for (int st = 0; st < N16; ++st) {
      const float2* tws = TWS ? tw + off : tw;
      if (st == 0)
        stockham_stage<16, DIR, TILE, NT, TWS>(s, lay, 0, tws, lgLt, hook, in, SmemIO{});
      else if (st == NST - 1)
        stockham_stage<16, DIR, TILE, NT, TWS>(s, lay, 4 * st, tws, lgLt, hook, SmemIO{}, out);
      else
        stockham_stage<16, DIR, TILE, NT, TWS>(s, lay, 4 * st, tws, lgLt, hook);
      if (st > 0) off += tw_rows(4) << (4 * st);
    }
    const float2* twr = TWS ? tw + off : tw;
    if constexpr (rem == 3) stockham_stage<8, DIR, TILE, NT, TWS>(s, lay, LGL - 3, twr, lgLt, hook, SmemIO{}, out);
    if constexpr (rem == 2) stockham_stage<4, DIR, TILE, NT, TWS>(s, lay, LGL - 2, twr, lgLt, hook, SmemIO{}, out);
    if constexpr (rem == 1) stockham_stage<2, DIR, TILE, NT, TWS>(s, lay, LGL - 1, twr, lgLt, hook, SmemIO{}, out);
  } else {
    static_assert(!IN::kGlobal && !OUT::kGlobal, "run-time layouts use the shared tile only");
    int lgLs = 0;
    const int lgL = lay.LG();
    while (lgL - lgLs >= 4) { stockham_stage<16, DIR, TILE, NT, TWS>(s, lay, lgLs, tw, lgLt, hook); lgLs += 4; }
    const int rem = lgL - lgLs;
    if (rem == 3) stockham_stage<8, DIR, TILE, NT, TWS>(s, lay, lgLs, tw, lgLt, hook);
    else if (rem == 2) stockham_stage<4, DIR, TILE, NT, TWS>(s, lay, lgLs, tw, lgLt, hook);
    else if (rem == 1) stockham_stage<2, DIR, TILE, NT, TWS>(s, lay, lgLs, tw, lgLt, hook);
  }
}

// Without element hooks (a pass that gives global ends passes a NoHook).
template <int DIR, int TILE, int NT, bool TWS = false, class LAY>
__device__ __forceinline__ void tile_fft(float2* s, const LAY& lay, const float2* __restrict__ tw, int lgLt) {
  NoHook h;
  tile_fft<DIR, TILE, NT, TWS>(s, lay, tw, lgLt, h);
}

// Entries of the stage-major twiddle table of a length-L FFT: stage s >= 1
// (span Ls, radix R) contributes tw_rows(log2 R) * Ls entries.
__host__ __device__ constexpr int stage_tw_count(int lgL) {
  int n = 0, lgLs = 0;
  while (lgLs < lgL) {
    const int lgR = (lgL - lgLs) >= 4 ? 4 : (lgL - lgLs);
    if (lgLs > 0) n += tw_rows(lgR) << lgLs;
    lgLs += lgR;
  }
  return n;
}

// Copy `count` (a multiple of 2) table entries from global to shared memory.
template <int NT>
__device__ __forceinline__ void copy_table(float2* dst, const float2* __restrict__ src, int count) {
  for (int i = 2 * threadIdx.x; i < count; i += 2 * NT) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(src + i));
    dst[i] = make_float2(v.x, v.y);
    dst[i + 1] = make_float2(v.z, v.w);
  }
}

}  // namespace csk
