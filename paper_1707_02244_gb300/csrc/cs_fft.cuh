// Shared-memory Stockham FFT building blocks (fp32, sm_103a).
//
// A CTA holds up to TILE complex values in shared memory, arranged as `nvec`
// vectors of length L (a power of two).  One Stockham stage of radix R reads
// R values per butterfly at stride L/R, twiddles them, applies an in-register
// DFT_R and writes them back in auto-sorted order, so no bit reversal is ever
// needed.  Stages use radix 16 while log2(L) allows it and one radix-2/4/8
// stage for the remainder.
//
// Shared-memory index of linear element e is e + (e >> 4): one pad slot per
// 16 complex values keeps the stride-16 writes of the first stage free of
// bank conflicts.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace csk {

constexpr int NT = 256;          // threads per CTA of the FFT passes
constexpr int TILE = 8192;       // complex values per CTA
constexpr int EPT = TILE / NT;   // complex values per thread

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

// exp(DIR * 2 pi i j / 16), folded to constants when j is known at compile time
template <int DIR>
__device__ __forceinline__ float2 w16(int j) { return make_float2(cos16(j), DIR * sin16(j)); }

// In-register DFT of length R (R in {2,4,8,16}), natural order in and out:
// X_k = sum_r a_r exp(DIR 2 pi i r k / R).
template <int R, int DIR> struct Dft;

template <int DIR> struct Dft<2, DIR> {
  __device__ __forceinline__ static void run(float2* a) {
    float2 t = a[1];
    a[1] = csub(a[0], t);
    a[0] = cadd(a[0], t);
  }
};

template <int DIR> struct Dft<4, DIR> {
  __device__ __forceinline__ static void run(float2* a) {
    float2 s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
    float2 s13 = cadd(a[1], a[3]), d13 = mul_diri<DIR>(csub(a[1], a[3]));
    a[0] = cadd(s02, s13);
    a[2] = csub(s02, s13);
    a[1] = cadd(d02, d13);
    a[3] = csub(d02, d13);
  }
};

// R = P*Q: n = Q*n1 + n2, k = k1 + P*k2.
//   b[n2][k1] = DFT_P over n1 of a[Q n1 + n2], times w_R^(n2 k1)
//   X[k1 + P k2] = DFT_Q over n2 of b[n2][k1]
template <int P, int Q, int DIR>
__device__ __forceinline__ void dft_split(float2* a) {
  constexpr int R = P * Q;
  float2 b[Q][P];
#pragma unroll
  for (int n2 = 0; n2 < Q; ++n2) {
    float2 t[P];
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) t[n1] = a[Q * n1 + n2];
    Dft<P, DIR>::run(t);
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
      const int j = (n2 * k1 * (16 / R)) & 15;
      b[n2][k1] = (j == 0) ? t[k1] : cmul(t[k1], w16<DIR>(j));
    }
  }
#pragma unroll
  for (int k1 = 0; k1 < P; ++k1) {
    float2 t[Q];
#pragma unroll
    for (int n2 = 0; n2 < Q; ++n2) t[n2] = b[n2][k1];
    Dft<Q, DIR>::run(t);
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) a[k1 + P * k2] = t[k2];
  }
}

template <int DIR> struct Dft<8, DIR> {
  __device__ __forceinline__ static void run(float2* a) { dft_split<4, 2, DIR>(a); }
};
template <int DIR> struct Dft<16, DIR> {
  __device__ __forceinline__ static void run(float2* a) { dft_split<4, 4, DIR>(a); }
};

// Geometry of the vectors held in shared memory.
//   rows layout (vec_fast = false): element (vec, idx) at vec*L + idx
//   cols layout (vec_fast = true):  element (vec, idx) at idx*nvec + vec
struct VecLayout {
  int lgL;      // log2 vector length
  int lgnv;     // log2 number of vectors
  bool vec_fast;
  __device__ __forceinline__ int at(int vec, int idx) const {
    return vec_fast ? ((idx << lgnv) + vec) : ((vec << lgL) + idx);
  }
};

// One Stockham stage of radix R over all vectors of the tile.
//   Ls   product of the radices of the stages already done
//   tw   twiddle table tw[q] = exp(-2 pi i q / Lt), Lt = 1 << lgLt >= L
template <int R, int DIR>
__device__ __forceinline__ void stockham_stage(float2* s, const VecLayout& lay, int lgLs,
                                               const float2* __restrict__ tw, int lgLt) {
  constexpr int BPT = TILE / (R * NT);   // butterflies per thread
  const int lgL = lay.lgL;
  const int lgLR = lgL - (R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4);  // log2(L/R)
  const int nb = 1 << (lay.lgnv + lgLR);                                // butterflies in the tile
  const int Ls = 1 << lgLs;
  // twiddle index step for w_{Ls R}^(r k): (Lt / (Ls R)) * r * k
  const int lgstep = lgLt - lgLs - (lgL - lgLR);
  float2 v[BPT][R];
#pragma unroll
  for (int i = 0; i < BPT; ++i) {
    const int b = threadIdx.x + i * NT;
    if (b < nb) {
      int vec, j;
      if (lay.vec_fast) { vec = b & ((1 << lay.lgnv) - 1); j = b >> lay.lgnv; }
      else { vec = b >> lgLR; j = b & ((1 << lgLR) - 1); }
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = s[pad(lay.at(vec, j + (r << lgLR)))];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < BPT; ++i) {
    const int b = threadIdx.x + i * NT;
    if (b < nb) {
      int vec, j;
      if (lay.vec_fast) { vec = b & ((1 << lay.lgnv) - 1); j = b >> lay.lgnv; }
      else { vec = b >> lgLR; j = b & ((1 << lgLR) - 1); }
      const int k = j & (Ls - 1);
      if (lgLs > 0) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = __ldg(tw + ((r * k) << lgstep));
          if (DIR > 0) w.y = -w.y;
          v[i][r] = cmul(v[i][r], w);
        }
      }
      Dft<R, DIR>::run(v[i]);
      const int base = ((j - k) * R) + k;
#pragma unroll
      for (int r = 0; r < R; ++r) s[pad(lay.at(vec, base + r * Ls))] = v[i][r];
    }
  }
  __syncthreads();
}

// Full FFT of every vector in the tile (in place, natural order in and out).
// Forward (DIR = -1): X_k = sum_j x_j exp(-2 pi i jk/L); inverse (DIR = +1)
// uses exp(+2 pi i jk/L) without the 1/L factor.
template <int DIR>
__device__ __forceinline__ void tile_fft(float2* s, const VecLayout& lay, const float2* __restrict__ tw,
                                         int lgLt) {
  int lgLs = 0;
  const int lgL = lay.lgL;
  while (lgL - lgLs >= 4) { stockham_stage<16, DIR>(s, lay, lgLs, tw, lgLt); lgLs += 4; }
  const int rem = lgL - lgLs;
  if (rem == 3) stockham_stage<8, DIR>(s, lay, lgLs, tw, lgLt);
  else if (rem == 2) stockham_stage<4, DIR>(s, lay, lgLs, tw, lgLt);
  else if (rem == 1) stockham_stage<2, DIR>(s, lay, lgLs, tw, lgLt);
}

}  // namespace csk
