// Column pass of the fused FFT iteration: inverse length-N2 FFTs down G
// columns of the N2 x N1 exchange array, the method's elementwise step
// (residual on the kept rows, soft threshold, ADMM updates) as the hook of
// the last inverse stage, then the forward FFTs of the next product.
#include "cs_passes.cuh"

namespace csk {

namespace {

// ---------------------------------------------------------------- column pass

// The column pass uses 4096-value tiles (4 CTAs per SM; 1D: N2 <= 1024
// gives G >= 4 columns), and 16384-value tiles of four 4096-long columns for
// 2D arrays of 4096 rows (1 CTA per SM): four columns make each row of the
// exchange buffer a full 32-byte sector (two would use half of it).
constexpr int COL_TILE = 4096;
constexpr int COL_MINB = 4;
constexpr int COL_TILE4 = 16384;
constexpr int COL_MINB4 = 1;

// Epilogue as the post hook of the inverse column FFT: runs on each value as
// the last stage produces it, so the elementwise step costs no extra pass
// over shared memory.
template <int KIND>
struct EpiHook {
  static constexpr bool kPre = false, kPost = true;
  const KParams& kp;
  const CallArgs& a;
  int col0, lgN1;
  Acc& acc;
  __device__ __forceinline__ void begin(int, int) {}
  __device__ __forceinline__ float2 pre(int, int, int, int, float2 v) const { return v; }
  int tbase;   // tile-order index of this CTA's first element: col0 * N2
  int lgG;
  __device__ __forceinline__ float2 post(int vec, int j, int r, int lgLR, float2 v) {
    const int idx = j + (r << lgLR);
    return Epi<KIND>::apply(kp, a, v, col0 + vec + (idx << lgN1), tbase + (idx << lgG) + vec, acc);
  }
};

// SHAPE 0: any geometry (shape read at run time); SHAPE 1: N2 = 1024 and
// G = 4 columns, the geometry of every N >= 2^20, fixed at compile time.
template <int SHAPE> struct ColShape;
template <> struct ColShape<0> {
  using Lay = DynLayout;
  __device__ static Lay lay(const Geo& g) { return Lay{g.lgN2, g.lgG, true}; }
  __device__ static int lgG(const Geo& g) { return g.lgG; }
  __device__ static int lgN2(const Geo& g) { return g.lgN2; }
};
template <> struct ColShape<1> {
  using Lay = StaticLayout<10, 2, true>;
  __device__ static Lay lay(const Geo&) { return Lay{}; }
  __device__ static constexpr int lgG(const Geo&) { return 2; }
  __device__ static constexpr int lgN2(const Geo&) { return 10; }
};

// SHAPE 3: N2 = 4096 and G = 4, 16384-value tiles (1024 threads).
template <> struct ColShape<3> {
  using Lay = StaticLayout<12, 2, true>;
  __device__ static Lay lay(const Geo&) { return Lay{}; }
  __device__ static constexpr int lgG(const Geo&) { return 2; }
  __device__ static constexpr int lgN2(const Geo&) { return 12; }
};

// Global source / sink of the tile's first and last FFT stages (static
// shapes): element (column c, row j2) of the tile is W[col0 + c + j2 N1].
struct ColIO {
  static constexpr bool kGlobal = true;
  float2* W;
  int col0, lgN1;
  __device__ __forceinline__ float2 load(int c, int j2) const {
    return __ldcg(W + col0 + c + ((size_t)j2 << lgN1));
  }
  __device__ __forceinline__ void store(int c, int j2, float2 v) const {
    __stcg(W + col0 + c + ((size_t)j2 << lgN1), v);
  }
};

template <int SHAPE> struct ColTile {
  static constexpr int kTile = SHAPE == 3 ? COL_TILE4 : COL_TILE;
  static constexpr int kMinB = SHAPE == 3 ? COL_MINB4 : COL_MINB;
  static constexpr int kLgN2 = SHAPE == 3 ? 12 : 10;   // static shapes
};

// The column pass of tile `blk` (columns blk G .. blk G + G - 1).
template <int KIND, int SHAPE>
__device__ __forceinline__ void col_body(const KParams& kp, const int blk) {
  constexpr int TILE = ColTile<SHAPE>::kTile;
  constexpr int NT = Cfg<TILE>::NT;
  constexpr int NLD = Cfg<TILE>::NLD;
  using E = Epi<KIND>;
  using S = ColShape<SHAPE>;
  extern __shared__ float2 sm[];
  pdl_trigger();
  const Geo& g = kp.geo;
  const int lgG = S::lgG(g), lgN2 = S::lgN2(g);
  const int G = 1 << lgG;
  const int col0 = blk << lgG;
  const int tot = G << lgN2;
  const auto lay = S::lay(g);
  constexpr bool TWS = SHAPE != 0;   // static shape: stage-major twiddles in shared memory
  constexpr int TW_N = TWS ? stage_tw_count(ColTile<SHAPE>::kLgN2) : 2;
  __shared__ __align__(16) float2 tws[TW_N];
  const float2* tw = TWS ? tws : g.tw2;
  if (TWS) copy_table<NT>(tws, g.tws2, TW_N);   // plan constant
  // the tile's row-mask and prefix words (plan constants): 2 bits per element
  // in the packed geometry, 1 in complex-n
  constexpr int MB = UsesMask<KIND>::kBits;
  constexpr int MW = MB ? TILE * MB / 32 : 1;
  __shared__ uint32_t smask[MW], spref[MW];
  const int wbase = MB ? (((col0 << lgN2) * MB) >> 5) : 0;
  if (MB) {
    const int words = (tot * MB) >> 5;
    for (int w = threadIdx.x; w < words; w += NT) {
      smask[w] = __ldg(kp.pp.mask + wbase + w);
      spref[w] = __ldg(kp.pp.prefix + wbase + w);
    }
  }
  pdl_wait();                                   // everything below may depend on earlier kernels
  const CallArgs a = *kp.ca;
  float2* __restrict__ W = kp.pp.W;
  Acc acc;
  acc.zero();
  acc.smask = smask;
  acc.spref = spref;
  acc.wbase = wbase;

  if constexpr (E::kRead && SHAPE != 0) {
    // static shapes: the first inverse stage reads the exchange buffer itself
    EpiHook<KIND> hook{kp, a, col0, g.lgN1, acc, col0 << lgN2, lgG};
    tile_fft<+1, TILE, NT, TWS>(sm, lay, tw, lgN2, hook, ColIO{W, col0, g.lgN1}, SmemIO{});
  } else if constexpr (E::kRead) {
    float4 buf[NLD];
#pragma unroll
    for (int i = 0; i < NLD; ++i) {
      const int e = 2 * (threadIdx.x + i * NT);
      if (e < tot) {
        const int j2 = e >> lgG, c = e & (G - 1);
        buf[i] = __ldcg(reinterpret_cast<const float4*>(W + col0 + c + ((size_t)j2 << g.lgN1)));
      }
    }
#pragma unroll
    for (int i = 0; i < NLD; ++i) {
      const int e = 2 * (threadIdx.x + i * NT);
      if (e < tot) {
        sm[pad(e)] = make_float2(buf[i].x, buf[i].y);
        sm[pad(e + 1)] = make_float2(buf[i].z, buf[i].w);
      }
    }
    __syncthreads();
    EpiHook<KIND> hook{kp, a, col0, g.lgN1, acc, col0 << lgN2, lgG};
    tile_fft<+1, TILE, NT, TWS>(sm, lay, tw, lgN2, hook);
  } else {
    for (int e = threadIdx.x; e < tot; e += NT) {
      const int j2 = e >> lgG, c = e & (G - 1);
      sm[pad(e)] = E::apply(kp, a, make_float2(0.f, 0.f), col0 + c + (j2 << g.lgN1), (col0 << lgN2) + e, acc);
    }
    __syncthreads();
  }
  if constexpr (KIND == COL_GRAD_W || KIND == COL_ADMM_REV) block_accum<NT>(acc.v[0], kp.pp.gpart, blk);
  if (kp.flags & FL_STATS) {
    constexpr int kSlots =
        KIND == COL_RESIDUAL ? (1 << ST_R2)
        : KIND == COL_POWER_OUT ? ((1 << ST_DX2) | (1 << ST_X2))
        : (KIND == COL_ISTA || KIND == COL_ISTA_LAST)
            ? ((1 << ST_ERR2) | (1 << ST_DX2) | (1 << ST_X2) | (1 << ST_L1) | (1 << ST_NONFIN))
        : (KIND == COL_ADMM || KIND == COL_ADMM_LAST) ? ((1 << ST_ERR2) | (1 << ST_DX2) | (1 << ST_X2) |
                                                         (1 << ST_L1) | (1 << ST_R2) | (1 << ST_NONFIN))
        : 0;
    if (kSlots) block_stats<kSlots, NT>(acc, kp.pp.partials, blk);
  }
  if constexpr (E::kFwd && SHAPE != 0) {
    // static shapes: the last forward stage writes the exchange buffer itself
    NoHook nh;
    tile_fft<-1, TILE, NT, TWS>(sm, lay, tw, lgN2, nh, SmemIO{}, ColIO{W, col0, g.lgN1});
  } else if constexpr (E::kFwd) {
    tile_fft<-1, TILE, NT, TWS>(sm, lay, tw, lgN2);
#pragma unroll
    for (int i = 0; i < NLD; ++i) {
      const int e = 2 * (threadIdx.x + i * NT);
      if (e < tot) {
        const int j2 = e >> lgG, c = e & (G - 1);
        const float2 lo = sm[pad(e)], hi = sm[pad(e + 1)];
        __stcg(reinterpret_cast<float4*>(W + col0 + c + ((size_t)j2 << g.lgN1)),
               make_float4(lo.x, lo.y, hi.x, hi.y));
      }
    }
  }
  if constexpr (KIND == COL_LOAD2) {
    // the second vector of the pair, to the second exchange buffer
    __syncthreads();
    for (int e = threadIdx.x; e < tot; e += NT) sm[pad(e)] = Epi<COL_LOAD2>::apply2(kp, a, (col0 << lgN2) + e);
    __syncthreads();
    tile_fft<-1, TILE, NT, TWS>(sm, lay, tw, lgN2);
    float2* __restrict__ W2 = kp.pp.W2;
#pragma unroll
    for (int i = 0; i < NLD; ++i) {
      const int e = 2 * (threadIdx.x + i * NT);
      if (e < tot) {
        const int j2 = e >> lgG, c = e & (G - 1);
        const float2 lo = sm[pad(e)], hi = sm[pad(e + 1)];
        __stcg(reinterpret_cast<float4*>(W2 + col0 + c + ((size_t)j2 << g.lgN1)),
               make_float4(lo.x, lo.y, hi.x, hi.y));
      }
    }
  }
}

template <int KIND, int SHAPE>
__global__ void __launch_bounds__(ColTile<SHAPE>::kTile / EPT, ColTile<SHAPE>::kMinB) col_kernel(const KParams kp) {
  col_body<KIND, SHAPE>(kp, blockIdx.x);
}

// Grouped launch over many plans (batched solves): CTA b runs tile
// map[b].y of plan map[b].x, whose parameters kps[map[b].x] are copied to
// shared memory first.  Run-time shapes only.
template <int KIND>
__global__ void __launch_bounds__(COL_TILE / EPT, COL_MINB)
    col_kernel_multi(const KParams* __restrict__ kps, const int2* __restrict__ map) {
  static_assert(sizeof(KParams) % 4 == 0 && sizeof(KParams) / 4 <= COL_TILE / EPT, "KParams copy");
  __shared__ KParams skp;
  const int2 it = map[blockIdx.x];
  if (threadIdx.x < sizeof(KParams) / 4)
    reinterpret_cast<int*>(&skp)[threadIdx.x] = reinterpret_cast<const int*>(kps + it.x)[threadIdx.x];
  __syncthreads();
  col_body<KIND, 0>(skp, it.y);
}

}  // namespace

// kinds of the 2D solves (no gradient)
#define CS_COL_KINDS_2D(X, S)                                                                  \
  X(COL_LOAD, S) X(COL_LOAD_SCALED, S) X(COL_STORE, S) X(COL_MASK, S) X(COL_RESIDUAL, S)         \
  X(COL_ISTA, S) X(COL_ISTA_LAST, S) X(COL_POWER_OUT, S) X(COL_ADMM_INIT, S) X(COL_ADMM, S)       \
  X(COL_ADMM_LAST, S)

#define CS_COL_KINDS(X, S)                                                                     \
  X(COL_LOAD, S) X(COL_LOAD_SCALED, S) X(COL_STORE, S) X(COL_MASK, S) X(COL_RESIDUAL, S)         \
  X(COL_ISTA, S) X(COL_ISTA_LAST, S) X(COL_POWER_OUT, S) X(COL_ADMM_INIT, S) X(COL_ADMM, S)       \
  X(COL_ADMM_LAST, S) X(COL_LOADT, S) X(COL_RES_SAVE, S) X(COL_ISTA_SEG, S) X(COL_GRAD_W, S)           \
  X(COL_GRAD_MASK, S) X(COL_GRAD_G, S) X(COL_LOAD2, S) X(COL_ADMM_SEG, S) X(COL_ADMM_REV, S) X(COL_STORE_RE, S)

cudaError_t init_col_kernels() {
  cudaError_t e = cudaSuccess;
#define CS_SET_COL(k, S) \
  if (e == cudaSuccess) e = set_smem(col_kernel<k, S>, ColTile<S>::kTile, ColTile<S>::kMinB);
  CS_COL_KINDS(CS_SET_COL, 0)
  CS_COL_KINDS(CS_SET_COL, 1)
  CS_COL_KINDS_2D(CS_SET_COL, 3)
#undef CS_SET_COL
  return e;
}

#define CS_COL_KINDS_MULTI(X) \
  X(COL_LOAD) X(COL_RESIDUAL) X(COL_ISTA) X(COL_ISTA_LAST) X(COL_ADMM_INIT) X(COL_ADMM) X(COL_ADMM_LAST)

cudaError_t init_col_multi_kernels() {
  cudaError_t e = cudaSuccess;
#define CS_SET_COLM(k) \
  if (e == cudaSuccess) e = set_smem(col_kernel_multi<k>, COL_TILE, COL_MINB);
  CS_COL_KINDS_MULTI(CS_SET_COLM)
#undef CS_SET_COLM
  return e;
}

template <typename K>
cudaError_t launch_multi(K kern, int grid, int tile, const KParams* kps, const int2* map, cudaStream_t s,
                         int smem_mult = 1) {
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
  return cudaLaunchKernelEx(&cfg, kern, kps, map);
}

cudaError_t launch_col_multi(ColKind kind, const KParams* kps, const int2* map, int nctas, cudaStream_t s) {
  if (nctas < 1) return cudaSuccess;
#define CS_L_COLM(k) case k: return launch_multi(col_kernel_multi<k>, nctas, COL_TILE, kps, map, s);
  switch (kind) {
    CS_COL_KINDS_MULTI(CS_L_COLM)
    default: break;
  }
#undef CS_L_COLM
  return cudaErrorInvalidValue;
}

cudaError_t launch_col(ColKind kind, const KParams& kp, cudaStream_t s) {
  const Geo& g = kp.geo;
  const int grid = g.col_ctas;
  const bool hot = g.lgN2 == 10 && g.lgG == 2;
#define CS_L_COL(k, S) case k: return launch_k(col_kernel<k, S>, grid, ColTile<S>::kTile, kp, s);
  if (g.col_tile == COL_TILE4) {
    if (g.lgN2 == 12 && g.lgG == 2) {
      switch (kind) { CS_COL_KINDS_2D(CS_L_COL, 3) default: break; }
    }
  } else if (hot) {
    switch (kind) { CS_COL_KINDS(CS_L_COL, 1) }
  } else {
    switch (kind) { CS_COL_KINDS(CS_L_COL, 0) }
  }
#undef CS_L_COL
  return cudaErrorInvalidValue;
}

}  // namespace csk
