// Host runtime of the C ABI declared in include/cs.h: plan construction,
// argument checks, CUDA-graph capture of the iteration loop, monitoring.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>

#include "../../include/cs.h"
#include "cs_fft.cuh"
#include "cs_internal.h"

using namespace csk;

struct cs_plan_s {
  int64_t n = 0, m = 0;
  cudaStream_t stream = nullptr;   // caller's stream
  cudaStream_t cap = nullptr;      // private stream used only for graph capture
  Geo gi{}, ga{};                  // real-FFT (N = n/2) and complex-n (N = n) geometry
  float2* W = nullptr;
  // Rows of Omega per geometry, in the tile order of its column pass.
  struct Sel {
    uint32_t* mask = nullptr;
    uint32_t* prefix = nullptr;
    int32_t* pos = nullptr;     // compact position of y[i]
    float* ys = nullptr;        // compact y in tile order
  } si, sa;                     // si: real-FFT geometry gi, sa: complex-n geometry ga
  int32_t* rows32 = nullptr;
  // Solver state in tile order (natural order only at the API boundary).
  float* xi_t = nullptr;        // ISTA iterate (float2[n/2])
  float* xt_i = nullptr;        // monitor ground truth, gi tile order (float2[n/2])
  float* xt_a = nullptr;        // monitor ground truth, ga tile order
  float *av = nullptr, *az = nullptr, *amu = nullptr, *anu = nullptr, *ax = nullptr;   // ADMM state
  double* partials = nullptr;
  double* stats = nullptr;
  int* status = nullptr;
  CallArgs* ca = nullptr;
  float4* tab_ista = nullptr;
  float2* tab_admm_c = nullptr;
  float* tab_admm_b = nullptr;
  double* abs2 = nullptr;
  float2* twi = nullptr;
  float2* twa = nullptr;
  float* dense = nullptr;
  float* dense2 = nullptr;
  float* dense3 = nullptr;
  double* host_stats = nullptr;    // pinned [NSTAT]
  int* host_status = nullptr;      // pinned
  double b_rho = -1.0, b_sigma = -1.0;
  const float* xtrue = nullptr;
  double xtrue2 = 0.0;
  double tol = 0.0;
  int check_every = 10;
  bool use_graphs = true;
  int latched = 0;                 // device status bits read back but not yet reported
  int launches = 0;                // kernels enqueued by the current call
  int graph_nodes_last = 0;
  bool ista_args = false, admm_args = false;   // last solve of each kind left valid arguments
  std::map<uint64_t, int> graph_nodes;
  std::map<uint64_t, cudaGraphExec_t> graphs;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // unrolled-ISTA gradient (cs_grad): allocated at the first call, grown on demand
  struct Grad {
    int ck_cap = 0, seg_cap = 0;
    float* ckpt = nullptr;   // [ck_cap][n]  x(sK), tile order
    float* seg = nullptr;    // [seg_cap + 1][n]  x(t) of the segment being replayed
    float* rseg = nullptr;   // [seg_cap][n]  r(t) of the segment
    float *g = nullptr, *w = nullptr, *q = nullptr;
    float* dy = nullptr;     // [m] dL/dy, compact in the tile order of the rows
    float2* W2 = nullptr;
    float4* gacc = nullptr;  // spectrum of dL/dc (before tau), per pair slot
    double* gpart = nullptr; // per column CTA: dL/dtheta
    CallArgs* ca = nullptr;  // [seg_cap + 1]: step j of a segment, and the output pass
  } gr;
  // unrolled-ADMM gradient (cs_grad_admm): allocated at the first call, grown on demand
  struct GradA {
    int ck_cap = 0, seg_cap = 0;
    float* ckpt = nullptr;   // [ck_cap][4][n]  state (v, z, mu, nu) entering iteration sK, tile order
    float2* wseg = nullptr;  // [seg_cap][n]  column transform of iteration j's forward pair v + i (z - nu)
    float* sseg = nullptr;   // [seg_cap][n]  iteration j's soft-threshold input x + nu
    float *mub = nullptr, *nub = nullptr;   // adjoint state (mu', nu' without -sigma b')
    float *gz = nullptr, *gx = nullptr;     // dL/dz(T), dL/dx(T) in tile order
    float* dy = nullptr;     // [m] dL/dy, compact in the tile order of the rows
    float2* Wr = nullptr;    // exchange buffer of the reverse pass
    float2* gacc = nullptr;  // per pair slot: spectrum of dL/dc (over N)
    double* gpart = nullptr; // per column CTA: sum of -sign(s) s'
    CallArgs* ca = nullptr;  // [2 seg_cap + 2]: replay steps, reverse steps, first reverse step, output
  } ga_;
};

namespace {

int ilog2(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l;
}

void make_geo(Geo& g, int lgN) {
  g.lgN = lgN;
  g.N = 1 << lgN;
  g.lgN2 = lgN / 2 < 10 ? lgN / 2 : 10;
  g.N2 = 1 << g.lgN2;
  g.lgN1 = lgN - g.lgN2;
  g.N1 = 1 << g.lgN1;
  // column pass: 4096-value tiles (256 threads), G = 4096 / N2 >= 4 columns
  const int lgCol = 12;
  g.lgG = (lgCol - g.lgN2) < g.lgN1 ? (lgCol - g.lgN2) : g.lgN1;
  g.G = 1 << g.lgG;
  g.col_ctas = g.N1 >> g.lgG;
  // mid pass: 4096-value tiles when a row pair fits, else 8192 (512 threads)
  const int lgMid = g.lgN1 <= 11 ? 12 : 13;
  g.tile = 1 << lgMid;
  const int lgUmax = lgMid - 1 - g.lgN1;
  const int lgUnits = g.lgN2 - 1;
  g.lgU = lgUmax < lgUnits ? lgUmax : lgUnits;
  g.U = 1 << g.lgU;
  g.mid_ctas = (g.N2 >> 1) >> g.lgU;
  g.col_tile = 4096;
  g.twod = 0;
}

// 2D DFT of an N2 x N1 array (2^lgN2 rows of 2^lgN1): the same two passes
// without the four-step twiddle.  Column pass: 4096-value tiles while
// N2 <= 2048, 8192-value tiles of two columns for N2 = 4096.
void make_geo2d(Geo& g, int lgN2, int lgN1) {
  g.lgN = lgN2 + lgN1;
  g.N = 1 << g.lgN;
  g.lgN2 = lgN2;
  g.N2 = 1 << lgN2;
  g.lgN1 = lgN1;
  g.N1 = 1 << lgN1;
  const int lgCol = lgN2 <= 11 ? 12 : 14;
  g.col_tile = 1 << lgCol;
  g.lgG = (lgCol - lgN2) < lgN1 ? (lgCol - lgN2) : lgN1;
  g.G = 1 << g.lgG;
  g.col_ctas = g.N1 >> g.lgG;
  const int lgMid = lgN1 <= 11 ? 12 : 13;
  g.tile = 1 << lgMid;
  int lgU = lgMid - 1 - lgN1;
  if (lgU > lgN2 - 1) lgU = lgN2 - 1;
  if (lgU > 5) lgU = 5;   // 2U <= 64 rows
  g.lgU = lgU;
  g.U = 1 << lgU;
  g.mid_ctas = (g.N2 >> 1) >> lgU;
  g.twod = 1;
}

// Geometry invariants the pass kernels rely on (checked for every plan).
bool geo_ok(const Geo& g) {
  if (g.twod)
    return g.N2 >= 2 && g.N1 >= 2 && g.G >= 2 && g.col_ctas >= 1 && g.mid_ctas >= 1 && g.U >= 1 &&
           2 * g.U <= 64 && (2 * g.U) * g.N1 <= g.tile && (g.G << g.lgN2) <= g.col_tile && g.N1 <= 4096 &&
           (g.col_tile == 4096 || (g.lgN2 == 12 && g.lgG == 2 && g.col_tile == 16384));
  return g.N1 >= g.N2 && g.N2 >= 2 && g.G >= 2 && g.col_ctas >= 1 && g.mid_ctas >= 1 &&
         2 * g.U <= 64 && (2 * g.U) * g.N1 <= g.tile && (g.G << g.lgN2) <= 4096;
}

cs_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return CS_OK;
  if (e == cudaErrorMemoryAllocation) return CS_ERR_NOMEM;
  return CS_ERR_CUDA;
}

#define CS_TRY(expr)                                   \
  do {                                                 \
    cudaError_t e_ = (expr);                           \
    if (e_ != cudaSuccess) return cuda_status(e_);     \
  } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T) + 256);
}

void free_plan(cs_plan_s* p) {
  if (!p) return;
  for (auto& kv : p->graphs) cudaGraphExecDestroy(kv.second);
  void* bufs[] = {p->W, p->si.mask, p->si.prefix, p->si.pos, p->si.ys, p->sa.mask, p->sa.prefix, p->sa.pos,
                  p->sa.ys, p->rows32, p->xi_t, p->xt_i, p->xt_a, p->av, p->az, p->amu, p->anu, p->ax,
                  p->partials, p->stats, p->status,
                  p->ca, p->tab_ista, p->tab_admm_c, p->tab_admm_b, p->abs2, p->twi, p->twa,
                  p->dense, p->dense2, p->dense3};
  for (void* b : bufs)
    if (b) cudaFree(b);
  void* gbufs[] = {p->gr.ckpt, p->gr.seg, p->gr.rseg, p->gr.g, p->gr.w, p->gr.q, p->gr.dy, p->gr.W2, p->gr.gacc,
                   p->gr.gpart, p->gr.ca};
  for (void* b : gbufs)
    if (b) cudaFree(b);
  void* abufs[] = {p->ga_.ckpt, p->ga_.wseg, p->ga_.sseg, p->ga_.mub, p->ga_.nub, p->ga_.gz, p->ga_.gx,
                   p->ga_.dy, p->ga_.Wr, p->ga_.gacc, p->ga_.gpart, p->ga_.ca};
  for (void* b : abufs)
    if (b) cudaFree(b);
  if (p->host_stats) cudaFreeHost(p->host_stats);
  if (p->host_status) cudaFreeHost(p->host_status);
  if (p->cap) cudaStreamDestroy(p->cap);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  delete p;
}

KParams kparams(const cs_plan_s* p, const Geo& g, int flags) {
  KParams k;
  k.geo = g;
  k.pp.W = p->W;
  const cs_plan_s::Sel& sel = (&g == &p->gi) ? p->si : p->sa;
  k.pp.mask = sel.mask;
  k.pp.prefix = sel.prefix;
  k.pp.ys = sel.ys;
  k.pp.partials = p->partials;
  k.pp.stats = p->stats;
  k.pp.tab_ista = p->tab_ista;
  k.pp.tab_admm_c = p->tab_admm_c;
  k.pp.tab_admm_b = p->tab_admm_b;
  k.pp.status = p->status;
  k.pp.W2 = p->gr.W2;
  k.pp.gacc = p->gr.gacc;
  k.pp.gpart = p->gr.gpart;
  k.ca = p->ca;
  k.flags = flags;
  return k;
}

cudaError_t make_tables(Geo& g, float2* base, cudaStream_t s) {
  // tw1 [2 N1] | tw2 [N2] | twl [N1] | twr [N2] | tw1h [N1] | tws1 [N1] | tws2 [N2]
  // (every block starts at an even index: 16-byte aligned)
  float2* tw1 = base;
  float2* tw2 = tw1 + 2 * g.N1;
  float2* twl = tw2 + g.N2;
  float2* twr = twl + g.N1;
  float2* tw1h = twr + g.N2;
  float2* tws1 = tw1h + g.N1;
  float2* tws2 = tws1 + g.N1;
  cudaError_t e = launch_twiddle(tw1, 2 * g.N1, 2 * (int64_t)g.N1, s);
  if (e == cudaSuccess) e = launch_twiddle(tw2, g.N2, g.N2, s);
  if (e == cudaSuccess) e = launch_twiddle(twl, g.N1, g.N, s);
  if (e == cudaSuccess) e = launch_twiddle(twr, g.N2, 2 * (int64_t)g.N, s);
  if (e == cudaSuccess) e = launch_twiddle(tw1h, g.N1, g.N1, s);
  if (e == cudaSuccess) e = launch_stage_tw(tws1, g.lgN1, stage_tw_count(g.lgN1), s);
  if (e == cudaSuccess) e = launch_stage_tw(tws2, g.lgN2, stage_tw_count(g.lgN2), s);
  g.tw1 = tw1;
  g.tw2 = tw2;
  g.twl = twl;
  g.twr = twr;
  g.tw1h = tw1h;
  g.tws1 = tws1;
  g.tws2 = tws2;
  return e;
}

size_t twiddle_count(const Geo& g) { return 5 * (size_t)g.N1 + 3 * (size_t)g.N2; }

// Read the device status word and the finalised stats into pinned memory.
cudaError_t read_back(cs_plan_s* p) {
  cudaError_t e = cudaMemcpyAsync(p->host_stats, p->stats, NSTAT * sizeof(double), cudaMemcpyDeviceToHost,
                                  p->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->host_status, p->status, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e == cudaSuccess) p->latched |= *p->host_status;
  return e;
}

cs_status latched_status(cs_plan_s* p) {
  if (p->latched & STS_TIMEOUT) return CS_ERR_TIMEOUT;
  if (p->latched & STS_NONFINITE) return CS_ERR_NONFINITE;
  return CS_OK;
}

// One solve chunk: `len` iterations, the last of which computes the check
// statistics; `final_chunk` drops the forward FFT after the last update.
enum SolveKind { K_ISTA = 1, K_ADMM = 2 };

cudaError_t enqueue_chunk(cs_plan_s* p, SolveKind kind, int len, bool final_chunk, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (int it = 0; it < len && e == cudaSuccess; ++it) {
    const bool last = it == len - 1;
    const int flags = last ? (FL_STATS | FL_WRITE_STATE) : 0;
    if (kind == K_ISTA) {
      const Geo& g = p->gi;
      e = launch_mid(MID_FWD, kparams(p, g, 0), s);
      if (e == cudaSuccess) e = launch_col(COL_RESIDUAL, kparams(p, g, flags), s);
      if (e == cudaSuccess) e = launch_mid(MID_ADJ, kparams(p, g, 0), s);
      if (e == cudaSuccess)
        e = launch_col((last && final_chunk) ? COL_ISTA_LAST : COL_ISTA, kparams(p, g, flags), s);
      if (e == cudaSuccess && last) e = launch_finalize(p->partials, g.col_ctas, p->stats, s);
    } else {
      const Geo& g = p->ga;
      e = launch_mid(MID_ADMM, kparams(p, g, 0), s);
      if (e == cudaSuccess)
        e = launch_col((last && final_chunk) ? COL_ADMM_LAST : COL_ADMM, kparams(p, g, flags), s);
      if (e == cudaSuccess && last) e = launch_finalize(p->partials, g.col_ctas, p->stats, s);
    }
  }
  return e;
}

int chunk_kernels(SolveKind kind, int len) { return (kind == K_ISTA ? 4 : 2) * len + 1; }

cudaError_t run_chunk(cs_plan_s* p, SolveKind kind, int len, bool final_chunk) {
  p->launches += chunk_kernels(kind, len);
  if (!p->use_graphs) return enqueue_chunk(p, kind, len, final_chunk, p->stream);
  const uint64_t key = ((uint64_t)kind << 40) | ((uint64_t)final_chunk << 32) | (uint32_t)len;
  auto it = p->graphs.find(key);
  if (it == p->graphs.end()) {
    cudaError_t e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t e2 = enqueue_chunk(p, kind, len, final_chunk, p->cap);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(p->cap, &graph);
    if (e2 != cudaSuccess || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return e2 != cudaSuccess ? e2 : e;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    it = p->graphs.emplace(key, exec).first;
  }
  return cudaGraphLaunch(it->second, p->stream);
}

// Iterate in chunks of check_every; with a monitor tolerance, stop at the
// first check point whose NMSE meets it.
cudaError_t solve_loop(cs_plan_s* p, SolveKind kind, int iters, int* iters_run, int* converged,
                       bool need_stats) {
  *iters_run = 0;
  *converged = 0;
  const int ce = p->check_every;
  const bool watch = p->xtrue != nullptr && p->tol > 0.0;
  int done = 0;
  while (done < iters) {
    const int len = (iters - done) < ce ? (iters - done) : ce;
    const bool final_chunk = done + len == iters;
    cudaError_t e = run_chunk(p, kind, len, final_chunk);
    if (e != cudaSuccess) return e;
    done += len;
    if (watch && !final_chunk) {
      e = read_back(p);
      if (e != cudaSuccess) return e;
      const double nm = p->host_stats[ST_ERR2] / p->xtrue2;
      if (p->host_stats[ST_NONFIN] > 0.0) p->latched |= STS_NONFINITE;
      if (nm <= p->tol || (p->latched & STS_NONFINITE)) {
        *converged = nm <= p->tol;
        break;
      }
    }
  }
  *iters_run = done;
  if ((need_stats || watch) && done > 0) {
    cudaError_t e = read_back(p);
    if (e != cudaSuccess) return e;
    if (p->host_stats[ST_NONFIN] > 0.0) p->latched |= STS_NONFINITE;
    if (watch) *converged = p->host_stats[ST_ERR2] / p->xtrue2 <= p->tol;
  }
  return cudaSuccess;
}

void fill_stats(const cs_plan_s* p, cs_stats* st, int iters_run, int converged, double lambda, bool admm) {
  const double* h = p->host_stats;
  st->iters_run = iters_run;
  st->converged = converged;
  st->launches = p->launches;
  if (iters_run == 0) {
    st->nmse = NAN;
    st->rel_change = NAN;
    st->objective = NAN;
    return;
  }
  st->nmse = p->xtrue ? h[ST_ERR2] / p->xtrue2 : NAN;
  st->rel_change = h[ST_X2] > 0.0 ? std::sqrt(h[ST_DX2] / h[ST_X2]) : (h[ST_DX2] > 0.0 ? INFINITY : 0.0);
  st->objective = 0.5 * h[ST_R2] + lambda * h[ST_L1];
  st->launches = p->launches;
  (void)admm;
}

bool valid_ptr(const void* q) { return q != nullptr && ((uintptr_t)q & 7u) == 0; }

}  // namespace

namespace {
cs_status build_plan(cs_plan_t* out, int64_t n0, int64_t n1, int64_t m, const int64_t* rows, const double* c,
                     void* stream);
}  // namespace

extern "C" {

int cs_version(void) { return 100; }

const char* cs_status_string(cs_status s) {
  switch (s) {
    case CS_OK: return "CS_OK";
    case CS_ERR_ARG: return "CS_ERR_ARG";
    case CS_ERR_NOMEM: return "CS_ERR_NOMEM";
    case CS_ERR_CUDA: return "CS_ERR_CUDA";
    case CS_ERR_TIMEOUT: return "CS_ERR_TIMEOUT";
    case CS_ERR_NONFINITE: return "CS_ERR_NONFINITE";
    case CS_ERR_UNSUPPORTED: return "CS_ERR_UNSUPPORTED";
  }
  return "CS_UNKNOWN";
}

cs_status cs_plan(cs_plan_t* out, int64_t n, int64_t m, const int64_t* rows, const double* c, void* stream) {
  if (!out || !rows || !c) return CS_ERR_ARG;
  *out = nullptr;
  if (m < 1 || m > n) return CS_ERR_ARG;
  if (n < 64 || n > (int64_t(1) << 22) || (n & (n - 1)) != 0) return CS_ERR_UNSUPPORTED;
  return build_plan(out, 0, n, m, rows, c, stream);
}

cs_status cs_plan_2d(cs_plan_t* out, int64_t n0, int64_t n1, int64_t m, const int64_t* pix, const double* c2,
                     void* stream) {
  if (!out || !pix || !c2) return CS_ERR_ARG;
  *out = nullptr;
  if (n0 < 8 || n1 < 16 || n0 > 4096 || n1 > 4096 || (n0 & (n0 - 1)) != 0 || (n1 & (n1 - 1)) != 0)
    return CS_ERR_UNSUPPORTED;
  if (m < 1 || m > n0 * n1) return CS_ERR_ARG;
  return build_plan(out, n0, n1, m, pix, c2, stream);
}

}  // extern "C"

namespace {

// Plan of the 1D operator (n0 = 0, n = n1) or of the 2D blur of an n0 x n1
// image (flattened row-major, n = n0 n1): geometry, FP64 spectrum, tables,
// row masks.
cs_status build_plan(cs_plan_t* out, int64_t n0, int64_t n1, int64_t m, const int64_t* rows, const double* c,
                     void* stream) {
  const bool twod = n0 > 0;
  const int64_t n = twod ? n0 * n1 : n1;
  cs_plan_s* p = new (std::nothrow) cs_plan_s();
  if (!p) return CS_ERR_NOMEM;
  p->n = n;
  p->m = m;
  p->stream = static_cast<cudaStream_t>(stream);
  const char* env = std::getenv("CS_GRAPHS");
  p->use_graphs = !(env && env[0] == '0');
  const int lgn = ilog2(n);
  if (twod) {
    make_geo2d(p->gi, ilog2(n0), ilog2(n1) - 1);
    make_geo2d(p->ga, ilog2(n0), ilog2(n1));
  } else {
    make_geo(p->gi, lgn - 1);
    make_geo(p->ga, lgn);
  }
  if (!geo_ok(p->gi) || !geo_ok(p->ga)) {
    delete p;
    return CS_ERR_UNSUPPORTED;
  }

  int64_t* d_rows = nullptr;
  double* d_c = nullptr;
  double2* fa = nullptr;
  double2* fb = nullptr;
  cs_status st = CS_OK;
  auto fail = [&](cs_status s) {
    if (d_rows) cudaFree(d_rows);
    if (d_c) cudaFree(d_c);
    if (fa) cudaFree(fa);
    if (fb) cudaFree(fb);
    free_plan(p);
    return s;
  };
#define CS_PLAN_TRY(expr)                                  \
  do {                                                     \
    cudaError_t e_ = (expr);                               \
    if (e_ != cudaSuccess) return fail(cuda_status(e_));   \
  } while (0)

  CS_PLAN_TRY(init_pass_kernels());
  CS_PLAN_TRY(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));
  CS_PLAN_TRY(cudaEventCreate(&p->ev0));
  CS_PLAN_TRY(cudaEventCreate(&p->ev1));
  const int64_t words = n / 32;
  const int maxctas = p->ga.col_ctas > p->gi.col_ctas ? p->ga.col_ctas : p->gi.col_ctas;
  const int64_t npart = (int64_t)maxctas * NSTAT > 256 ? (int64_t)maxctas * NSTAT : 256;
  CS_PLAN_TRY(dalloc(&p->W, n));
  for (cs_plan_s::Sel* sel : {&p->si, &p->sa}) {
    CS_PLAN_TRY(dalloc(&sel->mask, words));
    CS_PLAN_TRY(dalloc(&sel->prefix, words));
    CS_PLAN_TRY(dalloc(&sel->pos, m));
    CS_PLAN_TRY(dalloc(&sel->ys, m));
  }
  CS_PLAN_TRY(dalloc(&p->rows32, m));
  for (float** b : {&p->xi_t, &p->xt_i, &p->xt_a, &p->av, &p->az, &p->amu, &p->anu, &p->ax})
    CS_PLAN_TRY(dalloc(b, n));
  CS_PLAN_TRY(dalloc(&p->partials, npart));
  CS_PLAN_TRY(dalloc(&p->stats, NSTAT));
  CS_PLAN_TRY(dalloc(&p->status, 1));
  CS_PLAN_TRY(dalloc(&p->ca, 1));
  CS_PLAN_TRY(dalloc(&p->tab_ista, tab_count(p->gi)));
  CS_PLAN_TRY(dalloc(&p->tab_admm_c, tab_count(p->ga)));
  CS_PLAN_TRY(dalloc(&p->tab_admm_b, tab_count(p->ga)));
  CS_PLAN_TRY(dalloc(&p->abs2, tab_count(p->ga)));
  CS_PLAN_TRY(dalloc(&p->twi, twiddle_count(p->gi)));
  CS_PLAN_TRY(dalloc(&p->twa, twiddle_count(p->ga)));
  CS_PLAN_TRY(dalloc(&p->dense, n));
  CS_PLAN_TRY(dalloc(&p->dense2, n));
  CS_PLAN_TRY(dalloc(&p->dense3, n));
  CS_PLAN_TRY(cudaMallocHost(reinterpret_cast<void**>(&p->host_stats), NSTAT * sizeof(double)));
  CS_PLAN_TRY(cudaMallocHost(reinterpret_cast<void**>(&p->host_status), sizeof(int)));
  CS_PLAN_TRY(dalloc(&d_rows, m));
  CS_PLAN_TRY(dalloc(&d_c, n));
  CS_PLAN_TRY(dalloc(&fa, n));
  CS_PLAN_TRY(dalloc(&fb, n));

  cudaStream_t s = p->stream;
  CS_PLAN_TRY(cudaMemcpyAsync(d_rows, rows, m * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  CS_PLAN_TRY(cudaMemcpyAsync(d_c, c, n * sizeof(double), cudaMemcpyHostToDevice, s));
  CS_PLAN_TRY(cudaMemsetAsync(p->status, 0, sizeof(int), s));
  CS_PLAN_TRY(cudaMemsetAsync(p->si.mask, 0, words * sizeof(uint32_t), s));
  CS_PLAN_TRY(cudaMemsetAsync(p->sa.mask, 0, words * sizeof(uint32_t), s));
  CS_PLAN_TRY(cudaMemsetAsync(p->stats, 0, NSTAT * sizeof(double), s));
  CS_PLAN_TRY(make_tables(p->gi, p->twi, s));
  CS_PLAN_TRY(make_tables(p->ga, p->twa, s));
  double2* chat = nullptr;
  if (twod) {
    CS_PLAN_TRY(launch_fft64_2d(d_c, fa, fb, n0, n1, &chat, s));
    CS_PLAN_TRY(launch_tab_ista2d(chat, p->gi, n0, n1, p->tab_ista, s));
    CS_PLAN_TRY(launch_tab_admm2d(chat, p->ga, n0, n1, p->tab_admm_c, p->abs2, s));
  } else {
    CS_PLAN_TRY(launch_fft64(d_c, fa, fb, n, &chat, s));
    CS_PLAN_TRY(launch_tab_ista(chat, p->gi, n, p->tab_ista, s));
    CS_PLAN_TRY(launch_tab_admm(chat, p->ga, n, p->tab_admm_c, p->abs2, s));
  }
  CS_PLAN_TRY(launch_tab_admm_b(p->abs2, (int)tab_count(p->ga), n, 1.0, 1.0, p->tab_admm_b, s));
  p->b_rho = 1.0;
  p->b_sigma = 1.0;
  CS_PLAN_TRY(launch_build_mask(d_rows, m, n, p->gi, 1, p->si.mask, p->status, s));
  CS_PLAN_TRY(launch_build_mask(d_rows, m, n, p->ga, 0, p->sa.mask, p->status, s));
  CS_PLAN_TRY(launch_prefix(p->si.mask, words, p->si.prefix, s));
  CS_PLAN_TRY(launch_prefix(p->sa.mask, words, p->sa.prefix, s));
  CS_PLAN_TRY(cudaMemcpyAsync(p->host_status, p->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CS_PLAN_TRY(cudaStreamSynchronize(s));
  if (*p->host_status & (STS_BAD_ROW | STS_DUP_ROW)) return fail(CS_ERR_ARG);
  CS_PLAN_TRY(launch_row_pos(d_rows, m, p->gi, 1, p->si.mask, p->si.prefix, p->si.pos, p->rows32, s));
  CS_PLAN_TRY(launch_row_pos(d_rows, m, p->ga, 0, p->sa.mask, p->sa.prefix, p->sa.pos, nullptr, s));
  CS_PLAN_TRY(cudaStreamSynchronize(s));
#undef CS_PLAN_TRY
  cudaFree(d_rows);
  cudaFree(d_c);
  cudaFree(fa);
  cudaFree(fb);
  (void)st;
  *out = p;
  return CS_OK;
}

}  // namespace

extern "C" {

cs_status cs_plan_destroy(cs_plan_t plan) {
  if (!plan) return CS_ERR_ARG;
  cudaStreamSynchronize(plan->stream);
  free_plan(plan);
  return CS_OK;
}

cs_status cs_status_sync(cs_plan_t p) {
  if (!p) return CS_ERR_ARG;
  CS_TRY(cudaMemcpyAsync(p->host_status, p->status, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  CS_TRY(cudaStreamSynchronize(p->stream));
  p->latched |= *p->host_status;
  const cs_status s = latched_status(p);
  p->latched = 0;
  CS_TRY(cudaMemsetAsync(p->status, 0, sizeof(int), p->stream));
  return s;
}

cs_status cs_forward(cs_plan_t p, const float* x, float* y) {
  if (!p || !valid_ptr(x) || !y) return CS_ERR_ARG;
  CallArgs a{};
  a.src = x;
  a.dst = p->dense;
  cudaStream_t s = p->stream;
  p->ista_args = p->admm_args = false;
  CS_TRY(launch_set_args(a, p->ca, s));
  CS_TRY(launch_col(COL_LOAD, kparams(p, p->gi, 0), s));
  CS_TRY(launch_mid(MID_FWD, kparams(p, p->gi, 0), s));
  CS_TRY(launch_col(COL_STORE, kparams(p, p->gi, 0), s));
  CS_TRY(launch_gather_rows(p->dense, p->rows32, p->m, y, s));
  return CS_OK;
}

cs_status cs_adjoint(cs_plan_t p, const float* r, float* x) {
  if (!p || !r || !valid_ptr(x)) return CS_ERR_ARG;
  cudaStream_t s = p->stream;
  CS_TRY(cudaMemsetAsync(p->dense, 0, p->n * sizeof(float), s));
  CS_TRY(launch_scatter_rows(r, p->rows32, p->m, p->dense, s));
  CallArgs a{};
  a.src = p->dense;
  a.dst = x;
  p->ista_args = p->admm_args = false;
  CS_TRY(launch_set_args(a, p->ca, s));
  CS_TRY(launch_col(COL_LOAD, kparams(p, p->gi, 0), s));
  CS_TRY(launch_mid(MID_ADJ, kparams(p, p->gi, 0), s));
  CS_TRY(launch_col(COL_STORE, kparams(p, p->gi, 0), s));
  return CS_OK;
}

cs_status cs_opnorm2(cs_plan_t p, int iters, double* L) {
  if (!p || !L || iters < 1) return CS_ERR_ARG;
  cudaStream_t s = p->stream;
  CS_TRY(launch_power_init(p->dense2, p->n, s));
  CS_TRY(launch_norm2(p->dense2, p->n, p->partials, p->stats + ST_X2, s));
  CallArgs a{};
  a.src = p->dense2;
  a.aux = p->dense;
  a.dst = p->dense2;
  p->ista_args = p->admm_args = false;
  CS_TRY(launch_set_args(a, p->ca, s));
  for (int it = 0; it < iters; ++it) {
    CS_TRY(launch_col(COL_LOAD_SCALED, kparams(p, p->gi, 0), s));
    CS_TRY(launch_mid(MID_FWD, kparams(p, p->gi, 0), s));
    CS_TRY(launch_col(COL_MASK, kparams(p, p->gi, 0), s));
    CS_TRY(launch_mid(MID_ADJ, kparams(p, p->gi, 0), s));
    CS_TRY(launch_col(COL_POWER_OUT, kparams(p, p->gi, FL_STATS), s));
    CS_TRY(launch_finalize(p->partials, p->gi.col_ctas, p->stats, s));
  }
  CS_TRY(read_back(p));
  *L = p->host_stats[ST_DX2];
  return latched_status(p);
}

cs_status cs_set_monitor(cs_plan_t p, const float* x_true, double nmse_tol, int check_every) {
  if (!p || check_every < 1) return CS_ERR_ARG;
  if (x_true && !valid_ptr(x_true)) return CS_ERR_ARG;
  p->check_every = check_every;
  p->tol = nmse_tol;
  p->xtrue = x_true;
  p->xtrue2 = 0.0;
  if (x_true) {
    CS_TRY(launch_norm2(x_true, p->n, p->partials, p->stats + ST_ERR2, p->stream));
    CS_TRY(launch_to_tile(x_true, p->xt_i, p->gi, 1, p->stream));
    CS_TRY(launch_to_tile(x_true, p->xt_a, p->ga, 0, p->stream));
    CS_TRY(read_back(p));
    p->xtrue2 = p->host_stats[ST_ERR2];
    if (!(p->xtrue2 > 0.0)) {
      p->xtrue = nullptr;
      return CS_ERR_ARG;
    }
  }
  return CS_OK;
}

cs_status cs_ista(cs_plan_t p, const float* y, float lambda, float tau, int iters, float* x, cs_stats* stats) {
  if (!p || !y || !valid_ptr(x) || !(lambda >= 0.f) || !(tau > 0.f) || iters < 0 || !std::isfinite(tau) ||
      !std::isfinite(lambda))
    return CS_ERR_ARG;
  cudaStream_t s = p->stream;
  if (stats) CS_TRY(cudaEventRecord(p->ev0, s));
  CallArgs a{};
  a.src = x;             // the prologue transforms x(0) in natural order
  a.x = p->xi_t;         // the iterate lives in tile order during the solve
  a.xtrue = p->xtrue ? p->xt_i : nullptr;
  a.thr = (float)((double)tau * (double)lambda);
  a.tau = tau;
  p->launches = 0;
  CS_TRY(launch_set_args(a, p->ca, s));
  CS_TRY(launch_scatter_y(y, p->si.pos, p->m, p->si.ys, p->status, s));
  p->launches += 2;
  p->ista_args = true;
  p->admm_args = false;
  int run = 0, conv = 0;
  if (iters > 0) {
    CS_TRY(launch_to_tile(x, p->xi_t, p->gi, 1, s));
    CS_TRY(launch_col(COL_LOAD, kparams(p, p->gi, 0), s));
    p->launches += 2;
    CS_TRY(solve_loop(p, K_ISTA, iters, &run, &conv, stats != nullptr));
    CS_TRY(launch_from_tile(p->xi_t, x, p->gi, 1, s));
    p->launches += 1;
  }
  if (stats) {
    CS_TRY(cudaEventRecord(p->ev1, s));
    CS_TRY(cudaMemcpyAsync(p->host_status, p->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CS_TRY(cudaEventSynchronize(p->ev1));
    CS_TRY(cudaStreamSynchronize(s));
    p->latched |= *p->host_status;
    fill_stats(p, stats, run, conv, lambda, false);
    float ms = 0.f;
    CS_TRY(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
    stats->ms = ms;
    return latched_status(p);
  }
  return CS_OK;
}

}  // extern "C"

namespace {

// Algorithm 3 on the plan's tile-ordered state.  Natural-order state pointers
// may be null (then that vector is neither read nor returned); warm reads
// v, z, mu, nu (all non-null) as the starting state.
cs_status admm_impl(cs_plan_t p, const float* y, float lambda, const cs_admm_params* prm, int iters, int warm,
                    float* x, float* z, float* mu, float* nu, float* v, cs_stats* stats) {
  cudaStream_t s = p->stream;
  if (stats) CS_TRY(cudaEventRecord(p->ev0, s));
  const size_t nb = p->n * sizeof(float);
  p->launches = 0;
  float* tiled[4] = {p->av, p->az, p->amu, p->anu};
  float* natural[4] = {v, z, mu, nu};
  for (int i = 0; i < 4; ++i) {
    if (warm) {
      CS_TRY(launch_to_tile(natural[i], tiled[i], p->ga, 0, s));
      p->launches += 1;
    } else {
      CS_TRY(cudaMemsetAsync(tiled[i], 0, nb, s));
    }
  }
  if (prm->rho != p->b_rho || prm->sigma != p->b_sigma) {
    CS_TRY(launch_tab_admm_b(p->abs2, (int)tab_count(p->ga), p->n, prm->rho, prm->sigma, p->tab_admm_b, s));
    p->launches += 1;
    p->b_rho = prm->rho;
    p->b_sigma = prm->sigma;
  }
  CallArgs a{};
  a.x = p->ax;
  a.z = p->az;
  a.mu = p->amu;
  a.nu = p->anu;
  a.v = p->av;
  a.xtrue = p->xtrue ? p->xt_a : nullptr;
  a.thr = (float)((double)lambda / prm->sigma);
  a.rho = (float)prm->rho;
  a.sigma = (float)prm->sigma;
  a.tau1 = (float)prm->tau1;
  a.tau2 = (float)prm->tau2;
  a.d_on = (float)(1.0 / (1.0 + prm->rho));
  a.d_off = (float)(1.0 / prm->rho);
  CS_TRY(launch_set_args(a, p->ca, s));
  CS_TRY(launch_scatter_y(y, p->sa.pos, p->m, p->sa.ys, p->status, s));
  p->launches += 2;
  p->admm_args = true;
  p->ista_args = false;
  int run = 0, conv = 0;
  if (iters > 0) {
    CS_TRY(launch_col(COL_ADMM_INIT, kparams(p, p->ga, 0), s));
    p->launches += 1;
    CS_TRY(solve_loop(p, K_ADMM, iters, &run, &conv, stats != nullptr));
  }
  float* outs_t[5] = {p->av, p->az, p->amu, p->anu, p->ax};
  float* outs_n[5] = {v, z, mu, nu, iters > 0 ? x : nullptr};
  for (int i = 0; i < 5; ++i) {
    if (!outs_n[i]) continue;
    CS_TRY(launch_from_tile(outs_t[i], outs_n[i], p->ga, 0, s));
    p->launches += 1;
  }
  if (x && iters == 0) CS_TRY(cudaMemsetAsync(x, 0, nb, s));
  if (stats) {
    CS_TRY(cudaEventRecord(p->ev1, s));
    CS_TRY(cudaMemcpyAsync(p->host_status, p->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CS_TRY(cudaStreamSynchronize(s));
    p->latched |= *p->host_status;
    fill_stats(p, stats, run, conv, lambda, true);
    float ms = 0.f;
    CS_TRY(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
    stats->ms = ms;
    return latched_status(p);
  }
  return CS_OK;
}

}  // namespace

extern "C" {

cs_status cs_admm_ex(cs_plan_t p, const float* y, float lambda, const cs_admm_params* prm, int iters, int warm,
                     float* x, float* z, float* mu, float* nu, float* v, cs_stats* stats) {
  if (!p || !y || !prm || !z || !mu || !nu || !v || !(lambda >= 0.f) || iters < 0 || !std::isfinite(lambda))
    return CS_ERR_ARG;
  if (!(prm->sigma > 0.0) || !(prm->rho > 0.0) || !(prm->tau1 > 0.0) || !(prm->tau2 > 0.0) ||
      !std::isfinite(prm->sigma) || !std::isfinite(prm->rho) || !std::isfinite(prm->tau1) ||
      !std::isfinite(prm->tau2))
    return CS_ERR_ARG;
  return admm_impl(p, y, lambda, prm, iters, warm, x, z, mu, nu, v, stats);
}

cs_status cs_profile_pass(cs_plan_t p, int pass_id, int reps) {
  if (!p || reps < 1 || pass_id < 0 || pass_id > 5) return CS_ERR_ARG;
  if (pass_id <= 3 && !p->ista_args) return CS_ERR_ARG;
  if (pass_id >= 4 && !p->admm_args) return CS_ERR_ARG;
  cudaStream_t s = p->stream;
  for (int r = 0; r < reps; ++r) {
    switch (pass_id) {
      case 0: CS_TRY(launch_mid(MID_FWD, kparams(p, p->gi, 0), s)); break;
      case 1: CS_TRY(launch_col(COL_RESIDUAL, kparams(p, p->gi, 0), s)); break;
      case 2: CS_TRY(launch_mid(MID_ADJ, kparams(p, p->gi, 0), s)); break;
      case 3: CS_TRY(launch_col(COL_ISTA, kparams(p, p->gi, 0), s)); break;
      case 4: CS_TRY(launch_mid(MID_ADMM, kparams(p, p->ga, 0), s)); break;
      default: CS_TRY(launch_col(COL_ADMM, kparams(p, p->ga, 0), s)); break;
    }
  }
  return CS_OK;
}

cs_status cs_admm(cs_plan_t p, const float* y, float lambda, float rho, int iters, float* z, cs_stats* stats) {
  if (!p || !y || !z || !(rho > 0.f) || !(lambda >= 0.f) || iters < 0) return CS_ERR_ARG;
  cs_admm_params prm{rho, rho, 1.0, 1.0};
  // zero start; only z is returned
  return admm_impl(p, y, lambda, &prm, iters, 0, nullptr, z, nullptr, nullptr, nullptr, stats);
}

}  // extern "C"

// ------------------------------------------------------------------ gradient

namespace {

// (Re)allocate the gradient buffers for ck checkpoints and segments of up to
// seg steps; cached graphs of the gradient (which hold the old addresses)
// are dropped.
cudaError_t grad_reserve(cs_plan_s* p, int ck, int seg) {
  auto& G = p->gr;
  if (G.ckpt && ck <= G.ck_cap && seg <= G.seg_cap) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return e;
  for (auto it = p->graphs.begin(); it != p->graphs.end();) {
    if ((it->first >> 40) >= 3) {
      cudaGraphExecDestroy(it->second);
      it = p->graphs.erase(it);
    } else {
      ++it;
    }
  }
  const int nck = ck > G.ck_cap ? ck : G.ck_cap, nseg = seg > G.seg_cap ? seg : G.seg_cap;
  void* old[] = {G.ckpt, G.seg, G.rseg, G.g, G.w, G.q, G.dy, G.W2, G.gacc, G.gpart, G.ca};
  for (void* b : old)
    if (b) cudaFree(b);
  G = cs_plan_s::Grad{};
  const size_t n = (size_t)p->n;
  e = dalloc(&G.ckpt, (size_t)nck * n);
  if (e == cudaSuccess) e = dalloc(&G.seg, (size_t)(nseg + 1) * n);
  if (e == cudaSuccess) e = dalloc(&G.rseg, (size_t)nseg * n);
  if (e == cudaSuccess) e = dalloc(&G.g, n);
  if (e == cudaSuccess) e = dalloc(&G.w, n);
  if (e == cudaSuccess) e = dalloc(&G.q, n);
  if (e == cudaSuccess) e = dalloc(&G.dy, (size_t)p->m);
  if (e == cudaSuccess) e = dalloc(&G.W2, n / 2);
  if (e == cudaSuccess) e = dalloc(&G.gacc, (size_t)tab_count(p->gi));
  if (e == cudaSuccess) e = dalloc(&G.gpart, (size_t)p->gi.col_ctas);
  if (e == cudaSuccess) e = dalloc(&G.ca, (size_t)nseg + 1);
  if (e == cudaSuccess) {
    G.ck_cap = nck;
    G.seg_cap = nseg;
  }
  return e;
}

// Run `enqueue` on the plan's stream, as a cached CUDA graph under `key`.
template <class F>
cudaError_t run_graph(cs_plan_s* p, uint64_t key, F&& enqueue) {
  if (!p->use_graphs) return enqueue(p->stream);
  auto it = p->graphs.find(key);
  if (it == p->graphs.end()) {
    cudaError_t e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t e2 = enqueue(p->cap);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(p->cap, &graph);
    if (e2 != cudaSuccess || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return e2 != cudaSuccess ? e2 : e;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    it = p->graphs.emplace(key, exec).first;
  }
  return cudaGraphLaunch(it->second, p->stream);
}

KParams kp_step(const cs_plan_s* p, int j, int flags) {
  KParams k = kparams(p, p->gi, flags);
  k.ca = p->gr.ca + j;
  return k;
}

// Replay of one segment: x(0) of the segment in seg[0]; step j writes r(j)
// and x(j+1).
cudaError_t enqueue_replay(cs_plan_s* p, int L, cudaStream_t s) {
  const Geo& g = p->gi;
  cudaError_t e = launch_col(COL_LOADT, kp_step(p, 0, 0), s);
  for (int j = 0; j < L && e == cudaSuccess; ++j) {
    e = launch_mid(MID_FWD, kp_step(p, j, 0), s);
    if (e == cudaSuccess) e = launch_col(COL_RES_SAVE, kp_step(p, j, 0), s);
    if (e == cudaSuccess) e = launch_mid(MID_ADJ, kp_step(p, j, 0), s);
    if (e == cudaSuccess) e = launch_col(COL_ISTA_SEG, kp_step(p, j, 0), s);
  }
  (void)g;
  return e;
}

// Reverse steps L-1 .. 0 of one segment (g holds dL/dx at its end).
cudaError_t enqueue_reverse(cs_plan_s* p, int L, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (int j = L - 1; j >= 0 && e == cudaSuccess; --j) {
    e = launch_col(COL_GRAD_W, kp_step(p, j, 0), s);
    if (e == cudaSuccess) e = launch_mid(MID_FWD, kp_step(p, j, 0), s);
    if (e == cudaSuccess) e = launch_col(COL_GRAD_MASK, kp_step(p, j, 0), s);
    if (e == cudaSuccess) e = launch_mid(MID_ADJ, kp_step(p, j, 0), s);
    if (e == cudaSuccess) e = launch_col(COL_GRAD_G, kp_step(p, j, 0), s);
    if (e == cudaSuccess) e = launch_col(COL_LOAD2, kp_step(p, j, 0), s);
    if (e == cudaSuccess) e = launch_mid(MID_CORR, kp_step(p, j, 0), s);
    if (e == cudaSuccess) e = launch_col(COL_LOAD2, kp_step(p, j, FL_PAIR2), s);
    if (e == cudaSuccess) e = launch_mid(MID_CORR, kp_step(p, j, FL_PAIR2), s);
  }
  return e;
}

}  // namespace

extern "C" {

cs_status cs_grad(cs_plan_t p, const float* y, float lambda, float tau, int T, int K, const float* gx_T,
                  float* dc, float* dlambda, float* dy) {
  if (!p || !y || !valid_ptr(gx_T) || !valid_ptr(dc) || !dlambda || !dy || T < 1 || K < 1 || K > T ||
      !(lambda >= 0.f) || !(tau > 0.f) || !std::isfinite(lambda) || !std::isfinite(tau))
    return CS_ERR_ARG;
  if (p->gi.twod) return CS_ERR_UNSUPPORTED;
  cudaStream_t s = p->stream;
  const int S = (T + K - 1) / K;   // segments; segment s covers steps [sK, min((s+1)K, T))
  CS_TRY(grad_reserve(p, S, K));
  auto& G = p->gr;
  const size_t n = (size_t)p->n;
  p->launches = 0;
  const float thr = (float)((double)tau * (double)lambda);

  // forward: T steps of Algorithm 1 from x(0) = 0, x(sK) kept
  CallArgs a{};
  a.x = p->xi_t;
  a.thr = thr;
  a.tau = tau;
  CS_TRY(launch_set_args(a, p->ca, s));
  CS_TRY(launch_scatter_y(y, p->si.pos, p->m, p->si.ys, p->status, s));
  CS_TRY(cudaMemsetAsync(p->xi_t, 0, n * sizeof(float), s));
  CS_TRY(cudaMemsetAsync(p->W, 0, n * sizeof(float), s));   // FFT of x(0) = 0
  p->launches += 2;
  for (int sg = 0; sg < S; ++sg) {
    const int L = (sg + 1) * K <= T ? K : T - sg * K;
    CS_TRY(cudaMemcpyAsync(G.ckpt + sg * n, p->xi_t, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    CS_TRY(run_chunk(p, K_ISTA, L, sg == S - 1));
  }
  p->ista_args = false;
  p->admm_args = false;

  // per-step arguments of a segment
  for (int j = 0; j <= K; ++j) {
    CallArgs b{};
    b.x = G.seg + j * n;
    b.z = G.seg + (j + 1) * n;
    b.v = G.rseg + j * n;
    b.mu = G.w;
    b.nu = G.q;
    b.dst = j < K ? G.g : dc;   // entry K: the output pass (dL/dc, natural order)
    b.aux = G.dy;
    b.thr = thr;
    b.tau = tau;
    CS_TRY(launch_set_args(b, G.ca + j, s));
  }
  p->launches += K + 1;
  CS_TRY(launch_to_tile(gx_T, G.g, p->gi, 1, s));
  CS_TRY(cudaMemsetAsync(G.gacc, 0, tab_count(p->gi) * sizeof(float4), s));
  CS_TRY(cudaMemsetAsync(G.gpart, 0, p->gi.col_ctas * sizeof(double), s));
  CS_TRY(cudaMemsetAsync(G.dy, 0, p->m * sizeof(float), s));
  p->launches += 1;

  // reverse, segment by segment: replay from the checkpoint, then back-propagate
  for (int sg = S - 1; sg >= 0; --sg) {
    const int L = (sg + 1) * K <= T ? K : T - sg * K;
    CS_TRY(cudaMemcpyAsync(G.seg, G.ckpt + sg * n, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    CS_TRY(run_graph(p, (uint64_t(3) << 40) | (uint32_t)L, [&](cudaStream_t st) { return enqueue_replay(p, L, st); }));
    CS_TRY(run_graph(p, (uint64_t(4) << 40) | (uint32_t)L, [&](cudaStream_t st) { return enqueue_reverse(p, L, st); }));
    p->launches += 1 + 4 * L + 9 * L;
  }

  // outputs: dL/dc from its spectrum, dL/dlambda = tau dL/dtheta, dL/dy by row
  CS_TRY(launch_mid(MID_FROM_ACC, kp_step(p, K, 0), s));
  CS_TRY(launch_col(COL_STORE, kp_step(p, K, 0), s));
  CS_TRY(launch_sum_scaled(G.gpart, p->gi.col_ctas, tau, dlambda, s));
  CS_TRY(launch_gather_rows(G.dy, p->si.pos, p->m, dy, s));
  p->launches += 4;
  return CS_OK;
}

}  // extern "C"

// ------------------------------------------------------------ ADMM gradient

namespace {

cudaError_t grad_admm_reserve(cs_plan_s* p, int ck, int seg) {
  auto& G = p->ga_;
  if (G.ckpt && ck <= G.ck_cap && seg <= G.seg_cap) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return e;
  for (auto it = p->graphs.begin(); it != p->graphs.end();) {   // graphs holding the old addresses
    if ((it->first >> 40) >= 5) {
      cudaGraphExecDestroy(it->second);
      it = p->graphs.erase(it);
    } else {
      ++it;
    }
  }
  const int nck = ck > G.ck_cap ? ck : G.ck_cap, nseg = seg > G.seg_cap ? seg : G.seg_cap;
  void* old[] = {G.ckpt, G.wseg, G.sseg, G.mub, G.nub, G.gz, G.gx, G.dy, G.Wr, G.gacc, G.gpart, G.ca};
  for (void* b : old)
    if (b) cudaFree(b);
  G = cs_plan_s::GradA{};
  const size_t n = (size_t)p->n;
  e = dalloc(&G.ckpt, (size_t)nck * 4 * n);
  if (e == cudaSuccess) e = dalloc(&G.wseg, (size_t)nseg * n);
  if (e == cudaSuccess) e = dalloc(&G.sseg, (size_t)nseg * n);
  for (float** b : {&G.mub, &G.nub, &G.gz, &G.gx})
    if (e == cudaSuccess) e = dalloc(b, n);
  if (e == cudaSuccess) e = dalloc(&G.dy, (size_t)p->m);
  if (e == cudaSuccess) e = dalloc(&G.Wr, n);
  if (e == cudaSuccess) e = dalloc(&G.gacc, (size_t)tab_count(p->ga));
  if (e == cudaSuccess) e = dalloc(&G.gpart, (size_t)p->ga.col_ctas);
  if (e == cudaSuccess) e = dalloc(&G.ca, 2 * (size_t)nseg + 2);
  if (e == cudaSuccess) {
    G.ck_cap = nck;
    G.seg_cap = nseg;
  }
  return e;
}

// Pass parameters of the ADMM gradient: the complex-n geometry, the reverse
// exchange buffer and accumulators, and the CallArgs entry `ca`.
KParams kp_admm(const cs_plan_s* p, const CallArgs* ca, float2* W, const float2* W2) {
  KParams k = kparams(p, p->ga, 0);
  k.pp.W = W;
  k.pp.W2 = const_cast<float2*>(W2);
  k.pp.gacc_a = p->ga_.gacc;
  k.pp.gpart = p->ga_.gpart;
  k.ca = ca;
  return k;
}

// Replay of one segment of L iterations from the state in (av, az, amu, anu):
// iteration j keeps the column transform of its forward pair (wseg[j]) and
// its soft-threshold input (sseg[j]).
cudaError_t enqueue_admm_replay(cs_plan_s* p, int L, cudaStream_t s) {
  auto& G = p->ga_;
  const size_t n = (size_t)p->n;
  cudaError_t e = launch_col(COL_ADMM_INIT, kp_admm(p, G.ca, p->W, nullptr), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(G.wseg, p->W, n * sizeof(float2), cudaMemcpyDeviceToDevice, s);
  for (int j = 0; j < L && e == cudaSuccess; ++j) {
    e = launch_mid(MID_ADMM, kp_admm(p, G.ca + j, p->W, nullptr), s);
    if (e == cudaSuccess) e = launch_col(COL_ADMM_SEG, kp_admm(p, G.ca + j, p->W, nullptr), s);
    if (e == cudaSuccess && j + 1 < L)
      e = cudaMemcpyAsync(G.wseg + (j + 1) * n, p->W, n * sizeof(float2), cudaMemcpyDeviceToDevice, s);
  }
  return e;
}

// Reverse of iterations L-1 .. 0 of one segment; `first`: the segment that
// ends at iteration T (its last iteration takes dL/dz(T), dL/dx(T)).
cudaError_t enqueue_admm_reverse(cs_plan_s* p, int L, bool first, cudaStream_t s) {
  auto& G = p->ga_;
  const size_t n = (size_t)p->n;
  const int K = G.seg_cap;
  cudaError_t e = cudaSuccess;
  for (int j = L - 1; j >= 0 && e == cudaSuccess; --j) {
    const CallArgs* ca = (first && j == L - 1) ? G.ca + 2 * K : G.ca + K + j;
    e = launch_col(COL_ADMM_REV, kp_admm(p, ca, G.Wr, nullptr), s);
    if (e == cudaSuccess) e = launch_mid(MID_ADMM_REV, kp_admm(p, G.ca + K + j, G.Wr, G.wseg + j * n), s);
  }
  return e;
}

}  // namespace

extern "C" cs_status cs_grad_admm(cs_plan_t p, const float* y, float lambda, const cs_admm_params* prm, int T, int K,
                                  const float* gz_T, const float* gx_T, float* dc, float* dlambda, float* dy) {
  if (!p || !y || !prm || !valid_ptr(gz_T) || (gx_T && !valid_ptr(gx_T)) || !valid_ptr(dc) || !dlambda || !dy ||
      T < 1 || K < 1 || K > T || !(lambda >= 0.f) || !std::isfinite(lambda) || !(prm->sigma > 0.0) ||
      !(prm->rho > 0.0) || !std::isfinite(prm->sigma) || !std::isfinite(prm->rho) || !std::isfinite(prm->tau1) ||
      !std::isfinite(prm->tau2))
    return CS_ERR_ARG;
  if (p->ga.twod) return CS_ERR_UNSUPPORTED;
  cudaStream_t s = p->stream;
  const int S = (T + K - 1) / K;   // segments; segment sg covers iterations [sg K, min((sg+1) K, T))
  CS_TRY(grad_admm_reserve(p, S, K));
  auto& G = p->ga_;
  const int Kc = G.seg_cap;
  const size_t n = (size_t)p->n, nb = n * sizeof(float);
  p->launches = 0;
  if (prm->rho != p->b_rho || prm->sigma != p->b_sigma) {
    CS_TRY(launch_tab_admm_b(p->abs2, (int)tab_count(p->ga), p->n, prm->rho, prm->sigma, p->tab_admm_b, s));
    p->launches += 1;
    p->b_rho = prm->rho;
    p->b_sigma = prm->sigma;
  }
  CallArgs a{};
  a.x = p->ax;
  a.z = p->az;
  a.mu = p->amu;
  a.nu = p->anu;
  a.v = p->av;
  a.thr = (float)((double)lambda / prm->sigma);
  a.rho = (float)prm->rho;
  a.sigma = (float)prm->sigma;
  a.tau1 = (float)prm->tau1;
  a.tau2 = (float)prm->tau2;
  a.d_on = (float)(1.0 / (1.0 + prm->rho));
  a.d_off = (float)(1.0 / prm->rho);
  CS_TRY(launch_set_args(a, p->ca, s));
  CS_TRY(launch_scatter_y(y, p->sa.pos, p->m, p->sa.ys, p->status, s));
  p->launches += 2;
  p->ista_args = false;
  p->admm_args = false;

  // forward: T iterations of Algorithm 3 from the zero state, the state
  // entering iteration sK kept
  float* state[4] = {p->av, p->az, p->amu, p->anu};
  for (float* b : state) CS_TRY(cudaMemsetAsync(b, 0, nb, s));
  CS_TRY(launch_col(COL_ADMM_INIT, kparams(p, p->ga, 0), s));
  p->launches += 1;
  for (int sg = 0; sg < S; ++sg) {
    const int L = (sg + 1) * K <= T ? K : T - sg * K;
    for (int i = 0; i < 4; ++i)
      CS_TRY(cudaMemcpyAsync(G.ckpt + (sg * 4 + i) * n, state[i], nb, cudaMemcpyDeviceToDevice, s));
    CS_TRY(run_chunk(p, K_ADMM, L, sg == S - 1));
  }

  // per-iteration arguments: replay (state in the plan's buffers), reverse,
  // the reverse of iteration T-1 (with dL/dz(T), dL/dx(T)), the output pass
  for (int j = 0; j < Kc; ++j) {
    CallArgs r = a;
    r.x = nullptr;
    r.aux = G.sseg + j * n;
    CS_TRY(launch_set_args(r, G.ca + j, s));
    CallArgs b = a;
    b.x = nullptr;
    b.z = nullptr;
    b.mu = G.mub;
    b.nu = G.nub;
    b.v = G.dy;
    b.aux = G.sseg + j * n;
    CS_TRY(launch_set_args(b, G.ca + Kc + j, s));
  }
  {
    CallArgs b = a;
    b.x = nullptr;
    b.z = nullptr;
    b.mu = G.mub;
    b.nu = G.nub;
    b.v = G.dy;
    const int jl = (T - (S - 1) * K) - 1;   // last iteration of the last segment
    b.aux = G.sseg + jl * n;
    b.src = G.gz;
    b.xtrue = gx_T ? G.gx : nullptr;
    CS_TRY(launch_set_args(b, G.ca + 2 * Kc, s));
    CallArgs o{};
    o.dst = dc;
    CS_TRY(launch_set_args(o, G.ca + 2 * Kc + 1, s));
  }
  p->launches += 2 * Kc + 2;
  CS_TRY(launch_to_tile(gz_T, G.gz, p->ga, 0, s));
  if (gx_T) CS_TRY(launch_to_tile(gx_T, G.gx, p->ga, 0, s));
  CS_TRY(cudaMemsetAsync(G.mub, 0, nb, s));
  CS_TRY(cudaMemsetAsync(G.nub, 0, nb, s));
  CS_TRY(cudaMemsetAsync(G.Wr, 0, n * sizeof(float2), s));
  CS_TRY(cudaMemsetAsync(G.gacc, 0, tab_count(p->ga) * sizeof(float2), s));
  CS_TRY(cudaMemsetAsync(G.gpart, 0, p->ga.col_ctas * sizeof(double), s));
  CS_TRY(cudaMemsetAsync(G.dy, 0, p->m * sizeof(float), s));
  p->launches += gx_T ? 2 : 1;

  // reverse, segment by segment: replay from the checkpoint, then back-propagate
  for (int sg = S - 1; sg >= 0; --sg) {
    const int L = (sg + 1) * K <= T ? K : T - sg * K;
    for (int i = 0; i < 4; ++i)
      CS_TRY(cudaMemcpyAsync(state[i], G.ckpt + (sg * 4 + i) * n, nb, cudaMemcpyDeviceToDevice, s));
    CS_TRY(run_graph(p, (uint64_t(5) << 40) | (uint32_t)L,
                     [&](cudaStream_t st) { return enqueue_admm_replay(p, L, st); }));
    const bool first = sg == S - 1;
    CS_TRY(run_graph(p, (uint64_t(6) << 40) | ((uint64_t)first << 32) | (uint32_t)L,
                     [&](cudaStream_t st) { return enqueue_admm_reverse(p, L, first, st); }));
    p->launches += 1 + 2 * L + 2 * L;
  }

  // outputs: dL/dc from its spectrum, dL/dlambda = sum / sigma, dL/dy by row
  CS_TRY(launch_mid(MID_ADMM_FROM_ACC, kp_admm(p, G.ca + 2 * Kc + 1, G.Wr, nullptr), s));
  CS_TRY(launch_col(COL_STORE_RE, kp_admm(p, G.ca + 2 * Kc + 1, G.Wr, nullptr), s));
  CS_TRY(launch_sum_scaled(G.gpart, p->ga.col_ctas, (float)(1.0 / prm->sigma), dlambda, s));
  CS_TRY(launch_gather_rows(G.dy, p->sa.pos, p->m, dy, s));
  p->launches += 4;
  return CS_OK;
}

// ------------------------------------------------------ grouped launches

namespace csk {

PlanView plan_view(cs_plan_s* p) {
  PlanView v{};
  v.kp_i = kparams(p, p->gi, 0);
  v.kp_a = kparams(p, p->ga, 0);
  GroupDesc& d = v.desc;
  d.gi = p->gi;
  d.ga = p->ga;
  d.m = p->m;
  d.pos_i = p->si.pos;
  d.ys_i = p->si.ys;
  d.pos_a = p->sa.pos;
  d.ys_a = p->sa.ys;
  d.xi_t = p->xi_t;
  d.av = p->av;
  d.az = p->az;
  d.amu = p->amu;
  d.anu = p->anu;
  return v;
}

cudaError_t plan_admm_table(cs_plan_s* p, double rho, double sigma, cudaStream_t s) {
  if (rho == p->b_rho && sigma == p->b_sigma) return cudaSuccess;
  cudaError_t e = launch_tab_admm_b(p->abs2, (int)tab_count(p->ga), p->n, rho, sigma, p->tab_admm_b, s);
  if (e == cudaSuccess) {
    p->b_rho = rho;
    p->b_sigma = sigma;
  }
  return e;
}

}  // namespace csk
