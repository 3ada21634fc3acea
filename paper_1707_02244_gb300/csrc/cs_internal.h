// Internal declarations shared by the host runtime and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

struct cs_plan_s;

namespace csk {

// Four-step geometry of one complex FFT of length N = N1 * N2, stored as an
// N2 x N1 row-major array (element p = j1 + N1 * j2).
//   column pass: length-N2 FFTs down the columns, G columns per CTA
//   mid pass:    length-N1 FFTs along the rows, U row pairs per CTA; row
//                pair unit u holds rows (u, N2 - u) for u >= 1 and rows
//                (0, N2/2) for u = 0, so every frequency k meets its mirror
//                N - k inside one CTA.
struct Geo {
  int N, lgN, N1, lgN1, N2, lgN2;
  int G, lgG, col_ctas;
  int U, lgU, mid_ctas;
  int tile;            // mid pass: complex values per CTA (4096 or 8192); threads = tile / 16
  int col_tile;        // column pass: complex values per CTA (4096, or 8192 for N2 = 4096)
  int twod;            // 1: 2D DFT of the N2 x N1 array (no four-step twiddle; pairs (k2, k1) ~ (-k2, -k1))
  const float2* tw1;   // exp(-2 pi i q / (2 N1)), q < 2 N1
  const float2* tw2;   // exp(-2 pi i q / N2),     q < N2
  const float2* twl;   // exp(-2 pi i q / N),      q < N1
  const float2* twr;   // exp(-2 pi i q / (2 N)),  q < N2
  const float2* tw1h;  // exp(-2 pi i q / N1),     q < N1
  const float2* tws1;  // stage-major twiddles of the length-N1 FFT
  const float2* tws2;  // stage-major twiddles of the length-N2 FFT
};

constexpr int NSTAT = 8;

// Statistic slots (partials[block * NSTAT + slot]).
enum : int {
  ST_ERR2 = 0,   // ||x - x*||^2           (ISTA: x_t, ADMM: z_t)
  ST_DX2 = 1,    // ISTA ||x_t - x_{t-1}||^2, ADMM ||x_t - z_t||^2
  ST_X2 = 2,     // ||x_t||^2 (ADMM ||z_t||^2)
  ST_L1 = 3,     // ISTA ||x_{t-1}||_1, ADMM ||z_t||_1
  ST_R2 = 4,     // ||y - A x||^2 (ISTA at x_{t-1}, ADMM at x_t)
  ST_NONFIN = 5  // count of non-finite iterate values
};

// Plan-constant device pointers, passed by value to every pass kernel.
struct PlanPtrs {
  float2* W;                 // exchange buffer, complex[n]
  const uint32_t* mask;      // rows of Omega, one bit per row in tile order, [n/32]
  const uint32_t* prefix;    // set bits before word w, [n/32]
  const float* ys;           // y in tile order of its rows, [m]
  double* partials;          // [max_ctas * NSTAT]
  double* stats;             // [NSTAT] finalised sums
  const float4* tab_ista;    // (P, Q) per pair slot, real-FFT geometry (see op_real)
  const float2* tab_admm_c;  // chat_k per pair slot, complex-n geometry
  const float* tab_admm_b;   // 1 / (n (rho |chat_k|^2 + sigma)) per pair slot
  int* status;               // device status word
  // unrolled-ISTA gradient (cs_grad) only
  float2* W2;                // second exchange buffer, complex[N] of the real-FFT geometry
  float4* gacc;              // per pair slot: accumulated spectrum at (k, k + N)
  double* gpart;             // per column CTA: accumulated dL/dtheta
  // unrolled-ADMM gradient (cs_grad_admm) only
  float2* gacc_a;            // per pair slot of the complex-n geometry: accumulated spectrum of dL/dc at k
};

// Per-call arguments, resident in device memory and written by a one-thread
// kernel at the start of each call (kernel parameters are captured when the
// launch is enqueued, so this is safe while earlier work is in flight).
struct CallArgs {
  const float* src;     // load source (x, scattered r, power vector)
  float* dst;           // store target
  float* aux;           // power iteration: normalised u
  const float* xtrue;   // monitor ground truth or null
  float* x;             // ISTA iterate / ADMM x output (may be null)
  float* z;
  float* mu;
  float* nu;
  float* v;
  float thr;            // ISTA tau*lambda, ADMM lambda/sigma
  float tau;            // ISTA step
  float rho, sigma, tau1, tau2, d_on, d_off;
};

struct KParams {
  Geo geo;
  PlanPtrs pp;
  const CallArgs* ca;
  int flags;
};

enum : int { FL_STATS = 1, FL_WRITE_STATE = 2, FL_POWER_SCALE = 4, FL_PAIR2 = 8 };

// Column-pass epilogues and mid-pass spectrum operators.
enum ColKind : int {
  COL_LOAD = 0,        // forward FFT of src (real-FFT geometry: src float[2N])
  COL_LOAD_SCALED,     // same, times 1/sqrt(stats[ST_X2]); copies it to aux
  COL_STORE,           // inverse FFT, store to dst
  COL_MASK,            // inverse, keep rows of Omega, forward
  COL_RESIDUAL,        // inverse, r = M (y - Cx), forward
  COL_ISTA,            // inverse, x <- eta(x + tau g), forward
  COL_ISTA_LAST,       // same without the forward FFT
  COL_POWER_OUT,       // inverse, w -> dst, stats <u, w>, ||w||^2
  COL_ADMM_INIT,       // complex-n geometry: forward FFT of (v) + i (z - nu)
  COL_ADMM,            // inverse, Algorithm 3 elementwise steps, forward
  COL_ADMM_LAST,       // same without the forward FFT
  // unrolled-ISTA gradient (real-FFT geometry, vectors in tile order)
  COL_LOADT,           // forward FFT of x (tile order)
  COL_RES_SAVE,        // as COL_RESIDUAL, and r -> v
  COL_ISTA_SEG,        // inverse, z <- eta(x + tau g) (x kept), forward
  COL_GRAD_W,          // w = dst on the support of z -> mu, dtheta partials, forward
  COL_GRAD_MASK,       // inverse, q = M C w -> nu, aux += tau P C w, forward
  COL_GRAD_G,          // inverse, dst = mu - tau C^T q
  COL_LOAD2,           // forward FFTs of (v, mu) -> (W, W2); with FL_PAIR2 of (nu, x)
  // unrolled-ADMM gradient (complex-n geometry, vectors in tile order)
  COL_ADMM_SEG,        // as COL_ADMM (no state written), and s = x + nu -> aux
  COL_ADMM_REV,        // inverse (b' + i C b'), reverse of one Algorithm 3 iteration, forward FFT of (p' + i x')
  COL_STORE_RE         // inverse FFT, real part -> dst
};
enum MidKind : int {
  MID_FWD = 0, MID_ADJ, MID_ADMM,
  MID_CORR,            // forward FFTs of W and W2 -> gacc += s conj(a^) b^ (s = -1 with FL_PAIR2)
  MID_FROM_ACC,        // tau / N times the packed spectrum of gacc -> inverse FFT -> W
  // unrolled-ADMM gradient (complex-n geometry)
  MID_ADMM_REV,        // FFTs of W (p' + i x') and W2 (the forward pair): b' = B (C^T p' + x'), dL/dc spectrum
                       // -> gacc_a, inverse FFT of b' + i C b' -> W
  MID_ADMM_FROM_ACC    // the Hermitian spectrum of gacc_a -> inverse FFT -> W
};

// Launchers (cs_passes.cu).  Return cudaGetLastError() of the launch.
cudaError_t launch_col(ColKind kind, const KParams& kp, cudaStream_t s);
cudaError_t launch_mid(MidKind kind, const KParams& kp, cudaStream_t s);
size_t pass_smem_bytes(int tile);
cudaError_t init_pass_kernels();
cudaError_t init_col_kernels();
cudaError_t init_mid_kernels();
// Grouped launches over many plans (batched solves, run-time shapes,
// 4096-value tiles): CTA b runs tile map[b].y of the plan whose parameters
// are kps[map[b].x] (both device arrays).
cudaError_t launch_col_multi(ColKind kind, const KParams* kps, const int2* map, int nctas, cudaStream_t s);
cudaError_t launch_mid_multi(MidKind kind, const KParams* kps, const int2* map, int nctas, cudaStream_t s);
cudaError_t init_col_multi_kernels();
cudaError_t init_mid_multi_kernels();

// Small kernels (cs_aux.cu).
cudaError_t launch_set_args(const CallArgs& a, CallArgs* dst, cudaStream_t s);
cudaError_t launch_finalize(const double* partials, int nblk, double* stats, cudaStream_t s);
cudaError_t launch_twiddle(float2* dst, int count, int64_t M, cudaStream_t s);
cudaError_t launch_fft64(const double* c, double2* a, double2* b, int64_t n, double2** out,
                         cudaStream_t s);
// Forward FP64 FFT of the complex vector in a (b is work space); *out is
// whichever of a / b holds the result.
cudaError_t launch_fft64_complex(double2* a, double2* b, int64_t n, double2** out, cudaStream_t s);
cudaError_t launch_tab_ista(const double2* chat, const Geo& g, int64_t n, float4* tabA, cudaStream_t s);
// 2D: chat2 is the n0 x n1 FP64 spectrum (row-major); g the 2D geometry.
cudaError_t launch_tab_ista2d(const double2* chat2, const Geo& g, int64_t n0, int64_t n1, float4* tabA,
                              cudaStream_t s);
cudaError_t launch_tab_admm2d(const double2* chat2, const Geo& g, int64_t n0, int64_t n1, float2* tabc,
                              double* abs2, cudaStream_t s);
// FP64 2D DFT of the real n0 x n1 array c2 (row-major); a, b work space of
// n0 n1 values each; *out is whichever holds the result.
cudaError_t launch_fft64_2d(const double* c2, double2* a, double2* b, int64_t n0, int64_t n1, double2** out,
                            cudaStream_t s);
// Pair slots of the mid pass (spectrum tables' length).
inline int64_t tab_count(const Geo& g) { return ((int64_t)(g.N2 >> 1) << g.lgN1) + (g.twod ? 2 : 1); }
cudaError_t launch_stage_tw(float2* dst, int lgL, int count, cudaStream_t s);
cudaError_t launch_tab_admm(const double2* chat, const Geo& g, int64_t n, float2* tabc,
                            double* abs2, cudaStream_t s);
cudaError_t launch_tab_admm_b(const double* abs2, int count, int64_t n, double rho,
                              double sigma, float* tabb, cudaStream_t s);
// Row mask of Omega in the tile order of geometry g (packed: two spatial rows
// per complex element, the real-FFT geometry).
cudaError_t launch_build_mask(const int64_t* rows, int64_t m, int64_t n, const Geo& g, int packed,
                              uint32_t* mask, int* status, cudaStream_t s);
// Natural order <-> tile order of the column pass (float2 elements when
// complex_elems, else float), g.N elements.
cudaError_t launch_to_tile(const void* nat, void* tiled, const Geo& g, int complex_elems, cudaStream_t s);
cudaError_t launch_from_tile(const void* tiled, void* nat, const Geo& g, int complex_elems, cudaStream_t s);
cudaError_t launch_prefix(const uint32_t* mask, int64_t words, uint32_t* prefix,
                          cudaStream_t s);
cudaError_t launch_row_pos(const int64_t* rows, int64_t m, const Geo& g, int packed,
                           const uint32_t* mask, const uint32_t* prefix, int32_t* pos,
                           int32_t* rows32, cudaStream_t s);
cudaError_t launch_scatter_y(const float* y, const int32_t* pos, int64_t m, float* ys,
                             int* status, cudaStream_t s);
cudaError_t launch_gather_rows(const float* dense, const int32_t* rows32, int64_t m,
                               float* y, cudaStream_t s);
cudaError_t launch_scatter_rows(const float* r, const int32_t* rows32, int64_t m,
                                float* dense, cudaStream_t s);
cudaError_t launch_norm2(const float* x, int64_t n, double* partials, double* out,
                         cudaStream_t s);
cudaError_t launch_power_init(float* u, int64_t n, cudaStream_t s);
// out[0] = scale * sum(v[0 .. count)), summed in a fixed order in FP64.
cudaError_t launch_sum_scaled(const double* v, int count, float scale, float* out, cudaStream_t s);

// One plan of a grouped (batched) solve: what the grouped element-wise
// kernels need of it.
struct GroupDesc {
  Geo gi, ga;                  // real-FFT and complex-n geometry
  int64_t noff, moff, m;       // offsets of its x / z and y in the concatenated vectors; rows kept
  const int32_t* pos_i;        // compact position of y[i], real-FFT geometry
  float* ys_i;
  const int32_t* pos_a;        // the same, complex-n geometry
  float* ys_a;
  float* xi_t;                 // ISTA iterate (tile order of gi, float2[n/2])
  float *av, *az, *amu, *anu;  // ADMM state (tile order of ga)
};

// The plan's parameters of the pass kernels (flags 0, its own CallArgs), its
// geometries and buffers, for grouped launches (cs_api.cu).
struct PlanView {
  KParams kp_i, kp_a;          // real-FFT and complex-n geometry
  GroupDesc desc;
};
PlanView plan_view(cs_plan_s* p);
// Re-tabulate the plan's ADMM inverse spectrum for (rho, sigma) when it holds
// another pair.
cudaError_t plan_admm_table(cs_plan_s* p, double rho, double sigma, cudaStream_t s);

// Grouped element-wise kernels over `count` plans (cs_aux.cu): compact y of
// every plan (geometry: 0 real-FFT, 1 complex-n; non-finite values latch
// STS_NONFINITE in *status); x (natural order) to and from the ISTA iterates;
// the zero ADMM state; z from the ADMM state.
cudaError_t launch_group_scatter_y(const GroupDesc* d, int count, const float* y, int geo, int* status,
                                   cudaStream_t s);
cudaError_t launch_group_ista_in(const GroupDesc* d, int count, const float* x, cudaStream_t s);
cudaError_t launch_group_ista_out(const GroupDesc* d, int count, float* x, cudaStream_t s);
cudaError_t launch_group_admm_zero(const GroupDesc* d, int count, cudaStream_t s);
cudaError_t launch_group_admm_out(const GroupDesc* d, int count, float* z, cudaStream_t s);

// Device status bits.
enum : int { STS_NONFINITE = 1, STS_TIMEOUT = 2, STS_BAD_ROW = 4, STS_DUP_ROW = 8 };

// Batched instances whose n is 7-smooth but not a power of two (cs_smooth.cu):
// mixed-radix FFTs, one persistent launch per solve.  smooth_plan takes the
// batch's arrays and the `count` instances ids[] (rows and c as the batch
// plan's; noff / moff their offsets); status is the batch's status word.
struct SmoothSet;
bool smooth_size(int64_t n);
int smooth_plan(SmoothSet** out, const int* ids, int count, const int64_t* n, const int64_t* m,
                const int64_t* noff, const int64_t* moff, const int64_t* rows, const double* c, int* status,
                cudaStream_t s);
cudaError_t smooth_ista(SmoothSet* q, const float* y, const float* lambda, const float* tau, int iters, float* x,
                        cudaStream_t s);
cudaError_t smooth_admm(SmoothSet* q, const float* y, const float* lambda, const float* rho, int iters, float* z,
                        cudaStream_t s);
void smooth_free(SmoothSet* q);

}  // namespace csk
