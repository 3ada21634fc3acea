/*
 * cs.h -- C ABI of the GB300 circulant compressed-sensing recovery library
 * (ISTA and ADMM on a partial circulant sensing matrix, arXiv 1707.02244).
 *
 * Problem (Sec. 1, Eq. 1 and Eq. 3; Sec. 4.3):
 *   y = A x* (+ noise),  A = P C,  C the n x n circulant with first row c,
 *   C[i][j] = c[(j - i) mod n] (Sec. 4.2), P keeping the m distinct rows
 *   `rows` of C.  Both solvers minimise 0.5 ||y - A x||^2 + lambda ||x||_1,
 *   which has the minimiser of Eq. 3 with alpha = lambda.
 *
 * Conventions shared by every call
 *   - Vectors passed to a call are DEVICE pointers to fp32 arrays on the
 *     current device, used on the stream given to cs_plan.  The n-vectors
 *     of cs_forward, cs_adjoint, cs_ista, cs_set_monitor and the gradient
 *     calls are 8-byte aligned (CS_ERR_ARG otherwise); every other vector,
 *     and the batch calls' concatenations, may start at any 4-byte offset.
 *     Calls are
 *     asynchronous with respect to the host unless a cs_stats pointer is
 *     passed (then the call waits for its own work to finish).
 *   - y[i] always pairs with row rows[i] as given to cs_plan (any order).
 *   - The caller owns every vector it passes; the plan owns all of its own
 *     memory (spectrum, tables, exchange buffer) and frees it in
 *     cs_plan_destroy.  The plan copies `rows` and `c`.
 *   - cs_plan: n a power of two with 64 <= n <= 4194304 (2^22); 1 <= m <= n.
 *     cs_plan_2d: n = n0 n1 up to 4096 x 4096 (limits at that call).
 *   - Argument errors are returned at once and nothing is launched.
 *     Errors found on the device (non-finite input, a wait that ran out) are
 *     latched in the plan and returned by cs_status_sync or by the next call
 *     that synchronises.
 *   - A plan is used from one host thread at a time and one stream.
 */
#ifndef CS_H
#define CS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cs_plan_s* cs_plan_t;

typedef enum {
  CS_OK = 0,
  CS_ERR_ARG = 1,          /* bad argument (null, range, duplicate row, ...) */
  CS_ERR_NOMEM = 2,        /* device allocation failed */
  CS_ERR_CUDA = 3,         /* a CUDA runtime call failed */
  CS_ERR_TIMEOUT = 4,      /* a bounded device-side wait ran out */
  CS_ERR_NONFINITE = 5,    /* NaN/Inf in y or in the iterates */
  CS_ERR_UNSUPPORTED = 6   /* size outside the supported set */
} cs_status;

/* Convergence record of the last check point of a solve.
 * ISTA: nmse = ||x_T - x*||^2 / ||x*||^2 (NaN without a monitor),
 *       rel_change = ||x_T - x_{T-1}|| / ||x_T||,
 *       objective = 0.5 ||y - A x_{T-1}||^2 + lambda ||x_{T-1}||_1.
 * ADMM: nmse of z_T, rel_change = ||x_T - z_T|| / ||z_T|| (primal residual),
 *       objective = 0.5 ||y - A x_T||^2 + lambda ||z_T||_1.
 * ms = elapsed stream time of the call (CUDA events). */
typedef struct {
  int iters_run;
  int converged;      /* 1 when the monitor's NMSE tolerance was met */
  double nmse;
  double rel_change;
  double objective;
  double ms;
  int launches;       /* kernels this call enqueued (graph nodes included) */
} cs_stats;

/* Algorithm 3 parameters, named as in the paper: sigma weighs x = z,
 * rho weighs v = C x, tau1 / tau2 are the dual steps (converges for
 * tau1 = tau2 in (0, (sqrt(5)+1)/2), Sec. 4.3). */
typedef struct {
  double sigma;
  double rho;
  double tau1;
  double tau2;
} cs_admm_params;

/* Build a plan for A = P C (Sec. 4.3).
 *   n, m      signal length and number of measurements
 *   rows      HOST int64[m], distinct, each in [0, n); any order
 *   c         HOST float64[n], first row of C (Sec. 4.2)
 *   stream    cudaStream_t (NULL = legacy default stream)
 * The spectrum chat = DFT(c) is computed on the GPU in FP64 and rounded to
 * fp32 tables; for ADMM, B = (rho C^T C + sigma I)^-1 is applied through its
 * FP64-computed spectrum 1/(rho |chat|^2 + sigma) ("initial inversion" of
 * Algorithm 3, done by FFT as Sec. 4.3 and Sec. 5.1 describe).
 * Synchronises the stream.  Errors: CS_ERR_ARG (null pointer, m out of
 * range, row out of range, duplicate row), CS_ERR_UNSUPPORTED (n),
 * CS_ERR_NOMEM, CS_ERR_CUDA. */
cs_status cs_plan(cs_plan_t* out, int64_t n, int64_t m, const int64_t* rows,
                  const double* c, void* stream);

/* Free the plan and all its device memory (synchronises the stream). */
cs_status cs_plan_destroy(cs_plan_t plan);

/* ||A||_2^2 by `iters` power iterations on A^T A (products as in
 * cs_forward / cs_adjoint; fixed seeded start).  A lower estimate that
 * improves with iters; Algorithm 1 wants tau in (0, ||A||^-2).
 * Result in *L (HOST double).  Synchronises. */
cs_status cs_opnorm2(cs_plan_t plan, int iters, double* L);

/* y = A x: x DEVICE float[n] in natural order, y DEVICE float[m] with
 * y[i] = (C x)[rows[i]] (Algorithm 1, residual step; Sec. 4.3). */
cs_status cs_forward(cs_plan_t plan, const float* x, float* y);

/* x = A^T r = C^T P^T r: r DEVICE float[m] paired with rows, x DEVICE
 * float[n] (Algorithm 1, gradient step). */
cs_status cs_adjoint(cs_plan_t plan, const float* r, float* x);

/* Attach a ground truth for NMSE monitoring.
 *   x_true     DEVICE float[n] (caller keeps it alive while the plan uses
 *              it) or NULL to detach
 *   nmse_tol   stop a solve once NMSE <= nmse_tol at a check point (<= 0:
 *              never stop early; NMSE is still reported)
 *   check_every  iterations between check points (>= 1; default 10)
 * Sec. 6 counts a signal as recovered once its error reaches 1e-4.
 * Synchronises (computes ||x*||^2 on the device). */
cs_status cs_set_monitor(cs_plan_t plan, const float* x_true, double nmse_tol,
                         int check_every);

/* ISTA (Algorithm 1) for `iters` iterations (fewer if the monitor stops it):
 *   r = y - A x;  x <- eta_{tau*lambda}(x + tau A^T r)   (Eq. 4 threshold)
 *   y      DEVICE float[m] paired with rows
 *   x      DEVICE float[n], in: x(0) (the paper starts from 0), out: x(T)
 *   stats  HOST cs_stats* or NULL (non-NULL: the call synchronises)
 * Errors: CS_ERR_ARG (null, lambda < 0, tau <= 0, iters < 0). */
cs_status cs_ista(cs_plan_t plan, const float* y, float lambda, float tau,
                  int iters, float* x, cs_stats* stats);

/* ADMM (Algorithm 3) from the zero state with sigma = rho = `rho` and
 * tau1 = tau2 = 1; z DEVICE float[n] receives the sparse estimate z(T).
 * Errors: CS_ERR_ARG (null, lambda < 0, rho <= 0, iters < 0). */
cs_status cs_admm(cs_plan_t plan, const float* y, float lambda, float rho,
                  int iters, float* z, cs_stats* stats);

/* ADMM (Algorithm 3) with every parameter and the state exposed.
 *   v, z, mu, nu  DEVICE float[n] each, the state of Algorithm 3 (v is the
 *                 folded v + mu of the loop's last line).  warm = 0: the
 *                 state is set to zero first (the paper's start); warm = 1:
 *                 the given state is the starting point.  On return they
 *                 hold the state after the last iteration.
 *   x             DEVICE float[n] or NULL: receives x(T)
 * Errors: CS_ERR_ARG (null state, sigma/rho <= 0, tau1/tau2 <= 0). */
cs_status cs_admm_ex(cs_plan_t plan, const float* y, float lambda,
                     const cs_admm_params* params, int iters, int warm,
                     float* x, float* z, float* mu, float* nu, float* v,
                     cs_stats* stats);

/* Measurement hook (no counterpart in the paper; Sec. 6 reports throughput
 * in iterations per second).  Enqueue `reps` back-to-back launches of one
 * pass kernel of the iteration on the plan's stream, reusing the arguments
 * of the plan's last cs_ista / cs_admm_ex call (the buffers it named must
 * still be alive; the pass overwrites them as a real iteration would):
 *   0 mid pass C x      1 column pass residual   2 mid pass C^T r
 *   3 column pass ISTA update                   4 mid pass ADMM x-update
 *   5 column pass ADMM updates
 * For timing with CUDA events around the call.  Errors: CS_ERR_ARG
 * (pass_id, reps < 1, no earlier solve of that kind). */
cs_status cs_profile_pass(cs_plan_t plan, int pass_id, int reps);

/* Plan of the 2D operator (Sec. 7, compressed deblurring): A = P H with H
 * the periodic blur of an n0 x n1 image, block-circulant with circulant
 * blocks, following Sec. 4.2's index rule in both axes:
 *   (H x)[i0][i1] = sum_{j0,j1} c2[(j0 - i0) mod n0][(j1 - i1) mod n1] x[j0][j1]
 * (a convolution with a point-spread function psf is c2[d] = psf[-d]).
 *   n0, n1  powers of two, 8 <= n0 <= 4096, 16 <= n1 <= 4096
 *   pix     HOST int64[m]: kept pixels, flattened row-major (i0 n1 + i1),
 *           distinct, in any order; y[i] pairs with pix[i]
 *   c2      HOST float64[n0 n1], row-major
 * The returned plan is used with cs_forward, cs_adjoint, cs_opnorm2,
 * cs_set_monitor, cs_ista, cs_admm, cs_admm_ex on flattened images of
 * n = n0 n1 values (cs_grad returns CS_ERR_UNSUPPORTED).  Errors as
 * cs_plan. */
cs_status cs_plan_2d(cs_plan_t* out, int64_t n0, int64_t n1, int64_t m, const int64_t* pix,
                     const double* c2, void* stream);

/* Gradient of unrolled ISTA (no counterpart in the paper: reverse mode
 * through T steps of Algorithm 1, for calibration of c, lambda or y by
 * gradient descent).  With x(0) = 0 and x(t+1) = eta_{tau lambda}(x(t) +
 * tau A^T (y - A x(t))) as cs_ista computes it, and gx_T = dL/dx(T) for any
 * loss L(x(T)):
 *   dc      DEVICE float[n]: dL/dc (c as given to cs_plan, natural order)
 *   dlambda DEVICE float[1]: dL/dlambda
 *   dy      DEVICE float[m]: dL/dy (y[i] pairs with rows[i] as given)
 * tau is held fixed (it is not differentiated through ||A||^2).  The
 * soft threshold's derivative is taken as 1 where |u| > tau lambda and 0
 * elsewhere (its value at the kink is a convention).
 * The forward iterates are kept every K steps (checkpoints, (T/K + 1) n
 * floats) and each segment of K steps is replayed before it is
 * back-propagated ((2K + 4) n more floats, allocated by the first call and
 * kept by the plan).  1 <= K <= T.  Asynchronous; errors as cs_ista.
 * Uses the plan's solver state: not concurrent with cs_ista / cs_admm. */
cs_status cs_grad(cs_plan_t plan, const float* y, float lambda, float tau, int T, int K,
                  const float* gx_T, float* dc, float* dlambda, float* dy);

/* Gradient of unrolled circulant ADMM (no counterpart in the paper: reverse
 * mode through T iterations of Algorithm 3).  From the zero state, with
 * the iteration cs_admm_ex computes for the parameters prm (sigma, rho,
 * tau1, tau2 of Algorithm 3), and a loss L(z(T), x(T)) of the last
 * iteration's sparse estimate z and x-update x:
 *   gz_T    DEVICE float[n]: dL/dz(T)
 *   gx_T    DEVICE float[n]: dL/dx(T), or NULL (L does not depend on x(T))
 *   dc      DEVICE float[n]: dL/dc (c as given to cs_plan, natural order)
 *   dlambda DEVICE float[1]: dL/dlambda
 *   dy      DEVICE float[m]: dL/dy (y[i] pairs with rows[i] as given)
 * c enters through C, C^T and the inverse B = (rho C^T C + sigma I)^-1; the
 * soft threshold's derivative is 1 where |x + nu| > lambda / sigma and 0
 * elsewhere.  The state entering every K-th iteration is kept (4 n floats
 * per checkpoint); each segment of K iterations is replayed, keeping per
 * iteration the transform of its forward pair (2 n floats) and the soft
 * threshold's input (n floats), and then back-propagated, each iteration
 * as one column pass and one mid pass.  Buffers are allocated by the first
 * call and kept by the plan.  1 <= K <= T; 1D plans only (a 2D plan
 * returns CS_ERR_UNSUPPORTED).  Asynchronous; errors as cs_admm_ex.  Uses
 * the plan's solver state: not concurrent with cs_ista / cs_admm. */
cs_status cs_grad_admm(cs_plan_t plan, const float* y, float lambda, const cs_admm_params* prm, int T, int K,
                       const float* gz_T, const float* gx_T, float* dc, float* dlambda, float* dy);

/* ---------------------------------------------------------------------
 * Batched solves (no counterpart in the paper; its recovery problem solved
 * for many independent instances at once).  Instance i has its own n_i,
 * m_i, rows and c.  Three solvers share a call:
 *   - power-of-two n_i <= CS_BATCH_MAX_N: one CTA per instance, the iterate
 *     kept in shared memory for all iterations (one launch per size class,
 *     on up to 4 internal streams forked from the batch's stream);
 *   - larger power-of-two n_i: the buffers and tables of a plan, iterated
 *     together (every pass of an iteration is one launch over the tiles of
 *     all of them; their whole solve is one CUDA graph launch);
 *   - 7-smooth n_i = 2^a 3^b 5^c 7^d that is not a power of two: mixed-radix
 *     FFTs (radices 8, 4, 2, 7, 5, 3), one CTA per instance up to n_i = 4096,
 *     above it a four-step split n_i = N1 N2 chosen by a plan-time tuner
 *     (cached per n for the process; CS_BATCH_AUTOTUNE=0 in the
 *     environment keeps the heuristic split; CS_BATCH_TUNE_CACHE=<file>
 *     keeps the tuned splits across processes as JSON keyed by the GPU's
 *     name, read once per process and rewritten after each new tuning).  All of these
 *     instances are solved by ONE persistent launch per call whose CTAs take
 *     (instance, pass, tile) items from a device-side queue; a tile waits,
 *     bounded, for its instance's previous pass (CS_ERR_TIMEOUT from
 *     cs_batch_status_sync if a wait ran out: each wait gives up after 2 s,
 *     every CTA then stops and the launch returns).  For tests only, the
 *     environment variable CS_BATCH_STALL_TEST=k raises every count the
 *     first such instance waits for by k, so that a wait runs out.
 * The concatenated vectors may hold instances of odd length: any 4-byte
 * offset is accepted.
 * --------------------------------------------------------------------- */
#define CS_BATCH_MAX_N 8192
typedef struct cs_batch_s* cs_batch_t;

/*   count     number of instances (>= 1)
 *   n, m      HOST int64[count]: n_i a power of two with 64 <= n_i <= 2^21,
 *             or 7-smooth with 16 <= n_i <= 2^20; 1 <= m_i <= n_i
 *   rows      HOST int64[sum m_i]: instance i's rows, concatenated
 *   c         HOST float64[sum n_i]: instance i's first row of C, concatenated
 * Synchronises.  Errors as cs_plan; CS_ERR_UNSUPPORTED for any other n_i. */
cs_status cs_batch_plan(cs_batch_t* out, int count, const int64_t* n, const int64_t* m,
                        const int64_t* rows, const double* c, void* stream);
cs_status cs_batch_destroy(cs_batch_t batch);

/* ISTA (Algorithm 1) on every instance for `iters` iterations.
 *   y       DEVICE float[sum m_i], instance i's measurements concatenated
 *   lambda, tau  HOST float[count]
 *   x       DEVICE float[sum n_i]: in x(0), out x(T), concatenated
 * Asynchronous. */
cs_status cs_batch_ista(cs_batch_t batch, const float* y, const float* lambda,
                        const float* tau, int iters, float* x);

/* ADMM (Algorithm 3, sigma = rho, tau1 = tau2 = 1, zero start) on every
 * instance; z DEVICE float[sum n_i] receives z(T).  rho HOST float[count].
 * Asynchronous. */
cs_status cs_batch_admm(cs_batch_t batch, const float* y, const float* lambda,
                        const float* rho, int iters, float* z);

/* Waits for the batch's work; returns the first error latched by a
 * per-instance plan, else CS_ERR_TIMEOUT if a bounded wait of the
 * mixed-radix solver ran out, else CS_ERR_NONFINITE if a measurement was
 * not finite.  The latched status is cleared (each condition is reported
 * once). */
cs_status cs_batch_status_sync(cs_batch_t batch);

/* Direct circulant product (context comparator; Sec. 5.2's scheme of one
 * O(n) dot product per output, not the FFT path).  No plan:
 *   c     DEVICE float[n]: first row of C (fp32)
 *   rows  DEVICE int32[m]: kept rows, 0 <= rows[i] < n (a row outside
 *         that range is not read from; its y[i] is NaN)
 *   x     DEVICE float[n];  y DEVICE float[m] receives (A x)_i = (C x)_{rows[i]}
 * O(m n) work, one warp per row.  Asynchronous on `stream`. */
cs_status cs_forward_direct(int64_t n, int64_t m, const float* c, const int32_t* rows,
                            const float* x, float* y, void* stream);

/* Largest n accepted by cs_circulant_apply_static. */
#define CS_STATIC_MAX_N 16384

/* Allocation-free circulant product (no counterpart in the paper).
 * For callers that cannot call cudaMalloc: code whose device memory is all
 * owned by another allocator (a framework's caching allocator or a fixed
 * pool), and latency-critical loops that cannot take the device
 * synchronisation an allocation may cause.  No plan is needed and nothing
 * is allocated: the FFT work space is a fixed 768 KiB array inside this
 * library, held on every GPU that loads it until the process exits.
 *   y = C x (transpose = 0) or C^T x (transpose != 0), C[i][j] = c[(j-i) mod n]
 *   n          power of two, 64 <= n <= CS_STATIC_MAX_N (else CS_ERR_UNSUPPORTED)
 *   c          DEVICE float64[n], first row of C
 *   x, y       DEVICE float32[n]
 *   stream     cudaStream_t (NULL = legacy default stream)
 * Computed in FP64 (FFT of c and x, spectrum product, inverse FFT), rounded
 * to fp32 once.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  The lookup is kept per device and
 * repeated when the device's current CUDA context has changed since (as
 * after cudaDeviceReset).  Every call uses the same array and overwrites all
 * of it that it reads, so calls that overlap on the GPU race: order them on
 * one stream.  Asynchronous; errors: CS_ERR_ARG (null pointer),
 * CS_ERR_UNSUPPORTED (n), CS_ERR_CUDA (a launch failed, or a CUDA error was
 * already pending on the calling thread when the call started: that error is
 * left pending for its owner and nothing is launched). */
cs_status cs_circulant_apply_static(int64_t n, const double* c, const float* x, float* y,
                                    int transpose, void* stream);

/* Wait for the plan's stream and return the latched device status
 * (CS_OK, CS_ERR_NONFINITE, CS_ERR_TIMEOUT), then clear it. */
cs_status cs_status_sync(cs_plan_t plan);

/* Static, human-readable name of a status code. */
const char* cs_status_string(cs_status s);

/* Library ABI version (major * 100 + minor). */
int cs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CS_H */
