/*
 * air.h -- C ABI of the GB300 (sm_103a) implementation of AIR, the fused
 * Analytical and Iterative Reconstruction method for CT (Yang, Gao, Qi & Gao,
 * arXiv 1310.1434).
 *
 * The library solves the paper's 2-D proof-of-concept problem
 *     min_X 1/2 ||P (A X - Y)||^2 + lambda ||W X||_1,   P = C^{1/2}   (Eqs. 1-3)
 * by split Bregman, whose L2 step is the paper's Eq. (5) system with the
 * split penalty added,
 *     (A'^T A + mu I) X = A'^T Y + mu W^T (d - b),   A'^T = A^T C,
 * solved by conjugate gradients.  A is the fan-beam X-ray transform (exact
 * Siddon intersection lengths), C the ramp filtration of FBP (Eq. 2) and W a
 * piecewise-linear tensor framelet.
 *
 * Conventions shared by every call
 *   - Lengths in mm, angles in radians.
 *   - Image X: n*n float32, row-major, X[iy*n + ix]; pixel (ix, iy) covers
 *     x in [x0 + ix*dx, x0 + (ix+1)*dx), y likewise, x0 = -n*dx/2 (the image
 *     is centred on the isocentre).
 *   - Sinogram Y: n_views*n_bins float32, Y[v*n_bins + j].
 *   - View v: beta_v = beta0 + arc*v/n_views, source at dso*(cos, sin)(beta_v).
 *     Bin j: fan angle gamma_j = (j - (n_bins-1)/2)*dgamma; the ray leaves the
 *     source at angle beta_v + pi + gamma_j and is the whole line.
 *   - Framelet coefficients: 9*n*n float32, band-major [9][n][n], band 3a+b is
 *     the tensor product of 1-D filter a (along y) and b (along x).
 *   - Array arguments are DEVICE pointers unless the name ends in _host.  They
 *     are owned by the caller, must be 16-byte aligned, contiguous, and must
 *     not alias each other (AIR_ERR_INVALID_ARG where this is checkable).
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *     default stream) unless stated; errors are returned as status codes, never
 *     thrown, and air_last_error() gives a thread-local message.
 *   - A plan owns device workspace; calls that use it must not overlap on the
 *     GPU for the same plan (issue them on one stream, or synchronise).
 */
#ifndef AIR_H
#define AIR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define AIR_API __attribute__((visibility("default")))
#else
#define AIR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AIR_OK = 0,
    AIR_ERR_INVALID_ARG = -1,  /* bad geometry, size, pointer or parameter */
    AIR_ERR_OOM = -2,          /* device allocation failed */
    AIR_ERR_CUDA = -3,         /* a CUDA runtime call failed */
    AIR_ERR_TIMEOUT = -4,      /* a bounded device-side wait gave up */
    AIR_ERR_BUDGET = -5,       /* request can never fit the server's HBM budget */
    AIR_ERR_NOT_READY = -6,    /* server request not finished yet */
    AIR_ERR_INTERNAL = -7      /* a host-side consistency check of a plan's tables failed */
} air_status;

enum { AIR_FILTER_NONE = 0, AIR_FILTER_RAMLAK = 1 };
enum { AIR_PREC_FP32 = 0, AIR_PREC_BF16X3 = 1 };

typedef void *air_stream;      /* cudaStream_t */

/* Fan-beam geometry (Materials section: TomoTherapy MVCT, equiangular fan). */
typedef struct {
    int32_t n;          /* image side N (square image), 1..4096 */
    double  pixel_mm;   /* pixel pitch dx > 0 */
    int32_t n_views;    /* V, 1..65536 */
    int32_t n_bins;     /* detector bins n_b, 1..8192 */
    double  dso_mm;     /* source to isocentre; >= n*dx/sqrt(2) + 8*dx (source outside the image) */
    double  dsd_mm;     /* source to detector; fixes only the physical bin size */
    double  dgamma;     /* bin angular pitch; 0 = automatic: 2 asin(n dx/(sqrt2 dso))/n_b */
    double  beta0;      /* first view angle */
    double  arc;        /* angular range of the views (2 pi for a full rotation) */
    int32_t filter;     /* AIR_FILTER_RAMLAK (AIR) or AIR_FILTER_NONE (IR: C = I) */
    int32_t precision;  /* AIR_PREC_FP32, or AIR_PREC_BF16X3: filter C on tensor cores */
} air_geometry;

typedef struct air_plan air_plan;
typedef struct air_server air_server;

/* Thread-local description of the last error on this thread ("" if none). */
AIR_API const char *air_last_error(void);

/* Builds the geometry tables (per-ray line parameters, per-view source data,
 * filter taps) and the solver workspace on the current CUDA device.  The plan
 * owns all of it; free with air_plan_destroy.  Synchronous. */
AIR_API air_status air_plan_create(const air_geometry *geom, air_plan **out);
AIR_API air_status air_plan_destroy(air_plan *plan);
/* Kernel configuration of a plan.  air_plan_create times the projector's
 * tile shape (views per block: 1, 2, 4 or 8, with 256/that bins) and the
 * backprojector's split of the views over blocks on the plan's geometry and
 * keeps the fastest (cached per geometry for the life of the process).
 * air_plan_tune overrides the choice (AIR_ERR_INVALID_ARG outside the
 * allowed values: bwd_view_parts in 1..*bwd_view_parts_max); results agree
 * to rounding whatever the configuration (the summation order over views
 * depends on the split).  Either pointer of air_plan_config may be NULL. */
AIR_API air_status air_plan_tune(air_plan *plan, int fwd_views_per_block, int bwd_view_parts);
AIR_API air_status air_plan_config(const air_plan *plan, int *fwd_views_per_block, int *bwd_view_parts,
                                   int *bwd_view_parts_max);

/* Status recorded on the device by the plan's kernels: AIR_OK, or
 * AIR_ERR_TIMEOUT if a bounded wait inside a kernel gave up (the kernel then
 * returned without its result).  Synchronises the device.  Reading a status
 * other than AIR_OK clears it, so a later call reports only later failures. */
AIR_API air_status air_plan_status(const air_plan *plan);

/* Diagnostic control of the bounded device-side waits; the paper has no
 * counterpart.  Every spin-wait inside the library's kernels gives up after a
 * poll budget (a few seconds) and records AIR_ERR_TIMEOUT instead of hanging:
 * the persistent batch kernel's grid barrier (reported by
 * air_solve_batch_persistent) and the tensor-core filter's wait for a
 * pipeline stage's operands (reported by air_plan_status and by the calls
 * that check it).  polls >= 0 sets that budget for kernels launched
 * afterwards on the current device, polls < 0 restores the default; with 0 a
 * wait gives up without polling, which lets a test drive the failure path.
 * The waits with which a kernel that gave up drains its own asynchronous
 * copies and tensor-core operations before it exits keep the default budget.
 * Synchronous; process-wide for the device. */
AIR_API air_status air_set_wait_budget(int64_t polls);
/* Device bytes the plan holds (tables + workspace). */
AIR_API size_t     air_plan_bytes(const air_plan *plan);

/* Y = A X: fan-beam X-ray transform, exact Siddon lengths (Eq. 1).
 * X: n*n, Y: n_views*n_bins (output). */
AIR_API air_status air_project(const air_plan *plan, const float *X, float *Y, air_stream stream);

/* Z = C Y: ramp filtration of every view along the bins (Eq. 2): the linear
 * convolution with the band-limited Ram-Lak taps h[0] = 1/4,
 * h[odd k] = -1/(pi k)^2, scaled by pi/(n_views dx^2); Z = Y when the plan's
 * filter is AIR_FILTER_NONE.  Uses the plan's precision (FP32 or split-BF16
 * tensor cores).  Y, Z: n_views*n_bins; Z may not alias Y. */
AIR_API air_status air_filter(const air_plan *plan, const float *Y, float *Z, air_stream stream);

/* X = A^T Y: the exact transpose of air_project (same per-(ray, pixel)
 * lengths, gathered per pixel, no atomics). */
AIR_API air_status air_backproject(const air_plan *plan, const float *Y, float *X, air_stream stream);

/* X = A'^T Y = A^T C Y: the filtered adjoint X-ray transform (Eqs. 4-6).
 * Uses the plan's workspace for C Y. */
AIR_API air_status air_filtered_backproject(const air_plan *plan, const float *Y, float *X,
                                    air_stream stream);

/* The filtered adjoint of air_filtered_backproject for callers that cannot
 * allocate device memory when they call it: for example code that runs under
 * a fixed device-memory budget with no cudaMalloc after start-up, or a host
 * thread that holds a lock which another thread's allocation would need.
 * The paper has no counterpart; this is a deployment variant.
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 *     Its one scratch buffer is a static device array of 2^22 floats (16 MB):
 *     the filtered sinogram, then as many of the backprojector's view parts
 *     (n*n floats each, up to the plan's tuned split) as fit beside it.
 *   - CUDA allocates that array when it first loads the code that holds it
 *     on a device.  air_plan_create does so and records the array's device
 *     address (cudaGetSymbolAddress), so every device on which a plan has
 *     been created holds the 16 MB until the process exits: create the plans
 *     before a device-memory budget closes.  A call on a device where no plan
 *     was created looks the address up itself (loading the code then); make
 *     such a call before any stream capture.  After a cudaDeviceReset, create
 *     a plan again on that device before calling.
 *   - n_views * n_bins must be <= 2^20 (1,048,576); larger plans get
 *     AIR_ERR_INVALID_ARG.
 *   - All calls on a device share the array; calls that overlap on the GPU
 *     race.  Each call writes every sample it later reads.
 *   - Applies the FP32 filter whatever the plan's precision; Y, X as for
 *     air_filtered_backproject, and the plan's tables are read, not its
 *     workspace. */
AIR_API air_status air_filtered_backproject_noalloc(const air_plan *plan, const float *Y, float *X,
                                                    air_stream stream);

/* adjoint == 0: out = W in  (in: n*n, out: 9*n*n);
 * adjoint != 0: out = W^T in (in: 9*n*n, out: n*n).  Periodic boundary;
 * W^T W = I. */
AIR_API air_status air_framelet(const air_plan *plan, const float *in, float *out, int adjoint,
                        air_stream stream);

/* One d/b update of the split-Bregman loop (Methods section, ref. [24]):
 *   t = W X + b;  d = soft(t, thresh) on bands 1..8, d = t on band 0;
 *   b <- t - d (in place);  g = W^T (d - b_new).
 * X: n*n, b: 9*n*n (in/out), g: n*n (out).  resid: device double, may be
 * NULL; receives ||W X - d||_2 accumulated in FP64.  thresh >= 0. */
AIR_API air_status air_shrink(const air_plan *plan, const float *X, float *b, float *g, float thresh,
                      double *resid, air_stream stream);

/* The AIR split-Bregman solve (Eq. 1 with R = ||W X||_1):
 *   X^0 = 0, b^0 = 0; for k < n_outer: n_cg CG steps on
 *   (A^T C A + mu I) X = A^T C Y + mu W^T (d - b) warm-started from X, then
 *   the d/b update with threshold lambda/mu.
 * Y: n_views*n_bins (input), X: n*n (output only).  resid: device, n_outer
 * doubles, may be NULL: ||W X - d||_2 after each outer step.  lambda >= 0,
 * mu > 0, n_outer >= 0, n_cg >= 0.  CG dot products and the residual norms
 * are accumulated in FP64 on the device; no host synchronisation inside. */
AIR_API air_status air_solve(const air_plan *plan, const float *Y, float lambda, float mu,
                     int n_outer, int n_cg, float *X, double *resid, air_stream stream);

/* L2-regularised AIR, Eq. (5): (A'^T A + lambda I) X = A'^T Y, A'^T = A^T C,
 * solved by n_cg conjugate-gradient steps from X = 0 (CG dots in FP64 on the
 * device).  Y: n_views*n_bins (input), X: n*n (output only).  lambda > 0,
 * 0 <= n_cg <= 100000.  Uses the plan's filter and precision. */
AIR_API air_status air_solve_l2(const air_plan *plan, const float *Y, float lambda, int n_cg, float *X,
                                air_stream stream);

/* Forward-backward splitting AIR (Methods, Eq. 6, the paper's ref. [25]) for
 *   min_X 1/2 ||P (A X - Y)||^2 + lambda ||W X||_1:
 *   X^0 = 0; for k < n_iter:
 *     X^{k+1/2} = X^k - step A'^T (A X^k - Y)            (Eq. 6)
 *     X^{k+1}   = W^T S_{step*lambda}(W X^{k+1/2})        (proximal step)
 * with S the soft threshold on the high-pass bands 1..8 (band 0 kept) and W
 * the tensor framelet (W^T W = I).  Y: n_views*n_bins, X: n*n (output only).
 * lambda >= 0, step > 0, 0 <= n_iter <= 100000. */
AIR_API air_status air_solve_fbs(const air_plan *plan, const float *Y, float lambda, float step, int n_iter,
                                 float *X, air_stream stream);

/* Fan-beam filtered backprojection, the analytic reconstruction the paper
 * compares AIR with (Materials: "FBP was used as the AR method"), by the
 * textbook equiangular algorithm for a full 2 pi scan:
 *   Q_v(j)  = alpha sum_k D cos(gamma_k) Y_v(k) g((j-k) alpha),
 *             g(0) = 1/(8 alpha^2), g(odd m) = -1/(2 pi^2 sin^2(m alpha)), g(even) = 0;
 *   X(x, y) = dbeta sum_v Q_v(gamma') / L^2   (gamma', L: fan angle and
 *             source distance of the pixel centre; Q linear between bins,
 *             zero beyond the detector; dbeta = 2 pi / n_views).
 * alpha = fan pitch, D = dso_mm.  Y: n_views*n_bins (input), X: n*n (output),
 * in the units of Y per mm.  AIR_ERR_INVALID_ARG unless the plan's arc is
 * 2 pi.  FP32 whatever the plan's precision; uses the plan's workspace. */
AIR_API air_status air_fbp(const air_plan *plan, const float *Y, float *X, air_stream stream);

/* air_solve from and to HOST memory: copies Y_host in, solves, copies X out
 * and synchronises the stream before returning.  Y_host/X_host may be
 * pageable or pinned. */
AIR_API air_status air_solve_host(const air_plan *plan, const float *Y_host, float lambda, float mu,
                          int n_outer, int n_cg, float *X_host, air_stream stream);

/* Many independent slices of uneven geometry solved together: every slice i
 * is solved as by air_solve(plans[i], Y[i], lambda[i], mu[i], n_outer[i],
 * n_cg[i], X[i]).  The programs advance phase by phase, each phase one
 * grouped launch over the tiles of its slices (FP32 and BF16X3 plans may be
 * mixed); the launch sequence is captured into a CUDA graph once per batch
 * composition and replayed by later calls with the same arguments.  The
 * graph runs the slices as one chain of phases or as two independent chains
 * (slice i in chain i mod 2); the first call of a composition runs both
 * graphs once (twice each when they are within 3 %), keeps the faster and
 * returns the last run's result, so it takes two to four times as long
 * (batches too large for two chains to pay are run once).  plans must be distinct (each slice uses its plan's
 * workspace).  Arrays of length n are HOST arrays; Y[i], X[i] are device
 * pointers.  Returns after the batch has finished (synchronises `stream`). */
AIR_API air_status air_solve_batch(int n, air_plan *const *plans, const float *const *Y,
                           const float *lambda, const float *mu, const int *n_outer,
                           const int *n_cg, float *const *X, air_stream stream);

/* Diagnostic description of the grouped batch graph in use (built by the
 * last air_solve_batch or air_solve_batch_host call that built one; the
 * paper has no counterpart): its number of chains (1 or 2) and the kernels
 * one run of it launches (one per grouped phase launch, two per tensor-core
 * filter application).  Either pointer may be NULL, not both.
 * AIR_ERR_INVALID_ARG if no batch graph exists yet. */
AIR_API air_status air_batch_graph_info(int *chains, int64_t *kernels);
/* air_solve_batch from and to HOST memory: Y_host[i] (n_views*n_bins floats)
 * is copied into plan i's staging buffer, the batch is solved there (the
 * staging buffers are fixed per plan, so repeated calls replay one captured
 * graph), and X_host[i] (n*n floats) receives the image.  Pinned host memory
 * makes the copies asynchronous.  Returns after the images are on the host. */
AIR_API air_status air_solve_batch_host(int n, air_plan *const *plans, const float *const *Y_host,
                                        const float *lambda, const float *mu, const int *n_outer,
                                        const int *n_cg, float *const *X_host, air_stream stream);
/* The same batch in ONE persistent cooperative kernel launch (captured in a
 * CUDA graph) whose blocks run every phase of every slice, separated by a
 * grid barrier with a bounded wait (AIR_ERR_TIMEOUT if it gives up).  FP32
 * plans only.  Synchronises `stream`. */
AIR_API air_status air_solve_batch_persistent(int n, air_plan *const *plans, const float *const *Y,
                           const float *lambda, const float *mu, const int *n_outer,
                           const int *n_cg, float *const *X, air_stream stream);

/* ---- serving: continuous batching of reconstruction requests ---------- */
/* A server owns one device worker thread.  Requests are admitted while the
 * device bytes of all resident requests stay within hbm_budget_bytes; a
 * request that arrives while others are running joins the running set at
 * the next step boundary, and all resident requests advance together, one
 * operator phase per device step.  max_slots bounds the resident set. */
AIR_API air_status air_server_create(size_t hbm_budget_bytes, int max_slots, air_server **out);
/* Queues one request; copies Y_host (n_views*n_bins floats) before returning.
 * AIR_ERR_BUDGET if the request alone exceeds the budget. */
AIR_API air_status air_server_submit(air_server *srv, const air_geometry *geom, const float *Y_host,
                             float lambda, float mu, int n_outer, int n_cg,
                             uint64_t *request_id);
/* AIR_OK and X copied to X_host (n*n floats, may be NULL) once the request
 * has finished (the request is then forgotten); AIR_ERR_NOT_READY before. */
AIR_API air_status air_server_poll(air_server *srv, uint64_t request_id, float *X_host);
/* Blocks until request_id has finished, then behaves like air_server_poll. */
AIR_API air_status air_server_wait(air_server *srv, uint64_t request_id, float *X_host);
/* Per-request timing in seconds since the server was created:
 * t[0] submit, t[1] admitted, t[2] finished.  Valid after completion and
 * before the result is polled. */
AIR_API air_status air_server_times(air_server *srv, uint64_t request_id, double t[3]);
/* Stops the worker after the resident requests finish and frees everything. */
AIR_API air_status air_server_destroy(air_server *srv);

#ifdef __cplusplus
}
#endif
#endif /* AIR_H */
