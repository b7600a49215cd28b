/*
 * map_smoother.h - C ABI of the GB300 parallel-in-time MAP trajectory smoother.
 *
 * Problem (Section 2.1, Eq. 1-2): estimate the trajectory x(t) of
 *     dx/dt = f(x, t) + L w(t),     y(t) = h(x, t) + nu(t),
 * with white noises of spectral densities W and R and prior x(t0) ~ N(m0, P0),
 * by minimising the Onsager-Machlup functional on the grid t_k = t0 + k dt,
 * k = 0..T.  The observations are samples y_k = h(x_k) + N(0, R/dt) for
 * k = 1..T (no measurement at t0).  Each interval [t_k, t_{k+1}] becomes one
 * conditional value-function element (A, b, C, eta, J) (Section 4.1-4.2,
 * Eq. 35-37; one explicit Euler step, or the exact exponential solution for
 * linear time-invariant drift); the filter is the reversed-time all-suffix
 * scan of Eq. (32) with the combine of Eq. (36); the smoother is either the
 * RTS-type composition of closed-loop maps (Section 4.3, Eq. 40-42) or the
 * two-filter combination (Section 4.3, Eq. 43 in information form); nonlinear
 * models are iterated on their linearisation (Section 4.4).
 *
 * Conventions
 *  - Host arrays in map_problem_desc are FP64, row-major, owned by the caller
 *    and read only during map_smoother_create.
 *  - Device arrays passed to solve/grad are owned by the caller, contiguous,
 *    row-major, in the handle's precision (float for MAP_FP32, double for
 *    MAP_FP64), resident on the device that was current at create time, and
 *    16-byte aligned.
 *  - y has T rows of ny values: row k-1 holds y_k, k = 1..T.
 *  - x_out has T+1 rows of nx values: row k holds x*_k, k = 0..T.
 *  - The handle owns its device workspace; destroy frees it.
 *  - Calls enqueue work on the given CUDA stream (cudaStream_t passed as
 *    void*, NULL = legacy default stream) and return without waiting, except
 *    where a host output is requested (noted per call).
 *  - No exception crosses the ABI.  Every failure returns a negative status;
 *    map_smoother_last_error() describes the last one.
 */
#ifndef MAP_SMOOTHER_H
#define MAP_SMOOTHER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct map_smoother map_smoother;   /* opaque handle */

/*
 * Device errors.  The kernels never wait without a limit: a bulk copy into
 * shared memory or a grid barrier that does not complete within its poll limit
 * (about a second) is abandoned, and a pivot that is not positive even in FP64
 * is detected.  Either marks the launch's result invalid and raises a flag of
 * the handle in host-mapped memory.  Because solves are asynchronous, the flag
 * is reported by the handle's NEXT call that checks it: map_smoother_solve,
 * _solve_sequential, _dense and _grad check it before they launch; the calls
 * that synchronise (_solve_host, _grad, _stats, and _solve with cost_out) also
 * check it after their synchronisation.  That call returns MAP_ERR_TIMEOUT (a
 * wait ran out) or MAP_ERR_SINGULAR (a singular pivot), sets last_error and
 * clears the flag; the CUDA context stays usable and later calls run normally.
 */

typedef enum {
    MAP_OK = 0,
    MAP_ERR_INVALID_ARG = -1,   /* null pointer, bad enum, misaligned pointer */
    MAP_ERR_SHAPE = -2,         /* unsupported nx/ny combination, T < 1 */
    MAP_ERR_CUDA = -3,          /* a CUDA runtime call failed */
    MAP_ERR_SINGULAR = -4,      /* a matrix that must be invertible was not */
    MAP_ERR_TIMEOUT = -5,       /* a bounded device wait ran out (see "Device errors" below) */
    MAP_ERR_UNSUPPORTED = -6    /* valid request that this library does not implement */
} map_status;

typedef enum {
    MAP_MODEL_LINEAR = 0,       /* f = F x + c, h = H x + r (Eq. 14), time invariant */
    MAP_MODEL_COORD_TURN = 1,   /* Section 5.2, Eq. 46: nx = 5, ny = 2, range-bearing */
    MAP_MODEL_CUBIC = 2         /* f = F x + c - gamma x^3 (elementwise), h = H x + r */
} map_model;

typedef enum { MAP_FP64 = 0, MAP_FP32 = 1 } map_precision;

typedef enum {
    MAP_EULER = 0,              /* one explicit Euler step of Eq. 37 per interval */
    MAP_EXPM = 1,               /* exact A, b, C of Eq. 37 with constant coefficients; for
                                   nonlinear models per step, with the coefficients of the
                                   drift linearised at each Gauss-Newton iterate (Section 4.4) */
    MAP_AUTO = 2,               /* linear models: MAP_EXPM when |F|_inf dt > 0.05, else
                                   MAP_EULER; nonlinear models: MAP_EULER */
    MAP_BLOCK_EULER = 3,        /* Section 5.1 blocks: desc.substeps explicit Euler steps of all
                                   five rows of Eq. 37 per interval, the interval's sample held
                                   over its substeps (linear models, RTS smoother) */
    MAP_RICCATI_EXACT = 4       /* all five rows of Eq. 37 solved exactly with constant
                                   coefficients, the interval's sample held (the limit of
                                   MAP_BLOCK_EULER with many substeps; linear models, RTS) */
} map_discretisation;

typedef enum { MAP_RTS = 0, MAP_TWO_FILTER = 1 } map_smoother_kind;

typedef struct {
    int model;                  /* map_model */
    int nx, ny;                 /* state and measurement dimensions */
    int nw;                     /* columns of L (dimension of w) */
    int64_t T;                  /* number of intervals, >= 1 */
    double t0, dt;              /* grid t_k = t0 + k dt (t0 is unused by autonomous models) */
    const double *F, *c;        /* nx*nx, nx: linear / cubic drift (NULL c = 0) */
    const double *L, *W;        /* nx*nw, nw*nw: dispersion and spectral density, Q = L W L^T */
    const double *H, *r;        /* ny*nx, ny: linear measurement (NULL r = 0) */
    const double *R;            /* ny*ny: measurement spectral density (diagonal for nonlinear models) */
    const double *m0, *P0;      /* nx, nx*nx: Gaussian prior of x(t0) */
    double gamma;               /* cubic drift coefficient (MAP_MODEL_CUBIC) */
    int precision;              /* map_precision */
    int discretisation;         /* map_discretisation */
    int smoother;               /* map_smoother_kind */
    int gn_iters;               /* nonlinear models: number of linearisation iterations, >= 1 */
    double cond_max;            /* FP32: recompute a combine's (I + C J) inverse in FP64 when
                                   its infinity-norm condition estimate exceeds this (0 = 1e6);
                                   a diagonal pivot that fails the pivot test is first redone
                                   in FP32 with row pivoting, kept within this bound */
    int tile_threads;           /* threads per tile CTA: 32, 64 or 128 (0 = 128, reduced to fit) */
    int substeps;               /* MAP_BLOCK_EULER: Euler substeps per interval, 1..64 (0 = 10) */
    int steps_per_thread;       /* K of the scans, 1..64 (0 = chosen for whole waves of CTAs) */
} map_problem_desc;

/*
 * Validate the problem, discretise it on the device (Euler: Eq. 37 one step;
 * EXPM: Van Loan block exponentials in FP64) and allocate the workspace for T.
 * Synchronises the current device.  Returns MAP_ERR_SHAPE for (nx, ny) pairs
 * without compiled kernels (see map_smoother_supported).
 */
map_status map_smoother_create(map_smoother** out, const map_problem_desc* desc);

/*
 * MAP trajectory for observations y (device, T x ny).
 *   x_out     device, (T+1) x nx.  For nonlinear models it must hold, on entry,
 *             the trajectory of the first linearisation (x̄ of Section 4.4);
 *             on exit it holds the estimate after desc.gn_iters iterations.
 *   filt_out  device or NULL: (T+1) x (nx + nx(nx+1)/2) filter value functions
 *             V(x) = 1/2 x^T S_k x - v_k^T x, row k = [v_k, packed upper S_k]
 *             (S = P^-1 and v = P^-1 m of the Kalman-Bucy filter, Section 2.5);
 *             for nonlinear models those of the last iteration.
 *   cost_out  host or NULL: the discrete Onsager-Machlup cost of x_out (needs an
 *             invertible Q; synchronises the stream).
 * Asynchronous on `stream` unless cost_out is given.  Calls on one handle
 * must be ordered (one stream, or synchronised between streams): the handle's
 * workspace and its grid-barrier counter are shared by its solves.  Under
 * stream capture the solve records the multi-kernel pipeline (the single
 * cooperative launch keeps per-launch state that a graph replay would reuse).
 */
map_status map_smoother_solve(map_smoother* h, const void* y, void* x_out, void* filt_out,
                              double* cost_out, void* stream);

/*
 * Dense output between the grid points of a MAP_BLOCK_EULER handle
 * (Section 4.3, recovery of x*(tau) inside the intervals): for every interval
 * k the filter value function at x_k is carried across the interval's
 * substeps by the one-variable combine of Eq. 36 with the substep elements,
 * and the smoothed x_{k+1} is taken back through the substeps' closed-loop
 * maps (Eq. 40-41).
 *   y          device, T x ny: the observations of the solve;
 *   x          device, (T+1) x nx: the solve's trajectory;
 *   filt       device, (T+1) x (nx + nx(nx+1)/2): the solve's filter output
 *              (map_smoother_solve filt_out);
 *   dense_out  device, (T substeps + 1) x nx: row k substeps + j holds the
 *              state at t_k + j dt / substeps.
 * Asynchronous on `stream`.  MAP_ERR_UNSUPPORTED for other discretisations.
 */
map_status map_smoother_dense(map_smoother* h, const void* y, const void* x, const void* filt,
                              void* dense_out, void* stream);

/*
 * Sequential baseline on the GPU: the same elements, information-filter
 * recursion (Eq. 17 in discrete form, one element per step) and closed-loop
 * maps as map_smoother_solve, evaluated by a single GPU thread in time order
 * with no associative scan (the paper's sequential counterpart).  Same
 * arguments and results as map_smoother_solve without the optional outputs;
 * nonlinear models iterate desc.gn_iters times.  Asynchronous on `stream`.
 */
map_status map_smoother_solve_sequential(map_smoother* h, const void* y, void* x_out, void* stream);

/*
 * End-to-end variant with HOST buffers: copies y_host (T x ny) to the device,
 * solves, copies the estimate back to x_host ((T+1) x nx) and synchronises
 * the stream.  For nonlinear models x_host also carries the first
 * linearisation trajectory in.  Pinned host memory gives the fastest copies.
 */
map_status map_smoother_solve_host(map_smoother* h, const void* y_host, void* x_host,
                                   void* stream);

/*
 * Gradient of a loss of the MAP trajectory with respect to
 * theta = (F (nx*nx, row-major), log q, log r), where Q = q L W L^T and
 * R = r R_desc; q = r = 1 at create and map_smoother_update changes them.
 * The MAP trajectory x* = argmin M(x; theta) of the discrete cost solves
 * K(theta) x* = g(theta) with K symmetric, so (implicit-function adjoint):
 *   dL_dx != NULL: lambda = K^-1 dL/dx is the MAP trajectory of the same
 *     problem with b = 0, the measurement information vectors replaced by
 *     dL/dx_{k+1} and the prior term by dL/dx_0 (same scans as solve);
 *     dL/dtheta = -d_theta [lambda^T grad_x M(x*, theta)] at fixed x*, lambda.
 *   dL_dx == NULL: L = M(x*(theta), theta), the MAP cost itself (Eq. 2,
 *     constants omitted; flags & MAP_GRAD_LOGDET adds the Gaussian
 *     log-normalisers 1/2 sum log det(2 pi C_k) + 1/2 sum log det(2 pi R/dt));
 *     dL/dtheta = d_theta M at x* (envelope theorem).
 *   y, x      device arrays of the solve (x = its result), dL_dx device (T+1) x nx.
 *   dL_dtheta host, nx*nx + 2 values (synchronises the stream).
 * Linear models with Euler elements and invertible Q only (else
 * MAP_ERR_UNSUPPORTED).  No per-step state of the forward solve is kept: the
 * adjoint re-runs the blocked scan, whose per-tile prefixes (one per 2048
 * steps) are its only stored checkpoints.
 */
#define MAP_GRAD_LOGDET 1
map_status map_smoother_grad(map_smoother* h, const void* y, const void* x, const void* dL_dx,
                             int flags, double* dL_dtheta, void* stream);

/*
 * The Gaussian log-normalisers that the MAP cost of map_smoother_solve
 * (cost_out) omits, at the handle's current parameters:
 *   *out = T/2 log det(2 pi C) + T/2 log det(2 pi R / dt),  C = dt q L W L^T,
 * the per-interval transition covariance of the Euler element (Section 4.2)
 * and the measurement covariance of a sample over dt.  Their derivative is the
 * MAP_GRAD_LOGDET share of map_smoother_grad.  Host arithmetic, no device
 * work.  MAP_ERR_UNSUPPORTED for nonlinear models or other than Euler
 * elements; MAP_ERR_SINGULAR when C or R is not positive definite.
 */
map_status map_smoother_log_normaliser(const map_smoother* h, double* out);

/*
 * Set theta = (F, log q, log r) of the handle (F NULL keeps F) and redo the
 * device set-up (discretisation); synchronises the device.  The plan-time
 * constants of linear time-invariant models (folds, tile tables, tile-map
 * products) are recomputed by the next solve, on its stream.  For training
 * loops that differentiate through the solve.  Returns MAP_ERR_INVALID_ARG
 * for non-finite log_q or log_r and MAP_ERR_SINGULAR when the updated R or
 * interval map A is singular.
 */
map_status map_smoother_update(map_smoother* h, const double* F, double log_q, double log_r);

/*
 * Device-side counters since create or the last reset: [0] combines
 * recomputed in FP64 (precision policy), [1] singular pivots met, [2] bounded
 * device waits (bulk copies, grid barriers) that ran out (the result of their
 * launch is invalid; expected to stay 0).  Synchronises the stream; out is
 * written, and the return value is then MAP_ERR_TIMEOUT / MAP_ERR_SINGULAR
 * when the handle's error flag was raised (see "Device errors").
 */
map_status map_smoother_stats(map_smoother* h, unsigned long long out[3], int reset, void* stream);

/*
 * Test of the device-error path without a fault or a hang: one CTA of 32
 * threads waits on a shared-memory mbarrier that nothing arrives on, with the
 * poll-limited wait of the solve kernels, then on a grid-barrier counter that
 * nothing advances (spin limit `polls`); each wait runs out and is reported
 * exactly as in a solve (counter [2] and the handle's error flag), so the next
 * checking call returns MAP_ERR_TIMEOUT.  polls must be 1..1048576
 * (MAP_ERR_INVALID_ARG otherwise).  Asynchronous on `stream`.
 */
map_status map_smoother_wait_selftest(map_smoother* h, int polls, void* stream);

/*
 * Per-phase device timing.  With profiling on, every solve records CUDA events
 * on its stream between its kernel launches; map_smoother_phase_times then
 * returns the durations (ms) of the phases of the last solve, in launch order.
 * For the RTS smoother:
 *   0 filter_reduce  per-thread folds and tile totals of the elements
 *   1 filter_down    per-tile prefix from the totals before the tile, per-step
 *                    filter values, closed-loop maps and their folds
 *   2 rts_down       per-tile end state from the maps after the tile, per-step
 *                    smoothed states
 * (for nonlinear models: those of the last iteration); for the two-filter
 * smoother: forward reduce, forward states, backward reduce, backward
 * combination.  phase_times synchronises the stream of the last solve;
 * *n_out receives the count.
 */
map_status map_smoother_profile(map_smoother* h, int enable);
map_status map_smoother_phase_times(map_smoother* h, float* ms_out, int cap, int* n_out);

/*
 * Launch geometry of the handle's scans (host-side read, no GPU work): steps
 * per thread K, threads per tile CTA B and the number of tiles ceil(T / (B K)).
 * K is chosen at create time so that the tiles fill whole waves of the CTAs
 * that the GPU keeps resident (at least 8, at most 64 steps per thread).
 * After a solve that ran the tiled scan with per-step tables
 * (MAP_PATH_TABLES), K and tiles are that scan's: K steps per thread of the
 * tiles after the stationary point and its number of tiles.
 * Returns MAP_ERR_INVALID_ARG for a NULL argument.
 */
map_status map_smoother_geometry(const map_smoother* h, int* K, int* B, int* tiles);

/*
 * Kernels launched by the handle's last solve (host-side read): 1 when the
 * linear time-invariant RTS solve ran as one cooperative launch (all tiles'
 * CTAs resident at once, not under stream capture), otherwise the number of kernels of the scan
 * pipeline (plan-time constant kernels not counted); 0 before the first solve.
 * Returns MAP_ERR_INVALID_ARG for a NULL argument.
 */
map_status map_smoother_launches(const map_smoother* h, int* kernels);

/*
 * How the last solve's scan ran (host-side read): 0 before the first solve;
 * MAP_PATH_TABLES: one cooperative launch that reads the per-step constants of
 * a linear time-invariant model from plan-time tables (the Riccati factors of
 * Eq. 36 do not depend on the data and converge to those of the stationary
 * filter); MAP_PATH_SINGLE: one cooperative launch that forms every step's
 * one-variable combine itself; MAP_PATH_PIPELINE: the multi-kernel scan.
 * Returns MAP_ERR_INVALID_ARG for a NULL argument.
 */
#define MAP_PATH_TABLES 1
#define MAP_PATH_SINGLE 2
#define MAP_PATH_PIPELINE 3
map_status map_smoother_solve_path(const map_smoother* h, int* path);

/*
 * Allocation-free solve (no counterpart in the paper; a deployment entry point).
 * For callers that cannot call cudaMalloc at all, e.g. code running where the
 * device-memory budget is fixed up front (a real-time tracking loop, an
 * embedded service that pre-reserves all device memory, a plug-in whose host
 * owns the allocator).  Same result as map_smoother_create + map_smoother_solve
 * for a linear model with the RTS smoother, without a handle: the model
 * set-up and the scan workspace use file-scope __device__ arrays of this
 * library (64 MiB of scratch plus a few KB), which every GPU on which this call
 * has run holds until the process exits.  No cudaMalloc, cudaFree or other
 * allocating routine is called.
 *   desc   problem description as for map_smoother_create (MAP_MODEL_LINEAR,
 *          smoother MAP_RTS); the launch geometry is fixed (16 steps per
 *          thread, 128 threads per tile; desc->tile_threads is ignored), and T
 *          is limited by the 64 MiB scratch: at most 632 832 intervals at
 *          nx = 4, ny = 2 in FP32 (329 728 in FP64).  Beyond the limit
 *          MAP_ERR_SHAPE is returned with a message naming the bytes needed.
 *   y, x_out  device arrays as for map_smoother_solve.
 * The model set-up synchronises `stream`; the solve kernels are then enqueued
 * on it asynchronously.  Every call, with the target device current, looks up
 * the device addresses of the arrays (cudaGetSymbolAddress, which allocates
 * nothing; not cached, so a context re-created after cudaDeviceReset is
 * handled).  The first call on a device loads the module; make it before any
 * stream capture.  All calls share the arrays and they keep the last call's contents
 * (the precision-policy counters are cleared by each call); calls that overlap
 * on the GPU race and must be serialised by the caller.  Failures are described
 * by map_smoother_last_error(NULL).
 */
map_status map_smoother_solve_noalloc(const map_problem_desc* desc, const void* y, void* x_out,
                                      void* stream);

/*
 * Batches of independent trajectories (thousands of trajectories of uneven
 * length and state dimension in one launch).
 * models[m] describes a linear model (desc.T is ignored, smoother MAP_RTS,
 * nx <= 6, every model in the same precision); trajectory j has
 * lengths[j] >= 1 intervals of model model_of[j].  Per model m:
 *   y[m]  device, y_rows x ny: trajectory j's lengths[j] observation rows in
 *         order, with one unused row between consecutive trajectories;
 *   x[m]  device, x_rows x nx: trajectory j's lengths[j] + 1 states in order.
 * map_batch_rows gives y_rows and x_rows (0 for models without trajectories).
 * Every trajectory starts from its model's prior (Eq. 31 a_T), so its filter
 * factor at local step k is the model's tabulated one (the per-step tables of
 * the Eq. 36 one-variable combine, Section 4.2 elements), and its solve is the
 * affine filter and RTS recursions (Section 4.3, Eq. 40-42) on those tables.
 * map_batch_solve: on the first call (eager launches, synchronising `stream`)
 * every model plans its step tables; when all of them reach the stationary
 * filter the batch runs as ONE launch of a persistent kernel over all models
 * and trajectories (CTAs take whole trajectories, longest first, from a work
 * counter), whose threads per CTA and steps per thread are chosen by timing
 * the candidates on these arrays (autotuning); the launch is captured into a
 * CUDA graph and every later call is one graph launch on `stream`
 * (asynchronous; new arrays update the kernel's model records on `stream`).
 * Otherwise every model takes the segmented scan (its trajectories as one scan
 * with the prior element inserted before every trajectory but the first,
 * which restarts the filter), with its own autotuned (steps per thread,
 * threads per tile), and the per-model launches form one graph with
 * concurrent branches.
 */
typedef struct map_batch map_batch;
map_status map_batch_create(map_batch** out, const map_problem_desc* models, int nmodels,
                            const int64_t* lengths, const int* model_of, int ntraj);
map_status map_batch_rows(const map_batch* b, int model, int64_t* y_rows, int64_t* x_rows);
map_status map_batch_solve(map_batch* b, const void* const* y, void* const* x, void* stream);
/* the (steps per thread, threads per CTA) of model m (0, 0 before the first solve): the
 * persistent kernel's (the same for every model), or the model's segmented scan's */
map_status map_batch_tuning(const map_batch* b, int model, int* K, int* B);
/* 1 when the batch runs as one launch of the persistent kernel, else 0 */
int map_batch_persistent(const map_batch* b);
const char* map_batch_last_error(const map_batch* b);
void map_batch_destroy(map_batch* b);

/* Free the handle and its workspace (NULL is ignored). */
void map_smoother_destroy(map_smoother* h);

/* Description of the last failure on this handle (or of the last failed create
 * when h is NULL).  The string lives until the next call on the handle. */
const char* map_smoother_last_error(const map_smoother* h);

/* 1 when kernels for (model, nx, ny, precision) are compiled in, else 0. */
int map_smoother_supported(int model, int nx, int ny, int precision);

/*
 * FMA throughput of the current device (no counterpart in the paper: the
 * measured denominator of the ALU rooflines of this library's kernels).
 * Launches 8 CTAs of 256 threads per SM, each thread running 8 independent
 * multiply-add chains for iters x 16 rounds, timed with CUDA events on
 * `stream` (synchronises it).  kind: 0 FP32 FFMA, 1 FP32 paired FMA (f32x2,
 * two per instruction), 2 FP64 DFMA.  *flop_out receives the flops executed
 * (2 per multiply-add), *ms_out the device time.  MAP_ERR_INVALID_ARG for a
 * NULL output, iters < 1 or an unknown kind; MAP_ERR_CUDA if a CUDA call fails.
 */
map_status map_fma_peak(int kind, int iters, double* flop_out, float* ms_out, void* stream);

/* Library version string. */
const char* map_smoother_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MAP_SMOOTHER_H */
