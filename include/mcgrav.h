/*
 * mcgrav.h -- C ABI of libmcgrav, a GB300 (sm_103a) Monte Carlo solver for
 * the Newtonian potential and vertical gravity by the Feynman-Kac formula.
 *
 * Method: Donzelli, Bihlo, Kischinhevsky, Farquharson, "Massively parallel
 * stochastic solution of the geophysical gravity problem" (arXiv:1709.07469).
 *   - Problem (Sec. 2.1, Eq. 1 and its gravity form Eq. 4): a Dirichlet-
 *     Poisson problem for the potential in a bounded domain.  This library
 *     solves  Delta Phi = 4 pi G rho  in a box Omega with Dirichlet data g,
 *     i.e. Phi = -u of the paper's sign convention (Eq. 4-5).
 *   - Stochastic representation (Eq. 3, Eq. 5) with a standard Brownian
 *     motion W (the paper's gamma = sqrt(2) W runs at twice the speed):
 *       Phi(x0) = E[ g(W_tau) ] - 1/2 E[ int_0^tau 4 pi G rho(W_t) dt ].
 *   - Walk (Sec. 2.3, steps 1-4): Euler-Maruyama increments of per-axis
 *     standard deviation sigma sqrt(dt), trapezoid rule for the source
 *     integral, exit when the walk is no longer strictly inside Omega.  The
 *     last segment is clipped at its first crossing of the boundary and g is
 *     read at the crossing point.
 *   - Estimator (Eq. 7): the mean over N paths; g_z = dPhi/dz (Eq. 6) by the
 *     centred difference of Sec. 4.2 with common random numbers: three walks
 *     x0, x0 + h e_z, x0 - h e_z driven by the same increments.
 *   - Random numbers: the paper names no generator.  Path p of station s
 *     draws Philox4x32-10 (Salmon et al. 2011) with key (lo32 seed, hi32
 *     seed) and counter (j, p, s, 0); step block b (steps 4b..4b+3) uses
 *     j = 3b, 3b+1, 3b+2, whose 12 words give six Box-Muller pairs (cosine
 *     first) = the 12 increments of the four steps.
 *
 * Conventions for every entry point:
 *   - Status codes only; nothing is thrown across the ABI.  On error,
 *     mcg_last_error() returns a thread-local message.
 *   - "device" pointers are CUDA global memory of the current device,
 *     "host" pointers are ordinary host memory.  The caller owns every
 *     buffer it passes; the library keeps no pointer after the call returns
 *     (except inside the objects it creates, which say so).
 *   - Calls taking a stream are asynchronous on that stream (0 = the legacy
 *     default stream) unless documented as blocking.
 *   - The result is a deterministic function of (seed, station index, path
 *     index); it does not depend on batching, launch shape or what else is
 *     in flight.
 */
#ifndef MCGRAV_H
#define MCGRAV_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MCG_API __attribute__((visibility("default")))
#else
#define MCG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MCG_OK = 0,
    MCG_ERR_ARG = 1,        /* invalid argument (message says which)          */
    MCG_ERR_OOM = 2,        /* device allocation failed                       */
    MCG_ERR_CUDA = 3,       /* a CUDA runtime call failed                     */
    MCG_ERR_STEP_CAP = 4,   /* a path exceeded max_steps (its value is NaN)   */
    MCG_ERR_TIMEOUT = 5,    /* a bounded wait gave up                         */
    MCG_ERR_NONFINITE = 6,  /* a per-path value was not finite                */
    MCG_ERR_CANCELLED = 7   /* cancelled through the cancel flag              */
} mcg_status;

typedef enum { MCG_DOMAIN_BOX = 0, MCG_DOMAIN_BALL = 1 } mcg_domain_kind;

/* Domain Omega (open): the box (lo, hi), or the ball |x - center| < radius
 * (the paper's own domain, Sec. 2.2 and Sec. 3: a large ball around the
 * body with zero Dirichlet data).  Stations, and for g_z the two shifted
 * copies x0 +- h e_z, must lie strictly inside.  Tabulated boundary data and
 * the Brownian-bridge test need the box. */
typedef struct {
    double lo[3], hi[3];
    int32_t kind;
    double center[3];
    double radius;
} mcg_domain;

typedef enum { MCG_RHO_NONE = 0, MCG_RHO_SPHERE = 1, MCG_RHO_PRISM = 2, MCG_RHO_VOXEL = 3 } mcg_rho_kind;

/* Density model rho (kg/m^3 or any consistent unit), piecewise constant
 * like the paper's cube model (Sec. 3).
 *   SPHERE: rho0 where |x - center| < radius (strict), else 0.
 *   PRISM : rho0 on the half-open box [lo, hi), else 0.
 *   VOXEL : grid[ix + nx (iy + ny iz)] (float32, x fastest; DEVICE pointer,
 *           or HOST for mcgrav_solve)
 *           on cells [origin + i spacing, origin + (i+1) spacing); 0 outside.
 * G is the gravitational constant of the unit system (1 for nondimensional
 * problems, 6.67430e-11 in SI). */
typedef struct {
    int32_t kind;
    double G;
    double rho0;
    double center[3];
    double radius;
    double lo[3], hi[3];
    const float* grid;
    int64_t nx, ny, nz;
    double origin[3], spacing[3];
    const float* zpack;      /* VOXEL, optional DEVICE array from mcg_voxel_pack
                                (NULL: not used).  The mixed walk then reads the
                                densities of its three common-random-number
                                copies (z, z + h, z - h) with one 16-byte load
                                per step instead of three 4-byte loads; used when
                                h <= spacing[2] / 2.  Same values, same results. */
} mcg_density;

typedef enum { MCG_G_ZERO = 0, MCG_G_SPHERE = 1, MCG_G_PRISM = 2, MCG_G_TABLE = 3, MCG_G_POLY = 4 } mcg_g_kind;

/* Dirichlet data g on the boundary.
 *   ZERO  : g = 0 (the paper's own choice, Sec. 2.2).
 *   SPHERE: the analytic potential of the density's sphere.
 *   PRISM : the analytic potential of the density's prism (Nagy's corner
 *           function, the closed form the paper compares against).
 *   TABLE : six node-centred float32 tables (DEVICE pointer; HOST accepted
 *           by mcgrav_solve) of nv x nu
 *           nodes each (u fastest) in face order -x,+x,-y,+y,-z,+z; face
 *           +-x is tabulated over (y, z), +-y over (x, z), +-z over (x, y),
 *           nodes spanning the face edge to edge; read bilinearly.
 *   POLY  : c0 + c1 x + c2 y + c3 z + c4 x^2 + c5 y^2 + c6 z^2 + c7 xy
 *           + c8 yz + c9 zx + c10 xyz (test problems with known solutions). */
typedef struct {
    int32_t kind;
    const float* faces;
    int32_t nu, nv;
    double poly[11];
    const float* quads;      /* TABLE, optional DEVICE array from mcg_table_pack
                                (NULL: not used): the four corner values of every
                                table cell side by side, read with one 16-byte
                                load per exit.  Same values, same results.      */
} mcg_boundary;

typedef enum { MCG_FP64 = 0, MCG_MIXED = 1 } mcg_precision;

/* Options.  Zero-initialise and set what you need; mcg_options_default()
 * fills the defaults listed here. */
typedef struct {
    double h;                /* g_z finite-difference step (default 1e-2)          */
    double sigma;            /* Brownian scale, step std = sigma sqrt(dt) (1)      */
    int32_t precision;       /* MCG_FP64 plain walk or MCG_MIXED (default MIXED)   */
    int32_t clip;            /* 1: clip last segment (default); 0: paper's full step */
    int32_t crn_gz;          /* 1: three common-random-number walks, g_z (default)  */
    int32_t block;           /* threads per block of the walk kernel (0 = auto)   */
    int64_t max_steps;       /* RNG-step cap per path (default 2^31)               */
    int64_t batch_paths;     /* paths per station per launch in mcgrav_solve (0 = auto) */
    void* stream;            /* cudaStream_t (NULL = default stream)               */
    volatile int32_t* cancel;/* optional DEVICE int32; nonzero stops new work (the
                                walk polls it with a system-scope load; write it
                                with an asynchronous copy on another stream)       */
    int32_t bridge;          /* 1: Brownian-bridge exit test on steps that stay
                                inside (the paper's Remark on exit times, after
                                Gobet): a step from X to Y also ends the walk with
                                probability 1 - prod_faces (1 - exp(-2 d_X d_Y /
                                (sigma^2 dt))), one uniform per RNG-step from
                                Philox counter (n/4, p, s, 2) word n%4 shared by
                                the copies; the walk then ends on the face with the
                                largest term, below Y, after a full step (default 0) */
    int32_t refill_min;      /* a warp refills its lanes once at least this many are
                                free (1..32, default 1; mcg_autotune picks it)    */
    int32_t graph;           /* mcgrav_solve with several batches: capture the batch
                                sequence in one CUDA graph and launch it; a server's
                                walk options: capture each batch of rounds (walk,
                                reductions, result copies) and launch it as one graph
                                (default 1) */
    int32_t migrate;         /* mixed walk: once the work list is used up, warps with
                                few walks left hand them to warps with free lanes
                                through a pool in work_dev (default 1).  Results do
                                not depend on it for piecewise-constant densities;
                                for a voxel grid the single-precision partial sums
                                are flushed at other steps (rounding only).       */
    int32_t fault_unpublished;/* failure-detection test hook, 0..255 (default 0):
                                the launch starts with this many migration-pool
                                slots reserved but never published, as if a warp
                                had died between its reservation and its store.
                                A warp that claims one waits a bounded time
                                (about 0.1-1 s) for it, gives up, and the walk
                                reports MCG_ERR_TIMEOUT; every real walk still
                                finishes.  Needs the mixed walk with migrate = 1. */
    int32_t spill_max;       /* mixed walk with migrate = 1: once the work list is used
                                up, a warp with at most this many live walks (1..32,
                                default 24; 0 = default) hands them to warps with free
                                lanes (mcg_autotune picks it)                     */
} mcg_options;

/* Per-station outputs (caller-owned, length S; any pointer may be NULL). */
typedef struct {
    double* u;               /* potential estimate Phi(x0)                        */
    double* gz;              /* dPhi/dz estimate (NaN when crn_gz = 0)             */
    double* se_u;            /* standard error of u                               */
    double* se_gz;           /* standard error of gz                              */
    int64_t* n_paths;        /* paths averaged                                    */
    int64_t* path_steps;     /* Euler-Maruyama steps summed over paths and copies */
} mcg_result;

/* Running per-station statistics (device memory, 64 bytes each): two-pass
 * batch statistics merged batch after batch with Chan's formula. */
typedef struct {
    double n;
    double mean_u, m2_u;
    double mean_d, m2_d;
    double steps;            /* path-steps, exact below 2^53                      */
    double pad[2];
} mcg_station_state;

MCG_API void mcg_options_default(mcg_options* o);
MCG_API const char* mcg_last_error(void);
MCG_API const char* mcg_version(void);

/* ---------------------------------------------------------------------- */
/* One-call solver (Sec. 2.3 algorithm + Eq. 7 over all stations).          */
/* ---------------------------------------------------------------------- */

/* mcgrav_solve: estimates Phi and dPhi/dz at S stations from `paths` walks
 * each (paths 0 .. paths-1 of each station's stream).
 *   stations : HOST, S x 3 row-major (x, y, z).
 *   density, boundary : grid / faces in DEVICE or HOST memory (host arrays
 *            are copied into the call's workspace; the device-level entry
 *            points below take device pointers only).
 *   out      : HOST arrays of length S.
 * Blocking.  Allocates a device workspace for the duration of the call:
 * mcg_workspace_bytes(S, batch), plus the packed copies of a voxel grid and
 * of boundary tables (mcg_voxel_pack_bytes, mcg_table_pack_bytes) unless the
 * caller passes them, plus the grid and tables themselves when they are in
 * host memory.  With several batches, consecutive
 * batches alternate between two streams (the caller's and one of the
 * call's own) so that one batch's exit-time tail runs beside the next
 * batch; the reductions stay in batch order, so the result does not depend
 * on it.  Returns MCG_ERR_STEP_CAP /
 * MCG_ERR_NONFINITE when some path hit the cap / was not finite (the
 * statistics then include NaN). */
MCG_API int mcgrav_solve(const mcg_domain* domain, const mcg_density* density, const mcg_boundary* boundary,
                 const double* stations, int64_t S, int64_t paths, double dt, uint64_t seed,
                 const mcg_options* opts, mcg_result* out);

/* ---------------------------------------------------------------------- */
/* Device-resident building blocks (asynchronous on opts->stream).          */
/* ---------------------------------------------------------------------- */

/* mcg_walk: simulates paths p0 .. p0+N-1 of each of the S stations
 * (Sec. 2.3 steps 1-4) and writes per-path values, item i = s N + (p - p0):
 *   pp_u[i]     = g(x*) - 2 pi G I of the unshifted walk      (double)
 *   pp_d[i]     = (u(+h) - u(-h)) / (2h), or NaN without crn_gz (double)
 *   pp_steps[i] = Euler-Maruyama steps summed over the copies (int64)
 *   stations_dev: DEVICE, S x 3.   pp_*: DEVICE, length S*N.
 *   work_dev    : DEVICE scratch of mcg_walk_work_bytes(S, N, precision)
 *                 bytes (the mixed walk stores each copy's exit record
 *                 there and a second kernel evaluates the exits; it also
 *                 holds the migration pool and its counters, reset by this
 *                 call); may be NULL when that size is 0.  Caller-owned,
 *                 256-byte aligned.
 *   status_dev  : DEVICE int32, OR-ed with (1 << status) for every path that
 *                 hit the step cap, started outside Omega or produced a
 *                 non-finite value, and for a cancel or a bounded wait that
 *                 gave up (MCG_ERR_TIMEOUT); the caller zeroes it.
 *   counter_dev : DEVICE uint64 work counter, zeroed by this call.
 * Items that do not finish (cancelled, never started, capped, lost after a
 * timeout, station outside Omega) read pp_u = pp_d = NaN; pp_steps is 0 for
 * items never started.  The call marks every item "no result" before the
 * launch (a stream-ordered fill of the 8-byte step counts; the mixed walk
 * flags an item's count once all its copies have written their exit records,
 * and its exit kernel evaluates flagged items only), so nothing is read from
 * an earlier launch.
 * Allocates nothing. */
MCG_API int mcg_walk(const mcg_domain* domain, const mcg_density* density, const mcg_boundary* boundary,
             const double* stations_dev, int64_t S, int64_t p0, int64_t N, double dt, uint64_t seed,
             const mcg_options* opts, double* pp_u, double* pp_d, int64_t* pp_steps, void* work_dev,
             int32_t* status_dev, unsigned long long* counter_dev);

/* Bytes of scratch mcg_walk needs for S stations x N paths (0 for MCG_FP64). */
MCG_API size_t mcg_walk_work_bytes(int64_t S, int64_t N, int32_t precision);

/* mcg_walk_static: mcg_walk for callers that cannot allocate device memory.
 * No counterpart in the paper: this is a deployment variant of the walk.
 * Some callers only hand over the buffers they were given and may not call
 * cudaMalloc themselves: plug-in hosts that pass fixed input/output arrays,
 * services whose memory manager owns the whole device budget, and code on a
 * latency-critical path where an allocation would synchronise the device.
 * This entry point takes the same inputs and writes the same outputs as
 * mcg_walk (pp_u, pp_d, pp_steps, status_dev), but keeps its scratch -- the
 * work counter and the mixed walk's exit records -- in one fixed device
 * array inside the library (64 MiB, held by every GPU that loads the library
 * until the process exits).  It allocates nothing.
 *   - S * N may not exceed mcg_walk_static_max_items() (about 7.0e5 paths);
 *     larger requests return MCG_ERR_ARG with a message saying so.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls share the one array and it keeps the last call's contents;
 *     the call zeroes the counter and the caller's step counts (the
 *     completion flags) itself, so items that do not finish read NaN as
 *     with mcg_walk.  Calls
 *     that overlap on the GPU (other streams, other threads) race on it:
 *     serialise them.
 *   - The array's address is cached per device after the first call; a
 *     device reset (cudaDeviceReset) after that call is not supported.
 *   - opts->migrate is ignored: the array holds no migration pool, so each
 *     warp keeps its walks to the end (same results, longer exit-time tail).
 * Asynchronous on opts->stream like mcg_walk. */
MCG_API int mcg_walk_static(const mcg_domain* domain, const mcg_density* density, const mcg_boundary* boundary,
                            const double* stations_dev, int64_t S, int64_t p0, int64_t N, double dt, uint64_t seed,
                            const mcg_options* opts, double* pp_u, double* pp_d, int64_t* pp_steps,
                            int32_t* status_dev);

/* Largest S * N mcg_walk_static accepts. */
MCG_API int64_t mcg_walk_static_max_items(void);

/* mcg_reduce: folds one batch of per-path values (S x N, as written by
 * mcg_walk) into the running station states (Eq. 7 and the sample
 * variance): per station a fixed-order two-pass mean / sum of squares with
 * compensated partial sums, merged into states[s] with Chan's formula.
 * states_dev: DEVICE, S entries; zero them before the first batch.
 * Deterministic.  Allocates nothing. */
MCG_API int mcg_reduce(const double* pp_u, const double* pp_d, const int64_t* pp_steps, int64_t S, int64_t N,
               mcg_station_state* states_dev, void* stream);

/* mcg_finalize: states -> u, gz, se = sqrt(M2 / (n-1) / n), n, steps.
 * All output pointers DEVICE (may be NULL).  Allocates nothing. */
MCG_API int mcg_finalize(const mcg_station_state* states_dev, int64_t S, double* u, double* gz, double* se_u,
                 double* se_gz, int64_t* n_paths, int64_t* path_steps, void* stream);

/* mcg_states_merge: the multi-GPU exchange step.  A solve whose paths are
 * sharded over R ranks (each rank reducing its own path ranges with
 * mcg_reduce) combines the ranks' station states here: out[s] = Chan merge
 * of parts[0][s], parts[1][s], ..., parts[R-1][s] in that order (the same
 * parallel-variance combination mcg_reduce applies batch after batch), so
 * the result is deterministic for a fixed rank order and partition.
 * The paper gathers per-GPU partial means on one node (Sec. 4).
 *   parts: HOST, R x S states (rank-major).  out: HOST, S states (may alias
 *   parts[0 .. S-1]).  States with n = 0 are skipped.  Allocates nothing. */
MCG_API int mcg_states_merge(const mcg_station_state* parts, int64_t R, int64_t S, mcg_station_state* out);

/* mcg_autotune: picks the launch shape of the walk for this problem and
 * writes it into *opts, in two stages timed with CUDA events (one warm-up
 * launch, then the median of three timed launches per candidate):
 *   1. opts->block (64, 96, 128) on short walks of the given stations capped
 *      at 2048 RNG-steps (the stepping rate, every lane busy; all walks of a
 *      warp end together, so the refill policy plays no part);
 *   2. mixed walk: opts->refill_min (1, 4, 16) x opts->spill_max (8, 16, 24,
 *      32; with migrate = 1 only) on uncapped walks, two per resident lane,
 *      whose launch ends in the exit-time tail: lanes free up at random steps
 *      and walk migration shortens the tail.  The defaults (refill 1, the
 *      incoming spill threshold, 24 when unset) stay unless another pair is
 *      more than 1 % faster (skipped for the FP64 walk; stops early, keeping
 *      them, once one launch takes over 2 s).
 * stations_dev: DEVICE, S x 3.  Blocking; allocates and frees a scratch
 * area of mcg_walk's size for the larger of the two stages. */
MCG_API int mcg_autotune(const mcg_domain* domain, const mcg_density* density, const mcg_boundary* boundary,
                         const double* stations_dev, int64_t S, double dt, uint64_t seed, mcg_options* opts);

/* mcg_smooth_moving_average: the moving average the paper applies to the
 * potential along a line of stations before differencing (Sec. 4.1, MATLAB
 * smooth): out[i] = mean of y[i-k .. i+k] with k = min((span-1)/2, i,
 * n-1-i), i.e. the window shrinks symmetrically at the ends (out[0] = y[0],
 * out[n-1] = y[n-1]).  An even span is reduced by one.  HOST arrays; out may
 * not alias y.  Allocates nothing. */
MCG_API int mcg_smooth_moving_average(const double* y, int64_t n, int32_t span, double* out);

/* Bytes of device workspace mcgrav_solve uses at most for S stations and
 * batches of `batch` paths per station (two sets of per-batch buffers; a
 * solve of one batch uses one). */
MCG_API size_t mcg_workspace_bytes(int64_t S, int64_t batch);

/* ---------------------------------------------------------------------- */
/* Random numbers (the generator the walks use), for verification.          */
/* ---------------------------------------------------------------------- */

/* mcg_philox: out[4i..4i+3] = Philox4x32-10(ctr[4i..4i+3], key[2i..2i+1]).
 * All DEVICE pointers, n entries.  Allocates nothing. */
MCG_API int mcg_philox(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out, void* stream);

/* mcg_normals: the 12 normals of step blocks b0 .. b0+nblocks-1 of path
 * (s, p), in the precision of the walk: precision MCG_FP64 writes doubles
 * from u = (w + 1/2) 2^-32; MCG_MIXED writes floats from u = ((w >> 9) +
 * 1/2) 2^-23 with the single-precision transcendental path of the mixed
 * walk.  out: DEVICE, 12 * nblocks elements.  Allocates nothing. */
MCG_API int mcg_normals(uint64_t seed, uint32_t s, uint32_t p, uint32_t b0, int64_t nblocks, int32_t precision,
                void* out, void* stream);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching of solve requests.                          */
/* ---------------------------------------------------------------------- */
/* An inversion code calls the forward solver many times with different
 * station sets, models and accuracy targets (the paper's motivation, Sec. 1).
 * The server keeps models resident on the device, admits requests while
 * their buffers fit an HBM budget, and advances every admitted request in
 * rounds of whole chunks of `chunk_paths` paths per station (path indices
 * continue from round to round: the request's paths are 0, 1, 2, ... of
 * each station), each merged into the request's station statistics; after
 * each round the request stops once every station reaches its relative
 * standard error target (and has at least min_paths paths) or max_paths.
 * The first round walks min_paths (rounded up to chunks); later rounds walk
 * as many chunks (up to max_round_paths) as the request's own per-path
 * spread says it still needs, in one launch.  Rounds of different requests run on
 * a pool of streams and overlap on the GPU; a request's result depends only
 * on its own (seed, stations, target), never on what else is in flight.
 * All calls are thread-safe.  Objects are owned by the library until the
 * matching destroy / free call. */
typedef struct mcg_model mcg_model;
typedef struct mcg_server mcg_server;
typedef struct mcg_request mcg_request;

typedef struct {
    int32_t streams;          /* stream slots, one launch in flight on each (default 8) */
    int32_t max_active;       /* requests in flight at most (default 64)             */
    int64_t hbm_budget;       /* bytes of request buffers in flight (default 8 GiB)  */
    int64_t chunk_paths;      /* paths per station per round (default 4096)          */
    int64_t min_paths;        /* paths per station before the target is checked (default 2 chunks) */
    int64_t max_paths;        /* cap per station (default 10^7)                      */
    int64_t max_round_paths;  /* paths per station in one round at most (default 16 chunks):
                                 after min_paths the next round walks the chunks the
                                 request's own spread says it still needs, in one launch */
    mcg_options walk;         /* walk options (precision, h, sigma, clip, crn_gz, block, max_steps) */
    int32_t batch;            /* 1 (default): ready rounds of requests whose problems share
                                 every scalar (domain, density and boundary kinds, grid
                                 geometry, dt, h) share one walk launch, each request a
                                 segment with its own stations, seed and model arrays;
                                 0: one walk launch per round.  Box domain without the
                                 bridge test; other requests always run alone.    */
    int64_t batch_items;      /* walks in one shared launch at most (default 2^22); the
                                 ready rounds are spread over the free stream slots  */
} mcg_server_config;

MCG_API void mcg_server_config_default(mcg_server_config* c);

/* mcg_model_create: a device-resident copy of the problem (domain, density,
 * boundary data, time step dt and g_z difference step h; the server's walk
 * options supply the rest).  Grid and faces may be host or device pointers;
 * they are copied, so the caller may free its buffers afterwards.
 * Blocking. */
MCG_API int mcg_model_create(const mcg_domain* domain, const mcg_density* density, const mcg_boundary* boundary,
                             double dt, double h, mcg_model** out);
MCG_API int mcg_model_destroy(mcg_model* m);

/* mcg_server_create: starts the scheduler thread on the current device. */
MCG_API int mcg_server_create(const mcg_server_config* cfg, mcg_server** out);
/* mcg_server_destroy: cancels nothing; waits for every admitted and queued
 * request to finish, then stops the thread.  Requests stay valid until
 * freed. */
MCG_API int mcg_server_destroy(mcg_server* s);

/* mcg_submit: queues a request (non-blocking).  stations: HOST, S x 3
 * (copied).  target_rel_se: stop when se_u <= target |u| at every station.
 * The model must outlive the request. */
MCG_API int mcg_submit(mcg_server* s, const mcg_model* m, const double* stations, int64_t S, double target_rel_se,
                       uint64_t seed, mcg_request** out);
/* mcg_poll: *done = 1 and the HOST result arrays (length S) filled once the
 * request finished; returns the request's status then (MCG_OK, or the error
 * that ended it).  Non-blocking. */
MCG_API int mcg_poll(mcg_request* r, mcg_result* out, int* done);
/* mcg_wait: blocks until the request finished (at most timeout_ms, < 0 =
 * forever; MCG_ERR_TIMEOUT when the wait gives up), then as mcg_poll. */
MCG_API int mcg_wait(mcg_request* r, mcg_result* out, int64_t timeout_ms);
/* mcg_cancel: stops scheduling rounds of the request; it finishes with
 * MCG_ERR_CANCELLED and partial statistics. */
MCG_API int mcg_cancel(mcg_request* r);
/* mcg_request_info: paths per station done, rounds, latency in seconds from
 * submit to completion (or so far).  Any pointer may be NULL. */
MCG_API int mcg_request_info(const mcg_request* r, int64_t* paths, int64_t* rounds, double* seconds);
MCG_API int mcg_request_free(mcg_request* r);
/* mcg_server_stats: walk launches so far and the request rounds they ran
 * (rounds / launches = requests per shared launch).  Either pointer may be
 * NULL. */
MCG_API int mcg_server_stats(const mcg_server* s, int64_t* launches, int64_t* rounds);

/* ---------------------------------------------------------------------- */
/* Heterogeneous model set-up (once per model, outside the walk).            */
/* ---------------------------------------------------------------------- */

/* ---------------------------------------------------------------------- */
/* Packed copies of the model arrays for the walk's 16-byte loads.          */
/* ---------------------------------------------------------------------- */
/* The walk reads the voxel grid once per step and copy, and a boundary table
 * once per exit, at scattered positions: every read costs a cache sector of
 * its own.  The packed copies put what one step (or one exit) needs side by
 * side, so one aligned 16-byte load replaces three (or four) 4-byte loads.
 * Build them once per model (like the model itself) and pass them in
 * mcg_density.zpack / mcg_boundary.quads.  mcgrav_solve and mcg_model_create
 * build them on their own. */

/* Bytes of mcg_voxel_pack's output: 16 nx ny (nz + 2). */
MCG_API size_t mcg_voxel_pack_bytes(int64_t nx, int64_t ny, int64_t nz);

/* mcg_voxel_pack: out[((iz + 1) ny + iy) nx + ix] = (rho(ix, iy, iz - 1),
 * rho(ix, iy, iz), rho(ix, iy, iz + 1), 0) as four floats, for iz = -1 .. nz,
 * with rho = 0 outside the grid.  density: VOXEL with a DEVICE grid.
 * out: DEVICE, mcg_voxel_pack_bytes, 16-byte aligned.  Asynchronous on
 * `stream`.  Allocates nothing. */
MCG_API int mcg_voxel_pack(const mcg_density* density, float* out, void* stream);

/* Bytes of mcg_table_pack's output: 16 * 6 (nu - 1) (nv - 1). */
MCG_API size_t mcg_table_pack_bytes(int32_t nu, int32_t nv);

/* mcg_table_pack: out[(f (nv - 1) + iv) (nu - 1) + iu] = (t(iu, iv),
 * t(iu + 1, iv), t(iu, iv + 1), t(iu + 1, iv + 1)) of face f's table t (the
 * MCG_G_TABLE layout).  boundary: TABLE with DEVICE faces.  out: DEVICE,
 * mcg_table_pack_bytes, 16-byte aligned.  Asynchronous on `stream`.
 * Allocates nothing. */
MCG_API int mcg_table_pack(const mcg_boundary* boundary, float* out, void* stream);

/* Bytes of device scratch mcg_grf_density needs for an nx x ny x nz grid. */
MCG_API size_t mcg_grf_work_bytes(int64_t nx, int64_t ny, int64_t nz);

/* mcg_grf_density: a Gaussian-random-field density model on an nx x ny x nz
 * voxel grid (x fastest), the heterogeneous subsurface of the survey
 * workloads (the paper's models are a single homogeneous cube, Sec. 3):
 *   1. white noise N(0,1): voxels 4q..4q+3 take the two Box-Muller pairs of
 *      Philox4x32-10 counter (q, 0, 0, 1) under key (lo32 seed, hi32 seed);
 *   2. separable Gaussian smoothing of std sigma_vox voxels, taps |m| <=
 *      ceil(3 sigma_vox) (at most 63), weights summing to 1, zero outside;
 *   3. rescaled to zero mean and unit population standard deviation;
 *   4. rho = amp (exp(Z) - 1), stored as float32.
 * grid_out: DEVICE float32, nx*ny*nz.  work: DEVICE, mcg_grf_work_bytes.
 * Asynchronous on `stream`.  Allocates nothing. */
MCG_API int mcg_grf_density(uint64_t seed, int64_t nx, int64_t ny, int64_t nz, double sigma_vox, double amp,
                            float* grid_out, void* work, void* stream);

/* mcg_boundary_tables: Dirichlet data for MCG_G_TABLE -- the potential
 * Phi = -G sum_voxels rho_v [[[F]]]_v of the voxel model (prism summation,
 * the closed form the paper compares against, Sec. 1 and Sec. 4.2) at the
 * nu x nv nodes of each face of `domain` (layout as MCG_G_TABLE).  Voxels
 * whose centre lies within `near_cells` cell diagonals of a node use the
 * exact prism potential in double precision; farther voxels, which must be
 * cubes or close to them, use their point-mass term rho_v V / r in single
 * precision, whose relative error for a cube is O((d/r)^4).  Supports
 * nx <= 128.  faces_out: DEVICE float32, 6 nv nu.  density->grid: DEVICE.
 * Asynchronous on `stream`.  Allocates nothing. */
MCG_API int mcg_boundary_tables(const mcg_domain* domain, const mcg_density* density, int32_t nu, int32_t nv,
                                double near_cells, float* faces_out, void* stream);

/* ---------------------------------------------------------------------- */
/* Exact field of the density models (the reference the walk is checked     */
/* against).                                                                */
/* ---------------------------------------------------------------------- */

/* mcg_field: the exact potential Phi (Delta Phi = 4 pi G rho, Phi -> 0 far
 * away) and its vertical derivative dPhi/dz of the density model at n
 * points, the closed forms the paper compares its stochastic solution with
 * (Sec. 4.2: the analytic field of the prism):
 *   SPHERE: -G M / r outside, -G M (3 a^2 - r^2) / (2 a^3) inside.
 *   PRISM : Nagy's corner function F over the eight corners,
 *           Phi = -G rho0 [[[F]]], dPhi/dz = G rho0 [[[dF/dz]]].
 *   VOXEL : the sum of every voxel's prism field, regrouped by grid node:
 *           Phi(x) = -G sum_nodes w_n F(node - x), where w_n adds the
 *           densities of the (up to eight) cells sharing the node with the
 *           sign of that corner in each cell's prism sum.  Double precision
 *           with compensated sums; one block per point, (nx+1)(ny+1)(nz+1)
 *           corner evaluations per point (about 0.5 ms per point on a GB300
 *           for a 128 x 128 x 64 grid).
 *   NONE  : 0.
 * points_dev: DEVICE, n x 3 row-major.  phi_dev, gz_dev: DEVICE, length n
 * (either may be NULL).  density->grid: DEVICE.  Asynchronous on `stream`.
 * Allocates nothing. */
MCG_API int mcg_field(const mcg_density* density, const double* points_dev, int64_t n, double* phi_dev,
                      double* gz_dev, void* stream);

/* mcg_density_at: the density the walks read (Sec. 2.3 step 3: rho at the
 * walk's points), sampled at n points and at their common-random-number
 * copies: out[3 i + 0, 1, 2] = rho at (x, y, z), (x, y, z + h), (x, y, z - h).
 *   precision MCG_MIXED: the mixed walk's single-precision sampler, the point
 *     taken relative to the domain centre in single precision as the walk
 *     starts it (the packed grid when density->zpack is set and h <= half a
 *     cell, else the plain grid: the same values);
 *   precision MCG_FP64: the plain walk's double-precision sampler, the copies
 *     at z + h and z - h rounded in double precision.
 * Cells are half-open [lo, hi); outside the grid, the prism or the sphere the
 * density is 0, also for points far outside the domain.  points_dev: DEVICE,
 * n x 3 (absolute coordinates).  out_dev: DEVICE, 3 n doubles (single-
 * precision values widened exactly).  Asynchronous on `stream`; allocates
 * nothing.  MCG_ERR_ARG for a bad domain or density, h < 0, or a null buffer
 * with n > 0. */
MCG_API int mcg_density_at(const mcg_domain* domain, const mcg_density* density, double h, int32_t precision,
                           const double* points_dev, int64_t n, double* out_dev, void* stream);

/* ---------------------------------------------------------------------- */
/* Measured peaks (the denominators of the walk's roofline).                */
/* ---------------------------------------------------------------------- */

/* mcg_issue_probe: the lane-instruction rate the current GPU sustains on long
 * runs of independent single-precision FMAs (kind 0), of FMAs and three-input
 * xors side by side (kind 1, the two pipes the mixed walk's generator and
 * transform use) or of double-precision FMAs (kind 2, the pipe the plain
 * FP64 walk is bound by), one persistent launch over every SM, timed with
 * CUDA events after a warm-up launch.  Any other kind: MCG_ERR_ARG before any
 * CUDA call.  No counterpart in the paper: it measures
 * the hardware the walk runs on.  lane_ops_per_s, seconds: HOST (either may
 * be NULL).  Blocking; allocates and frees 4 bytes of device memory. */
MCG_API int mcg_issue_probe(int32_t kind, int32_t iters, double* lane_ops_per_s, double* seconds);

#ifdef __cplusplus
}
#endif
#endif /* MCGRAV_H */
