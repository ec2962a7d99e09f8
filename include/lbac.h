/*
 * lbac.h -- C ABI of the GB300 (sm_103a) linear lattice-Boltzmann acoustic
 * solver.  The method is the linear LB scheme of Dhuri, Hanasoge, Perlekar and
 * Robertsson, arXiv:1704.03172 ("the paper"): Chopard's linear equilibrium
 * (Eq. linear eqm dist), BGK (Eq. BGK-LB) or MRT (Eq. MRT-LB basic / Eq. MRT-LB)
 * collision on the D2Q5 or D2Q9 lattice (Table I, App. A), a point source added
 * as w_i S (Eq. MRT-LB linear acoustic), a spatially varying sound speed set
 * through the rest-particle weight (Eq. 0th lattice weight), and the two-level
 * grid refinement of Sec. 4 (Eq. grid refinement eqm dist, Eq. coarse-fine
 * dist connect).
 *
 * Conventions shared by every call:
 *  - Every call returns an lb_status; nothing throws or exits across the ABI.
 *  - Lattice units: one cell per step.  Arrays are row-major [y][x], x fastest.
 *    Population index i follows the rows of M in App. A: c_0 = (0,0),
 *    c_1 = (1,0), c_2 = (0,1), c_3 = (-1,0), c_4 = (0,-1), and for D2Q9
 *    c_5 = (1,1), c_6 = (-1,1), c_7 = (-1,-1), c_8 = (1,-1).
 *  - "Time t" is the number of steps taken.  Step t collides the state at time
 *    t, adds the source sample S[t] at the source site, applies the sponge and
 *    streams, producing the state at time t+1.
 *  - Input arrays are read (copied) during the call; the caller keeps
 *    ownership.  Output buffers are caller-owned.  A pointer flagged
 *    "on_device" must be a device pointer on the context's device.
 *  - Work is queued asynchronously on the context's CUDA stream; a device-side
 *    error surfaces as LB_ECUDA from the next call that synchronises
 *    (lb_sync, lb_record_receivers, lb_get_pressure, lb_get_state, ...).
 *  - A context is not thread-safe; distinct contexts are independent.
 *  - lb_last_error(ctx) returns a message for the last failing call on ctx
 *    (or, with ctx == NULL, the last lb_create failure of this thread).
 */
#ifndef LBAC_H
#define LBAC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_ctx lb_ctx;

typedef enum {
    LB_OK = 0,
    LB_EINVAL = -1,     /* invalid argument or configuration */
    LB_ENOMEM = -2,     /* device or host allocation failed */
    LB_ECUDA = -3,      /* a CUDA call or kernel failed */
    LB_EUNSTABLE = -4,  /* the state became non-finite */
    LB_ETIMEOUT = -5,   /* a bounded device wait gave up */
    LB_ESTATE = -6      /* call not valid in the context's current state */
} lb_status;

enum { LB_D2Q5 = 5, LB_D2Q9 = 9, LB_D3Q7 = 7 };   /* lattice (Table I; D3Q7: the 3-D
                                                      extension of D2Q5, w_0 = 1 - eta^2,
                                                      w_1..6 = eta^2 / 6, c_s^2 = eta^2 / 3) */
enum { LB_BGK = 0, LB_MRT = 1 };                   /* collision operator */
enum { LB_F32 = 0, LB_BF16 = 1, LB_F16 = 2,       /* population storage in HBM */
       LB_F64 = 3 };                               /* test only: FP64 populations, medium,
                                                      source and arithmetic (the same
                                                      per-site code as FP32), a plain
                                                      one-site-per-thread step; no patch,
                                                      time blocking, adjoint, invariants,
                                                      mode projection or serving */
enum { LB_ZERO_GHOST = 0, LB_PERIODIC = 1 };       /* outer boundary */

/* One refined patch (Sec. 4).  The fine grid covers the coarse rectangle of
 * nodes [x0, x0 + nx_c] x [y0, y0 + ny_c] with (2 nx_c + 1) x (2 ny_c + 1) fine
 * nodes; fine node (2a, 2b) coincides with coarse node (x0 + a, y0 + b).
 * ratio must be 2 (the paper's n).  Larger ratios ("multiples of 2", Sec. 4)
 * are nested patches: patches[k], k >= 1, lies inside the fine grid of
 * patches[k - 1], in that grid's node coordinates, and refines it by 2 again;
 * each patch keeps a margin of at least one node inside the grid above it. */
typedef struct {
    int x0, y0;
    int nx_c, ny_c;
    int ratio;
    int coupling;  /* LB_COUPLE_BOTH (0): both ways, population by population;
                      LB_COUPLE_C2F: coarse -> fine only, the grid above is never corrected
                      from this patch; LB_COUPLE_F2C: fine -> coarse only, nothing enters
                      the patch across its interface (zero, as at a zero-ghost boundary) --
                      the paper's switch on the direction of propagation (Sec. 4) */
} lb_patch;

enum { LB_COUPLE_BOTH = 0, LB_COUPLE_C2F = 1, LB_COUPLE_F2C = 2 };

typedef struct {
    int lattice;              /* LB_D2Q5 or LB_D2Q9 */
    int collision;            /* LB_BGK or LB_MRT */
    int storage;              /* LB_F32, LB_BF16, LB_F16 (FP16: per-population scale) or
                                 LB_F64 (test only) */
    int boundary;             /* LB_ZERO_GHOST or LB_PERIODIC */
    int nx, ny;               /* grid size in nodes (coarse grid when refined) */
    int sponge_width;         /* absorbing layer width W in cells, 0 = none */
    double sponge_sigma_max;  /* sigma(d) = sigma_max ((W - d)/W)^2, d = distance to edge */
    const float *c_map;       /* [ny][nx] sound speed (> 0), host unless c_map_on_device */
    int c_map_on_device;
    double c_ref;             /* eta = c / c_ref <= 1 (Eq. 0th lattice weight); <= 0: max(c_map) */
    double dx;                /* metres per cell, informational (lb_info) */
    double tau;               /* BGK relaxation time, tau >= 1/2 (Eq. BGK-LB) */
    double s[9];              /* MRT: diagonal of S in the moment order of App. A, 0 < s <= 2 */
    double w_ref[3];          /* D2Q9 weights (w0, w1, w5) at eta = 1; ignored for D2Q5 */
    const lb_patch *patches;  /* refinement patches, nested (see lb_patch), or NULL */
    int n_patches;            /* 0 .. LB_MAX_PATCHES */
    void *cuda_stream;        /* cudaStream_t to run on; NULL: the context creates its own
                                 non-blocking stream (pass cudaStreamLegacy for the legacy
                                 default stream, whose handle is NULL) */
    int time_block;           /* steps fused per launch (temporal blocking); <= 1: one.
                                 D2Q5: 2, 4, 6, 8 or 16 with FP32 or BF16 storage (the fused
                                 levels in between are FP32); D2Q9: 2 or 4 with FP32 storage */
    /* Optional device allocator (e.g. PyTorch's caching allocator).  NULL: cudaMalloc. */
    void *(*dev_alloc)(size_t bytes, void *user);
    void (*dev_free)(void *ptr, void *user);
    void *alloc_user;
    int step_kernel;          /* LB_STEP_AUTO (0): the TMA-staged persistent step for 16-bit
                                 storage on rows of >= 1024 sites without a patch, the
                                 register-streaming step otherwise; LB_STEP_DIRECT (1) / LB_STEP_STAGED
                                 (2, no patch): always that step.  All give bit-identical results. */
    int nz;                   /* planes of a 3-D grid (LB_D3Q7 only, BGK, no patch, no time
                                 blocking); <= 1: 2-D.  3-D arrays are [nz][ny][nx] (c_map,
                                 pressure) and [Q][nz][ny][nx] (state). */
    int streaming;            /* LB_STREAM_AB (0): each step pulls from one population buffer
                                 into the other (two buffers).  LB_STREAM_AA (1): in place, one
                                 buffer (half the population memory): steps alternate between
                                 a site-local update and a neighbour exchange in which every
                                 slot is read and written by one thread only.  D2Q5 / D2Q9,
                                 FP32 or BF16, no patch, time blocking, slab, checkpoint, tape
                                 or adjoint.  Results equal LB_STREAM_AB's bit for bit. */
} lb_config;

enum { LB_STEP_AUTO = 0, LB_STEP_DIRECT = 1, LB_STEP_STAGED = 2 };
enum { LB_STREAM_AB = 0, LB_STREAM_AA = 1 };
enum { LB_MAX_PATCHES = 3 };  /* nesting depth: ratio up to 8 to the coarse grid */

/* Fill *cfg with defaults: D2Q5, BGK tau = 1/2, F32, zero ghost, no sponge,
 * conventional D2Q9 weights (4/9, 1/9, 1/36), c_ref = max(c_map). */
lb_status lb_config_default(lb_config *cfg);

/* Validate cfg, allocate the device state and build the per-site medium
 * (eta^2 = (c / c_ref)^2, from which every weight and c_s^2 follow).
 * Errors: LB_EINVAL (bad sizes, tau < 1/2, s outside (0, 2], eta > 1,
 * c <= 0, negative weights, bad patch, a linearly unstable scheme -- see
 * lb_stability_radius), LB_ENOMEM, LB_ECUDA.  *out is NULL on failure. */
lb_status lb_create(const lb_config *cfg, lb_ctx **out);
lb_status lb_destroy(lb_ctx *ctx);

/* Point source at node (x, y) with samples S[n] for steps t = n (Eq. source
 * gives the paper's wavelet; any samples are accepted).  Steps t >= nt add
 * nothing.  The populations receive w_i(x, y) S[t] (Eq. MRT-LB linear
 * acoustic).  nt = 0 removes the source.  Host pointer, FP64 samples. */
lb_status lb_set_source(lb_ctx *ctx, int x, int y, const double *wavelet, int nt);

/* 3-D grids (nz > 1): the source at node (x, y, z) and receivers at xyz[r] =
 * (x, y, z), otherwise as lb_set_source / lb_set_receivers (which a 3-D context
 * refuses with LB_EINVAL).  Host pointers. */
lb_status lb_set_source_3d(lb_ctx *ctx, int x, int y, int z, const double *wavelet, int nt);
lb_status lb_set_receivers_3d(lb_ctx *ctx, const int *xyz, int nrec, int nt_capacity);

/* Receivers at nodes xy[r] = (x, y).  Row n of the trace is the pressure
 * p = c_s^2 rho (Eq. state) at time t0 + n, where t0 is the context time when
 * this call is made; at most nt_capacity rows are kept.  Host pointer. */
lb_status lb_set_receivers(lb_ctx *ctx, const int *xy, int nrec, int nt_capacity);

/* Set the state to equilibrium with pressure p0 and zero velocity:
 * g_i = (w_i / c_s^2) p0 (Eq. linear eqm dist with j = 0).  p0 == NULL sets
 * every population to 0.  Resets the time to 0.  p0: [ny][nx] FP32. */
lb_status lb_init_pressure(lb_ctx *ctx, const float *p0, int on_device);

/* Advance n >= 0 steps (asynchronous, unless lb_watch_stability is on). */
lb_status lb_step(lb_ctx *ctx, int n);

/* Linear (von Neumann) stability of a configuration's scheme, Sec. 3: the largest modulus
 * of the eigenvalues of the one-step map T(k) = D(k) (I - C A) of a homogeneous medium
 * (Eq. MRT-LB dispersion; A from Eq. linear eqm dist, C = I / tau or M^-1 S M, D(k) =
 * diag(exp(-i k.c_i))) over the nk x nk wave vectors k = 2 pi (m, n) / nk, at eta =
 * c / c_ref (0 < eta <= 1), with the rates of refinement level `level` (0: the coarse grid;
 * level l relaxes with tau_l - 1/2 = 2^l (tau - 1/2), reading R6).  Uses cfg's lattice
 * (D2Q5 / D2Q9), collision, tau, s and w_ref only.  Host computation, no CUDA call;
 * results are cached per configuration.  Sec. 2.3 ties the stability of D2Q9 to its
 * rates and weights.  lb_create runs the same computation with nk = 64 for D2Q9 and for
 * MRT at the medium's eta values (its distinct values when there are at most 8, else 8
 * values spread over its range) and every refinement level, and refuses the configuration
 * with LB_EINVAL when the radius exceeds 1 + 1e-12.  Errors: LB_EINVAL for an invalid
 * argument or an iteration that did not converge. */
lb_status lb_stability_radius(const lb_config *cfg, double eta, int level, int nk,
                              double *radius);

/* Detect instability while stepping: with every > 0, lb_step stops after each multiple of
 * `every` steps since this call, reads the FP64 invariants of the state (lb_invariants; the
 * stream is synchronised) and returns LB_EUNSTABLE when a value is non-finite or, for
 * max_growth > 0, when the energy sum_x sum_i g_i^2 / w_i grew by more than the factor
 * max_growth since the previous check (a source adds energy: choose the bound above what
 * it injects in `every` steps).  The steps before the failing check have been taken.
 * every = 0 turns the watch off.  LB_ESTATE for 3-D and LB_F64 contexts. */
lb_status lb_watch_stability(lb_ctx *ctx, int every, double max_growth);

/* Copy trace rows [0, min(recorded, nt_max)) to out ([rows][nrec], FP32) and
 * report the row count in *nt_out.  Synchronises the stream. */
lb_status lb_record_receivers(lb_ctx *ctx, float *out, int nt_max, int *nt_out, int on_device);

/* Pressure p = c_s^2 sum_i g_i at the current time, [ny][nx] FP32.
 * With refined patches, nodes inside a patch come from the finest level that
 * holds them (as do receiver traces). */
lb_status lb_get_pressure(lb_ctx *ctx, float *out, int on_device);

/* Populations g_i(x) at the current time (before its collision), as
 * [Q][ny][nx] FP32.  lb_set_state is the inverse and resets nothing else. */
lb_status lb_get_state(lb_ctx *ctx, float *out, int on_device);
lb_status lb_set_state(lb_ctx *ctx, const float *in, int on_device);

/* LB_F64 contexts only (LB_EINVAL otherwise): the same transforms in FP64 --
 * populations g_i(x) [Q][ny][nx] (get and set, as above) and the pressure
 * p = c_s^2 sum_i g_i [ny][nx] (Eq. state), so that results can be compared
 * with an FP64 reference at rounding level.  Caller-owned arrays, host or
 * device (on_device); synchronises the stream. */
lb_status lb_get_state_f64(lb_ctx *ctx, double *out, int on_device);
lb_status lb_set_state_f64(lb_ctx *ctx, const double *in, int on_device);
lb_status lb_get_pressure_f64(lb_ctx *ctx, double *out, int on_device);

/* Current time (steps taken since lb_init_pressure / lb_create). */
lb_status lb_get_time(const lb_ctx *ctx, long long *t);

/* Wait for all queued work; LB_ECUDA if any of it failed.  LB_ETIMEOUT if a
 * bounded device wait gave up since the last lb_sync (the TMA-staged step waits
 * at most one second for each of its bulk copies); the flag is then cleared,
 * so the status is reported once.  After LB_ETIMEOUT the state is undefined
 * until lb_init_pressure or lb_set_state; the context stays usable. */
lb_status lb_sync(lb_ctx *ctx);

/* Self-test of the bounded-wait failure path, for tests: queues one block
 * that waits on a shared-memory mbarrier phase that nothing completes, with
 * the staged step's polling, gives up after timeout_us microseconds
 * (1 .. 1000000) and raises the fault flag exactly as the step does.  The
 * state is not touched; the next lb_sync returns LB_ETIMEOUT. */
lb_status lb_wait_selftest(lb_ctx *ctx, int timeout_us);

/* Keep adjoint checkpoints: from now on (time t0 = current time), lb_step copies
 * the state into device memory before every step t with (t - t0) % every == 0.
 * every = 0 stops.  lb_init_pressure and lb_set_state restart the run of
 * checkpoints at their time.  Needs FP32 or BF16 storage and no patch
 * (LB_ESTATE); BF16 checkpoints are BF16 states (half the memory). */
lb_status lb_checkpoint_every(lb_ctx *ctx, int every);

/* Record the forward density tape for lb_adjoint: from now on (time t0 =
 * current time) every step t < t0 + nt_capacity also writes rho(x, t) =
 * sum_i g_i(x, t) of the state it pulls, FP32, nt_capacity x ny x pitch x 4
 * bytes of device memory (a 4096^2 run of 1000 steps: 67 GB).  lb_adjoint
 * then needs neither checkpoints nor replays when the tape covers its nt steps
 * and the receivers were set at t0.  nt_capacity = 0 frees the tape.
 * lb_init_pressure and lb_set_state restart it at their time.  Any storage
 * (FP16 included: the adjoint needs only rho), 2-D, no patch (LB_ESTATE);
 * LB_ENOMEM when the tape does not fit.  Synchronises. */
lb_status lb_record_rho(lb_ctx *ctx, int nt_capacity);

/* Discrete adjoint of the nt steps that followed the checkpointed start time
 * t0 (the paper has no adjoint; the scheme is linear in g, so the adjoint step is
 * the exact transpose: reverse streaming, K^T = (I - C (I - E))^T, receiver
 * injection).  dJdp[n][r] is dJ/dp at receiver r, trace row n (time t0 + n),
 * e.g. p - d for J = 1/2 sum (p - d)^2; the receivers must have been set at t0.
 * Outputs (any may be NULL): grad_c [ny][nx] = dJ/dc_map (c_ref held fixed),
 * grad_src [nt] = dJ/dS[t0 + n], grad_g0 [Q][ny][nx] = dJ/dg(t0).
 * on_device applies to dJdp and all outputs.  With a rho tape covering the nt
 * steps (lb_record_rho; t0 is then the tape's start) the sweep reads rho from
 * it; otherwise forward states are replayed from the checkpoints (two levels,
 * ~2 sqrt(every) + 3 extra states of device memory).  The context's own state
 * is left untouched.  Synchronises.
 * With BF16 storage the replayed forward states are the stored BF16 ones and the
 * adjoint runs in FP32: the gradient of the exact scheme along that trajectory,
 * which differs from the FP32 run's by about the forward's BF16 error. */
lb_status lb_adjoint(lb_ctx *ctx, const float *dJdp, int nt, float *grad_c, double *grad_src,
                     float *grad_g0, int on_device);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of independent shots (one simulation each).
 * The paper runs one simulation at a time; this layer serves many.  A
 * scheduler thread admits submitted requests in arrival order whenever a slot
 * and enough device memory (lb_footprint) are free, and advances every active
 * FP32/BF16 shot by one step per scheduling round with a single batched launch
 * per (lattice, collision, boundary, storage) group, so small shots share the
 * GPU and requests that arrive while others run join the batch at the next
 * round.  Under load, D2Q5 shots take 4 steps per batched launch instead
 * (lb_server_config.tb_min_ctas).  FP16 shots step on their own.  A request that asks for a gradient
 * records the forward rho tape or keeps checkpoints during its forward run
 * (lb_request.checkpoint_every) and its adjoint (lb_adjoint, J = 1/2
 * sum (p - d)^2 over its traces) runs on a worker thread on its own stream,
 * overlapping the batched forward work.  Results do not depend on what else
 * is in the batch: each shot runs the same kernels with the same arithmetic.
 */
typedef struct lb_server lb_server;

typedef struct {
    int max_active;          /* shots resident at once, >= 1 */
    size_t hbm_budget;       /* device bytes the server may hold; 0: 80% of free memory */
    int rounds_per_pass;     /* steps per scheduling pass between admission checks, >= 1 */
    int adjoint_workers;     /* threads running gradient sweeps, >= 1 */
    int tb_min_ctas;         /* D2Q5 FP32/BF16 shots with no checkpoint or tape can advance
                                4 steps per launch (a wavefront time-blocked batch).
                                0: they do, with the rows per CTA (at most 64) that fill
                                one wave of the GPU, when that is at least 12 rows and
                                their states outgrow three quarters of L2 (a few small
                                shots step one launch at a time).  > 0: they do, at
                                64 rows per CTA, when together they make at least this
                                many CTAs.  < 0: never.  Both forms give the same results
                                to FP32 rounding. */
} lb_server_config;

typedef struct {
    lb_config cfg;           /* shot configuration; c_map is a host array; cuda_stream,
                                allocator and time_block are ignored */
    int src_x, src_y;        /* source node */
    const double *wavelet;   /* S[n], n < nt_wavelet, host */
    int nt_wavelet;
    const int *rec_xy;       /* [nrec][2] receivers, host */
    int nrec;
    int nt;                  /* steps to run; traces have nt rows */
    const float *observed;   /* [nt][nrec] host data d (gradient requests only) */
    int want_gradient;       /* 1: also dJ/dc_map and dJ/dS for J = 1/2 sum (p - d)^2 */
    int checkpoint_every;    /* gradient requests: > 0 checkpoints every that many steps
                                (FP32 / BF16); < 0 the forward rho tape (lb_record_rho, any
                                storage); 0: the tape when it needs at most half of the
                                server's budget, else checkpoints every 200 steps */
} lb_request;

lb_status lb_server_create(const lb_server_config *cfg, lb_server **out);
/* Copies every input array; returns the request id.  LB_ENOMEM if the request
 * can never fit the budget, LB_EINVAL for an invalid configuration. */
lb_status lb_server_submit(lb_server *srv, const lb_request *req, long long *id);
/* *done = 1 once results are ready (or the request failed). */
lb_status lb_server_poll(lb_server *srv, long long id, int *done);
/* Block until done; LB_ETIMEOUT after timeout_ms (< 0: no limit). */
lb_status lb_server_wait(lb_server *srv, long long id, int timeout_ms);
/* Copy the results of a finished request and release it.  traces [nt][nrec];
 * grad_c [ny][nx] and grad_src [nt_wavelet] for gradient requests (any may be
 * NULL); times[3] = submit, start (admission), done, in seconds on the
 * server's monotonic clock.  Returns the request's own status (e.g. LB_ENOMEM). */
lb_status lb_server_result(lb_server *srv, long long id, float *traces, float *grad_c,
                           double *grad_src, double *times);
/* Counters: out[0] requests done, out[1] active, out[2] pending, out[3] device
 * bytes held, out[4] batched launches issued. */
lb_status lb_server_stats(lb_server *srv, double *out, int n);
/* Stop after finishing active and pending work; frees everything. */
lb_status lb_server_destroy(lb_server *srv);
const char *lb_server_last_error(const lb_server *srv);

/* FP64 invariants of the current state g(t), reduced on the device in a fixed
 * order (bit-reproducible): out[0] = mass sum_x rho(x), out[1] = energy
 * sum_x sum_i g_i^2 / w_i(x) over w_i > 0 (conserved by a tau = 1/2 step on a
 * homogeneous periodic grid, because g^eq is the W^-1-orthogonal projection of g
 * -- Eq. linear eqm dist -- and the collision reflects g about it),
 * out[2] = max |g_i|, out[3] = number of non-finite values.  out: host [4].
 * Returns LB_EUNSTABLE (with out filled) when out[3] > 0.  Uses a scratch
 * array of 4 ny + 4 doubles that the context allocates on first use.
 * Synchronises the stream. */
lb_status lb_invariants(lb_ctx *ctx, double *out);

/* lb_invariants without any allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory at the
 * point of the call -- code running under a fixed device-memory budget that
 * another framework owns, real-time loops where an allocation (and the
 * implicit synchronisation cudaMalloc/cudaFree may bring) is not allowed, or
 * code that has no lb_ctx at all.  It computes the same four FP64 values as
 * lb_invariants, with the same kernels and summation order, from caller
 * buffers:
 *   g       device, [Q][ny][nx] FP32 populations at one time (the layout
 *           lb_get_state writes), Q = lattice
 *   c_map   device, [ny][nx] FP32 sound speed; eta = c / c_ref
 *   w_ref   host, D2Q9 reference weights (w0, w1, w5); ignored for D2Q5
 *   out     device, 4 doubles: mass, energy, max |g|, non-finite count
 *   cuda_stream  cudaStream_t to queue on (NULL: the legacy default stream)
 * The work is queued asynchronously; nothing is copied to the host.  Zero-ghost
 * (non-periodic) state only.  If an earlier CUDA call left an error pending on the
 * calling thread, nothing is queued and LB_ECUDA is returned with a message saying
 * so; that error is left pending for its owner.
 * Scratch: a file-scope static device array of 16384 x 4 + 4 doubles
 * (512 KiB), held by every GPU that loads the library until the process exits.
 * ny > 16384 (or nx * ny > 2^31) is rejected with LB_EINVAL and a message in
 * lb_last_error(NULL).  No cudaMalloc, cudaFree or other allocating routine is
 * called.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it; make that
 * first call before any stream capture.  Every call on a device shares the
 * same array and each call overwrites every part of it that it reads, so
 * nothing needs clearing; calls that overlap on the GPU (other streams, or
 * other host threads) race on the array and must be serialised by the caller. */
lb_status lb_invariants_noalloc(const float *g, const float *c_map, int lattice, int nx,
                                int ny, double c_ref, const double *w_ref, double *out,
                                void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Row-slab domain decomposition of one shot (the method is local: a step reads only the
 * nearest neighbours, so a grid split into row slabs needs, per step and per cut, only
 * the populations that cross the cut -- D2Q5: g2 up and g4 down; D2Q9: g2, g5, g6 up and
 * g4, g7, g8 down).  Each slab is an ordinary context created for its own rows (its c_map
 * rows, source and receivers in local coordinates) and then marked with lb_set_slab.
 * Its steps pull across a cut from halo rows that the caller keeps filled with the
 * neighbour's cut rows, and write their own cut rows into send buffers in the same
 * launch.  lb_slab_step does the steps and the copies for slabs held by one process (on
 * one or several devices: a copy goes into the receiving slab's own memory); across
 * processes the caller moves the send buffers into the neighbours' halo buffers itself
 * (e.g. NCCL send / recv) between steps.  The sponge is measured in the whole grid, so a
 * decomposed run performs exactly the per-site arithmetic of the whole grid. */

/* Mark ctx as the rows [y_offset, y_offset + ny) of a grid of ny_global rows.  The four
 * buffers are caller-owned device memory of lb_slab_halo_bytes bytes each, 16-byte
 * aligned, on the context's device: send_lo / send_hi receive, from every step, the
 * crossing populations of the slab's first / last output row (stored type, [slot][pitch]);
 * recv_lo / recv_hi must hold the same rows of the slab below / above before each step
 * (NULL: no neighbour on that side -- the zero ghost, or the periodic wrap within the
 * slab).  2-D, FP32 or BF16 storage, no patch, no time blocking (LB_ESTATE); a slab has
 * no adjoint, checkpoints, rho tape or invariants.  The first step after lb_set_state /
 * lb_init_pressure reads the state in place and needs no halo rows; lb_get_pressure and
 * lb_get_state read the halo rows at the cuts. */
lb_status lb_set_slab(lb_ctx *ctx, int y_offset, int ny_global, void *send_lo, void *send_hi,
                      const void *recv_lo, const void *recv_hi);
/* Size of one slab row buffer of ctx: crossing populations x row pitch x stored bytes. */
lb_status lb_slab_halo_bytes(const lb_ctx *ctx, size_t *bytes);
/* Advance n slabs that tile one grid (slabs[k] directly above slabs[k - 1]) by `steps`
 * steps: every slab steps on its own stream, then each slab's halo rows are filled from
 * its neighbours' send buffers (the last and the first slab are neighbours when the grid
 * is periodic), ordered with events so that no step reads a halo row before its copy and
 * no copy reads a send buffer that the next step overwrites.  Asynchronous. */
lb_status lb_slab_step(lb_ctx **slabs, int n, int steps);

/* Device bytes lb_create would allocate for cfg (refinement patches included),
 * plus the receiver trace for nt steps when nrec > 0, plus what lb_adjoint needs
 * for nt steps when want_adjoint > 0 (the checkpoint interval; 1 means the
 * default 200) or, for want_adjoint = -1, the rho tape of nt steps
 * (lb_record_rho) and what lb_adjoint needs beside it. */
lb_status lb_footprint(const lb_config *cfg, int nt, int nrec, int want_adjoint, size_t *bytes);

/* Fourier projections of the pressure for dispersion diagnostics (the
 * single-mode analysis of Sec. 3, Eq. MRT-LB dispersion; Fig. 3 / Fig. 4):
 * for m < n_modes, with integer wave numbers (mx, my) = modes[2m], modes[2m+1]
 * and k = 2 pi (mx / nx, my / ny),
 *   out[2m] + i out[2m+1] = sum_x p(x) exp(-i k . x),  p = c_s^2 rho (Eq. state),
 * of the state at the current time, summed in FP64 on the device in a fixed
 * order.  Host arrays.  LB_ESTATE for a refined context.  Synchronises. */
lb_status lb_mode_projection(lb_ctx *ctx, const int *modes, int n_modes, double *out);

/* Sizes and derived constants: info[0] = Q, info[1] = row pitch in elements,
 * info[2] = bytes per stored population value, info[3] = physical time step
 * dt = dx c_s(eta=1) / c_ref (seconds; 0 when dx or c_ref is 0), info[4] = number
 * of distinct speeds when the step reads a 1-byte medium index (host c_map with at
 * most 256 distinct values), 0 when it reads eta^2 per site, info[5] = 1 when a step
 * runs the TMA-staged persistent kernel, else 0.  Fills min(n_info, 6) entries. */
lb_status lb_info(const lb_ctx *ctx, double *info, int n_info);

const char *lb_last_error(const lb_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* LBAC_H */
