/*
 * lbm.h -- C ABI of a GB300 (sm_103a) D3Q27 lattice Boltzmann solver with the
 * central-Hermite-moment multiple-relaxation-time collision of
 * "Simulation of the FDA Nozzle Benchmark: A Lattice Boltzmann Study"
 * (arXiv 2204.10566).
 *
 * One call of lbm_step advances every active cell of the lattice by one time
 * step of the pull-stream/collide update:
 *   f_i(x + c_i, t + 1) - f_i(x, t) = T^-1 S T (f^eq(rho, u) - f)(x, t)
 * (Sec. 2.1, MRT evolution eq.), T the central Hermite transform
 * (Sec. 2.1, central moment eq.; Appendix A), f^eq the full Hermite expansion
 * supported by D3Q27 (Sec. 2.1 equilibrium eq.; Appendix A), second-order
 * moments relaxed at omega = 1/(3 nu + 1/2) (Sec. 2.1 relaxation-time relation)
 * and higher orders at the ghost rates (1 by default, Appendix A), with
 * halfway bounce-back walls, a velocity inlet and a constant-pressure outlet
 * by non-equilibrium extrapolation (Sec. 2.2, "Simulation details").
 *
 * Conventions shared by every call
 *   - Lattice units: dr = dt = 1, theta0 = 1/3.
 *   - Direction i = 9 (cz+1) + 3 (cy+1) + (cx+1), c in {-1,0,1}^3; the
 *     opposite direction is 26 - i.
 *   - Box cell b = x + nx (y + ny z) ("x fastest").
 *   - Active cells are the cells whose flag is FLUID, INLET or OUTLET.  The
 *     "active order" lists them by increasing b.  Host arrays use either that
 *     order (LBM_LAYOUT_ACTIVE, n = number of active cells) or the full box
 *     (LBM_LAYOUT_BOX, n = nx ny nz, solid cells written as 0 and ignored on input).
 *   - Population arrays are [n][27] doubles holding f_i (not deviations).
 *   - Velocity arrays are [n][3] doubles.
 *   - Every pointer argument is a HOST pointer unless the comment says
 *     otherwise; the library copies what it needs and the caller keeps ownership.
 *   - Every call returns an lbm_status.  No call throws or aborts.  After an
 *     error, lbm_last_error(ctx) describes it; the string is owned by ctx and
 *     valid until the next call on ctx.
 *   - Device work is enqueued on the context's stream.  Calls that return
 *     host data synchronise that stream; lbm_step does not.  lbm_step also
 *     uses a second stream that the context owns: each step forks onto it
 *     with an event recorded on the context's stream and joins back with
 *     another before the step ends, so the step stays ordered on the
 *     context's stream and can be captured into a CUDA graph there.
 *   - A context is not thread-safe: one host thread at a time.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,      /* invalid argument, inconsistent geometry or parameters */
    LBM_ERR_OOM = 2,      /* device allocation failed / does not fit */
    LBM_ERR_CUDA = 3,     /* a CUDA runtime call failed */
    LBM_ERR_STATE = 4,    /* call out of order (e.g. lbm_step before lbm_set_geometry) */
    LBM_ERR_UNSTABLE = 5, /* a health check found non-finite populations */
    LBM_ERR_TIMEOUT = 6   /* a bounded device-side wait gave up */
} lbm_status;

typedef enum {
    LBM_FP64 = 0,  /* populations stored as FP64 deviations f_i - w_i, FP64 arithmetic */
    LBM_FP32 = 1,  /* FP32 deviations f_i - w_i, FP32 arithmetic */
    LBM_FP16S = 2  /* FP16 (f_i - w_i) * s, FP32 arithmetic */
} lbm_precision;

enum { LBM_SOLID = 0, LBM_FLUID = 1, LBM_INLET = 2, LBM_OUTLET = 3 };
enum { LBM_PROFILE_PLUG = 0, LBM_PROFILE_PARABOLIC = 1 };
enum { LBM_LAYOUT_ACTIVE = 0, LBM_LAYOUT_BOX = 1 };
enum { LBM_PERIODIC_X = 1, LBM_PERIODIC_Y = 2, LBM_PERIODIC_Z = 4 };
/* Axis along which the populations are stored in contiguous rows (a storage
 * choice: results do not depend on it beyond floating-point contraction).
 * AUTO takes z when the box is longer in z than in x (the flow axis of a
 * nozzle), else x. */
enum { LBM_ROWS_AUTO = 0, LBM_ROWS_X = 1, LBM_ROWS_Z = 2 };

typedef struct lbm_ctx lbm_ctx;

/* Device memory provider.  alloc(bytes, user) returns a device pointer
 * (256-byte aligned) or NULL; free(ptr, user) releases it.  With alloc == NULL
 * the library uses cudaMalloc / cudaFree.  Called only from lbm_create,
 * lbm_set_geometry, lbm_stats_begin, the population/field transfer calls and
 * lbm_destroy, never from lbm_step. */
typedef struct {
    void *(*alloc)(size_t bytes, void *user);
    void (*free)(void *ptr, void *user);
    void *user;
} lbm_allocator;

/* Lattice and device description (lbm_create). */
typedef struct {
    int32_t nx, ny, nz;   /* box size in cells, each >= 1 */
    int32_t periodic;     /* LBM_PERIODIC_* bits; other faces are solid walls */
    int32_t precision;    /* lbm_precision */
    float fp16_scale;     /* FP16S scale s: a power of two > 0 (0 selects 4096 = 2^12, which keeps
                             deviations of 1e-4..10 in the normal FP16 range) */
    int32_t device;       /* CUDA device ordinal */
    int32_t row_axis;     /* LBM_ROWS_AUTO (0), LBM_ROWS_X or LBM_ROWS_Z */
    void *stream;         /* cudaStream_t for all work of this context (NULL: default stream) */
    lbm_allocator allocator;
} lbm_desc;

/* Flow parameters (lbm_set_params).  Fill with lbm_params_default first. */
typedef struct {
    double nu;            /* kinematic viscosity (lattice units); if <= 0 it is
                             derived as nu = u_char L_char / Re (Sec. 2.2 Re definition) */
    double Re;            /* Reynolds number */
    double u_char;        /* characteristic velocity (throat mean velocity) */
    double L_char;        /* characteristic length (throat diameter, cells) */
    double omega3, omega4, omega5, omega6;  /* ghost rates of orders 3..6 (default 1,
                             Appendix A); 0 < rate < 2 */
    double u_in;          /* mean inlet velocity u0 (lattice units), |u_in| < 1/sqrt(3) */
    double d_in;          /* inlet diameter d0 in cells (parabolic profile); <= 0: nx */
    double axis_x, axis_y;/* nozzle axis position in cell-face coordinates;
                             negative: box centre nx/2, ny/2 */
    double noise_amp;     /* relative inlet perturbation: u_b += noise_amp u0 U(-1,1) per component */
    double rho_out;       /* outlet density (default 1) */
    uint64_t noise_seed;  /* perturbation seed */
    int32_t inlet_profile;/* LBM_PROFILE_PLUG or LBM_PROFILE_PARABOLIC */
    int32_t inlet_ramp;   /* steps T of a smooth inlet start, u_b(t) = u_b r(t/T) with
                             r(s) = s^2 (3 - 2 s) for t < T (0: impulsive start) */
} lbm_params;

/* Human-readable name of a status code (static string). */
const char *lbm_status_string(lbm_status s);

/* Defaults: nu = 0, Re = 0 (must be set), ghost rates 1, plug inlet u_in = 0,
 * d_in = 0 (box width), axis at the box centre, no noise, rho_out = 1. */
void lbm_params_default(lbm_params *p);

/* Create a context on desc->device bound to desc->stream.  Allocates nothing
 * on the device until lbm_set_geometry, apart from the second stream (highest
 * priority) and its two events; if those cannot be created, or with
 * LBM_SIDE_STREAM=0 in the environment at creation, every kernel of a step
 * runs on desc->stream in sequence.  *out receives the context.
 * Lattices of 2^32 / 27 slots or more step with 64-bit element offsets; with
 * the environment variable LBM_WIDE_OFFSETS=1 at creation, every lattice
 * does (for testing that path on small lattices).  LBM_FLUID_KERNEL at
 * creation selects another fluid kernel than the default for tests and
 * measurements: "chunk", "tile" or "pairs" (same results within rounding).
 * Errors: LBM_ERR_ARG (bad sizes, precision, scale), LBM_ERR_CUDA. */
lbm_status lbm_create(const lbm_desc *desc, lbm_ctx **out);

/* Free every device buffer of ctx (through its allocator) and ctx itself.
 * Synchronises the stream first.  NULL is accepted. */
lbm_status lbm_destroy(lbm_ctx *ctx);

/* Description of the last error on ctx ("" if none). */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Voxelise the axisymmetric FDA-type nozzle of Sec. 2.2 along z into a host
 * flag array out[L_total][D][D] (x fastest): inlet pipe of diameter D and
 * length L_in, a cone of half-angle half_angle_deg down to diameter d
 * (L_cone < 0: its length is round((D - d) / 2 / tan(angle))), a throat of
 * length L_throat, then diameter D to L_total.  Voxel (x,y,z) is inside iff
 * (x+1/2-D/2)^2 + (y+1/2-D/2)^2 <= r(z+1/2)^2, the cone radius following the
 * half-angle and never below d/2.  Inside voxels of plane z = 0 are INLET, of
 * plane z = L_total-1 OUTLET, other inside voxels FLUID, the rest SOLID.
 * Errors: LBM_ERR_ARG. */
lbm_status lbm_make_nozzle(int32_t D, int32_t d, int32_t L_in, int32_t L_cone, int32_t L_throat,
                           int32_t L_total, double half_angle_deg, uint8_t *out);

/* Host-only check of a flag field (no device needed): builds the sparse index
 * exactly as lbm_set_geometry would with rows along row_axis (LBM_ROWS_*) and
 * re-verifies, independently, the invariants the kernels rely on (every
 * chunk lane a unique fluid cell, every position the step touches owning its
 * slot, every pull slot inside the buffer and stored).  out (may be NULL)
 * receives: active cells, storage slots, row records, fluid chunks,
 * inlet/outlet nodes, wall links, rows, row axis used (LBM_ROWS_X or _Z).
 * Errors: LBM_ERR_ARG (inconsistent flag field, same rules as
 * lbm_set_geometry; bad row_axis), LBM_ERR_STATE (an index invariant does
 * not hold). */
lbm_status lbm_check_layout(const uint8_t *flags, int32_t nx, int32_t ny, int32_t nz, int32_t periodic,
                            int32_t row_axis, int64_t out[8]);

/* Install the geometry: flags[nz][ny][nx] host array of LBM_SOLID / FLUID /
 * INLET / OUTLET (copied).  Builds the fluid-only sparse index (rows of
 * x-contiguous active cells, per-cell bounce-back link mask) and allocates the
 * population buffers.  Every INLET/OUTLET cell needs exactly one axis
 * neighbour that is FLUID (its extrapolation partner).  Resets the step
 * counter; populations are undefined until an init call.
 * Errors: LBM_ERR_ARG (bad flag value, inconsistent boundary node, too many
 * cells), LBM_ERR_OOM, LBM_ERR_CUDA. */
lbm_status lbm_set_geometry(lbm_ctx *ctx, const uint8_t *flags);

/* Number of active (FLUID + INLET + OUTLET) cells. */
lbm_status lbm_fluid_count(lbm_ctx *ctx, int64_t *n);

/* Wall distances for Bouzidi's interpolated bounce-back (Sec. 2.2 wall
 * treatment).  cells[n]: box indices x + nx (y + ny z) of FLUID cells next to
 * the wall; q[n][27]: for each wall link i of cell r (pull source x - c_i
 * solid or outside the box), the wall's distance from the cell centre along
 * the link as q = q[r][i] / 256, 1..255 (128 = halfway, the default of every
 * link not listed; entries of other links are ignored).  The reflected
 * population is then interpolated:
 *   q <  1/2: f_i(x) = 2q f*_ib(x) + (1 - 2q) f*_ib(x + c_i)
 *             (halfway when x + c_i is solid too),
 *   q >= 1/2: f_i(x) = f*_ib(x) / (2q) + (1 - 1/(2q)) f*_i(x),
 * with ib the direction opposite to i.  Copies both arrays to the device;
 * n = 0 restores halfway bounce-back everywhere; lbm_set_geometry clears
 * them.  LBM_ERR_ARG for a cell that is not FLUID, a cell listed twice, or
 * q = 0.  The request server always uses halfway bounce-back. */
lbm_status lbm_set_wall_q(lbm_ctx *ctx, const int64_t *cells, const uint8_t *q, int64_t n);

/* Set the flow parameters.  omega = 1/(3 nu + 1/2) (Sec. 2.1).
 * Errors: LBM_ERR_ARG unless 0 < omega < 2, ghost rates in (0, 2),
 * |u_in| and u_char below the lattice sound speed 1/sqrt(3). */
lbm_status lbm_set_params(lbm_ctx *ctx, const lbm_params *p);

/* The checks of lbm_set_params without a context (host only, no device
 * needed).  On LBM_OK, *nu receives the lattice viscosity (p->nu, or
 * u_char L_char / Re, Sec. 2.2 Reynolds number) and *omega the relaxation
 * rate 1/(3 nu + 1/2) (Sec. 2.1 relaxation time tau = nu / theta0 + 1/2);
 * on LBM_ERR_ARG both receive 0.  *why receives a static string naming the
 * failed check ("" on success).  Any of nu, omega, why may be NULL. */
lbm_status lbm_params_check(const lbm_params *p, double *nu, double *omega, const char **why);

/* A run given in physical units (SI), as Sec. 2.2 states the problem. */
typedef struct {
    double Re;       /* Reynolds number on the throat, Re = rho u_thr d_thr / mu */
    double d_thr;    /* throat diameter (m) */
    double rho;      /* fluid density (kg / m^3) */
    double mu;       /* dynamic viscosity (Pa s) */
    double delta_r;  /* grid spacing (m) */
    double delta_t;  /* time step (s); <= 0: the CFL rule below gives it */
    double CFL;      /* used when delta_t <= 0: CFL = 2 u_thr delta_t / delta_r (Sec. 2.2) */
} lbm_physical;

/* Lattice parameters of a physical run (host only, no device needed), from
 * the relations of Sec. 2.2: the throat mean velocity
 * u_thr = mu Re / (rho d_thr); the time step, when not given, of the CFL rule
 * delta_t = rho d_thr delta_r CFL / (2 mu Re); and in cells and steps the
 * characteristic length L_char = d_thr / delta_r, velocity
 * u_char = u_thr delta_t / delta_r and viscosity nu = mu delta_t / (rho delta_r^2),
 * so that omega = 1/(3 nu + 1/2) equals delta_t / tau with the relaxation time
 * tau = mu / (rho theta0) + delta_t / 2 of Sec. 2.1.  On LBM_OK it sets
 * p->Re, p->u_char and p->L_char, and p->nu = 0 (nu then follows from Re),
 * leaving the other fields of p as they were (fill it with
 * lbm_params_default first); out (may be NULL) receives L_char, u_char, nu,
 * CFL and delta_t (s).  The result must pass lbm_params_check (u_char below
 * the lattice sound speed, 0 < omega < 2); otherwise p is unchanged, out is
 * zero and the call returns LBM_ERR_ARG.  *why (may be NULL) receives "" or a
 * static string naming the failed check. */
lbm_status lbm_params_from_physical(const lbm_physical *ph, lbm_params *p, double out[5], const char **why);

/* The relaxation rate omega in use. */
lbm_status lbm_get_omega(lbm_ctx *ctx, double *omega);

/* f = f^eq(rho, u) on every active cell (uniform state); resets the step
 * counter and the statistics. */
lbm_status lbm_init_equilibrium(lbm_ctx *ctx, double rho, const double u[3]);

/* f = f^eq(rho(x), u(x)) from host arrays rho[n], u[n][3] in the given layout. */
lbm_status lbm_init_fields(lbm_ctx *ctx, const double *rho, const double *u, int32_t layout);

/* Set / read the populations f_i (post-collision state at the current time)
 * from / to a host array f[n][27].  Values are converted to the storage
 * precision (FP16S rounds (f - w) s to nearest even). */
lbm_status lbm_set_populations(lbm_ctx *ctx, const double *f, int32_t layout);
lbm_status lbm_get_populations(lbm_ctx *ctx, double *f, int32_t layout);

/* Enqueue n >= 0 time steps on the context stream (asynchronous).  Each step
 * is the fluid kernel (FP32: one warp per tile of up to 32 cells of a row;
 * FP16S, FP64 and general ghost rates: one thread per cell) on the context's
 * stream, and the inlet/outlet and interpolated-wall kernels on the second
 * stream beside it; they read the same input and write disjoint outputs, so
 * their order changes no result.  The health check and the statistics
 * sampling ride on these kernels when due.
 * Errors: LBM_ERR_STATE (no geometry / params / init), LBM_ERR_CUDA. */
lbm_status lbm_step(lbm_ctx *ctx, int64_t n);

/* Wait for the stream; report a deferred LBM_ERR_UNSTABLE (a health check saw
 * a non-finite value) or LBM_ERR_CUDA.  The unstable flag stays set until the
 * next init call. */
lbm_status lbm_sync(lbm_ctx *ctx);

/* Number of steps taken since the last init. */
lbm_status lbm_step_count(lbm_ctx *ctx, int64_t *t);

/* Every k >= 1 steps, fold the health check (FP64 mass, momentum, non-finite
 * count, max |u|) into the step kernel; k = 0 disables it (default). */
lbm_status lbm_set_check_every(lbm_ctx *ctx, int64_t k);

/* Density and velocity of every active cell (moments of the current state;
 * equal to the pre-collision moments by conservation): rho[n], u[n][3]. */
lbm_status lbm_get_moments(lbm_ctx *ctx, double *rho, double *u, int32_t layout);

/* FP64 totals over active cells: mass = sum rho, mom = sum rho u, computed
 * on the device by a deterministic fixed-order reduction (Sec. 2.1 moments). */
lbm_status lbm_get_totals(lbm_ctx *ctx, double *mass, double mom[3]);

/* Health record of the last check (check_every or lbm_get_totals):
 * out[0] mass, out[1..3] momentum, out[4] max |u|, out[5] non-finite count. */
lbm_status lbm_get_health(lbm_ctx *ctx, double out[6]);

/* Time averages (Sec. 2.2, mean/fluctuation decomposition and Reynolds
 * stress): from the next step on, every stride-th step adds u_z and u_z^2 of
 * every active cell to FP64 accumulators.  lbm_stats_end stops sampling. */
lbm_status lbm_stats_begin(lbm_ctx *ctx, int64_t stride);
lbm_status lbm_stats_end(lbm_ctx *ctx);
lbm_status lbm_stats_reset(lbm_ctx *ctx);

/* Statistics modes.  LBM_STATS_AXIAL (default): sum u_z and u_z^2, 16 bytes
 * per slot.  LBM_STATS_FULL: additionally the three velocity components, the
 * six products u_a u_b, the six components of the viscous stress
 * sigma_ab = -(1 - omega/2) a_ab from each cell's pre-collision second-order
 * central Hermite moments a_ab (Appendix A strain-rate relation with the sign
 * of the non-equilibrium stress; Sec. 2.2 viscous shear stress), and rho;
 * 144 bytes per slot.  An inlet/outlet node takes the stress of its interior
 * partner, whose non-equilibrium part it copies.  lbm_stats_set_mode takes
 * effect at the next lbm_stats_begin; changing the mode while sampling is
 * LBM_ERR_STATE, and a new mode discards the accumulated samples. */
#define LBM_STATS_AXIAL 0
#define LBM_STATS_FULL 1
#define LBM_STATS_FULL_COMPONENTS 16
lbm_status lbm_stats_set_mode(lbm_ctx *ctx, int32_t mode);

/* Means over the samples: mean_uz[n] = <u_z>, mean_uzuz[n] = <u_z^2> (either
 * may be NULL), and the sample count.  RMS = sqrt(<u_z^2> - <u_z>^2); the
 * axial Reynolds normal stress is rho (<u_z^2> - <u_z>^2). */
lbm_status lbm_stats_get(lbm_ctx *ctx, double *mean_uz, double *mean_uzuz, int64_t *n_samples,
                         int32_t layout);

/* Full-mode means, mean[n][16] row-major per cell: <u_x>, <u_y>, <u_z>,
 * <u_x u_x>, <u_y u_y>, <u_z u_z>, <u_x u_y>, <u_x u_z>, <u_y u_z>,
 * <sigma_xx>, <sigma_yy>, <sigma_zz>, <sigma_xy>, <sigma_xz>, <sigma_yz>,
 * <rho> (lattice units; solid cells of the box layout are 0).  The Reynolds
 * stress tensor (Sec. 2.2) is <rho> (<u_a u_b> - <u_a><u_b>).  mean may be
 * NULL to read the sample count.  LBM_ERR_STATE if the accumulators were
 * filled in axial mode. */
lbm_status lbm_stats_get_full(lbm_ctx *ctx, double *mean, int64_t *n_samples, int32_t layout);

/* Checkpoint: the current populations (native storage precision, bitwise),
 * the step counter and the statistics accumulators (either mode).  lbm_restore needs a
 * context with the same geometry, precision and scale. */
lbm_status lbm_checkpoint_size(lbm_ctx *ctx, size_t *bytes);
lbm_status lbm_checkpoint(lbm_ctx *ctx, void *buf, size_t bytes);
lbm_status lbm_restore(lbm_ctx *ctx, const void *buf, size_t bytes);

/* Largest cell count lbm_totals_noalloc accepts (set by its static scratch). */
#define LBM_NOALLOC_MAX_CELLS 16777216

/* FP64 totals of a caller-owned population array, allocating nothing.
 * The paper has no counterpart: this is a service for callers that cannot let
 * the library allocate device memory -- applications whose device memory
 * belongs to their own pool and fixed budget, and latency-critical loops in
 * which cudaMalloc / cudaFree would synchronise the device.  Nothing is
 * allocated: no cudaMalloc, no cudaFree, no allocator callback.
 *   f:      DEVICE pointer to the populations in this library's storage form:
 *           array i at f + i * stride elements, cells 0 .. n-1 contiguous,
 *           each element f_i - w_i (FP64 / FP32) or (f_i - w_i) * fp16_scale
 *           as an FP16 (FP16S; fp16_scale 0 selects 4096).
 *   n:      cells, 1 <= n <= LBM_NOALLOC_MAX_CELLS; stride >= n.
 *   out:    DEVICE pointer to 6 doubles, written with: mass sum rho, momentum
 *           sum rho u (3), max |u|, count of non-finite cells.
 *   stream: cudaStream_t (NULL: default stream); the call only enqueues work.
 * The per-block partial sums live in one static device array (256 KB) that
 * every GPU which loads the library holds until the process exits.  The first
 * call in a CUDA context (per device, and again after a context is re-created,
 * e.g. after cudaDeviceReset) looks up that array's device address with the
 * device current; host threads may call concurrently, the lookup is guarded.
 * Make that first call before any stream capture: if it finds `stream`
 * capturing it returns LBM_ERR_STATE and enqueues nothing.  All calls share
 * the array: calls whose work overlaps on the GPU (e.g. on two streams) race
 * and must be serialised by the caller.  Every call overwrites all the
 * partials it reads, so nothing needs clearing between calls.  The returned
 * status covers this call's own launches only.
 * Errors: LBM_ERR_ARG (NULL pointer, n out of range, stride < n, bad
 * precision or scale), LBM_ERR_STATE (first call in a context inside a stream
 * capture), LBM_ERR_CUDA. */
lbm_status lbm_totals_noalloc(const void *f, int32_t precision, float fp16_scale, int64_t n, int64_t stride,
                              double *out, void *stream);

/* Layout facts for measurement: number of storage slots (active cells plus
 * row padding), bytes of one population buffer, device bytes held. */
lbm_status lbm_layout_info(lbm_ctx *ctx, int64_t *slots, int64_t *buffer_bytes, int64_t *device_bytes);

/* Kernels lbm_step has launched on this context since its creation, counted
 * at each launch: the fluid kernel(s) of the variant that runs (FP32: the
 * tile kernel; FP16S: the chunk kernel and the pair kernel; FP64 and general
 * ghost rates: the chunk kernel), the interpolated-wall kernel, the
 * inlet/outlet kernel and, on health-check steps, the final reduction pass.
 * The difference of two readings is the launch count of the steps between
 * them.  LBM_ERR_ARG if ctx or n is NULL. */
lbm_status lbm_kernel_launches(lbm_ctx *ctx, int64_t *n);

/* ------------------------------------------------------------------ serving
 * A request server runs many lattices (nozzle / pipe runs of different
 * sizes, Re, step counts and storage precisions) on one GPU with continuous
 * batching: queued requests are admitted into resident slots as memory and
 * slots free up (admission by exact device footprint against a budget),
 * and every scheduling tick advances all resident lattices together with one
 * persistent multi-lattice launch per precision and step, replayed from a
 * captured CUDA graph.  Finished lattices are read back (rho, u) and freed.
 * Each lattice is advanced by exactly the arithmetic of lbm_step, so a
 * result does not depend on what else is resident.  (This is a service
 * around the method of the paper, which has no counterpart.) */

#define LBM_SERVER_MAX_SLOTS 64

typedef struct lbm_server lbm_server;

typedef struct {
    int32_t device;
    void *stream;            /* cudaStream_t (NULL: default stream) */
    lbm_allocator allocator; /* alloc == NULL: cudaMalloc / cudaFree */
    int64_t budget_bytes;    /* device bytes the resident lattices may hold (> 0) */
    int32_t max_slots;       /* resident lattices at most, 1..LBM_SERVER_MAX_SLOTS */
    int32_t steps_per_tick;  /* lattice steps per tick, even, 2..1024 */
} lbm_server_desc;

typedef struct {
    int32_t nx, ny, nz, periodic;
    int32_t precision;       /* LBM_FP32 or LBM_FP16S */
    float fp16_scale;        /* 0 selects 4096 */
    const uint8_t *flags;    /* host flag field [nz][ny][nx], copied by lbm_server_submit */
    lbm_params params;       /* default ghost rates only */
    int64_t steps;           /* time steps to run, >= 1; the lattice starts at rest (rho 1, u 0) */
} lbm_request;

enum { LBM_REQ_QUEUED = 0, LBM_REQ_RUNNING = 1, LBM_REQ_DONE = 2, LBM_REQ_CANCELLED = 3, LBM_REQ_FAILED = 4 };

/* Create / destroy a server.  Errors: LBM_ERR_ARG, LBM_ERR_CUDA. */
lbm_status lbm_server_create(const lbm_server_desc *desc, lbm_server **out);
lbm_status lbm_server_destroy(lbm_server *s);
const char *lbm_server_last_error(const lbm_server *s);

/* Queue a request; *id receives its handle.  The flag field is checked and
 * its sparse index built in a background host thread.  The server's
 * multi-lattice kernels address populations with 32-bit offsets, so a
 * lattice needs fewer than 2^32 / 27 storage slots (active cells plus row
 * padding and bounce-back ghost slots, about 159 M); larger ones run with
 * lbm_step.  Errors: LBM_ERR_ARG (bad request; more active cells than that
 * limit), LBM_ERR_OOM (its lattice can never fit the budget).  A request
 * whose index turns out to need too many slots, or whose exact footprint
 * exceeds the budget, ends FAILED at a later tick. */
lbm_status lbm_server_submit(lbm_server *s, const lbm_request *req, int64_t *id);

/* Every check lbm_server_submit and the later admission apply to a request,
 * on the host, without a server or a device: the checks of submit, the
 * sparse index build with the 32-bit slot limit, and the exact device
 * footprint against budget_bytes.  out (may be NULL) receives: active cells,
 * storage slots, device footprint in bytes, inlet/outlet nodes.  *why (may
 * be NULL) receives "" or the reason of a refusal (valid until the next
 * call of this function on the same thread).
 * Errors: LBM_ERR_ARG, LBM_ERR_OOM (as lbm_server_submit). */
lbm_status lbm_server_check_request(const lbm_request *req, int64_t budget_bytes, int64_t out[4],
                                    const char **why);

/* One scheduling tick: admit queued requests whose index is built (in
 * submission order, while a slot is free and the footprint fits), advance
 * every resident lattice by up to steps_per_tick steps, retire the finished
 * ones (read back rho, u; free their memory).  The last step a lattice takes
 * in a tick is its health check: a lattice with a non-finite density or
 * velocity is evicted (its memory freed) and ends FAILED with
 * LBM_ERR_UNSTABLE; the others are not affected.  Blocks until the tick's
 * work is done.  Outputs (may be NULL): resident lattices, queued requests. */
lbm_status lbm_server_tick(lbm_server *s, int32_t *running, int32_t *queued);

/* State (LBM_REQ_*) and steps done of a request. */
lbm_status lbm_server_poll(lbm_server *s, int64_t id, int32_t *state, int64_t *steps_done);

/* Number of active cells of a request (known once its index is built;
 * LBM_ERR_STATE before). */
lbm_status lbm_server_cells(lbm_server *s, int64_t id, int64_t *active_cells);

/* Final density rho[n] and velocity u[n][3] of a finished (DONE) request,
 * in the active order of its flag field.  Called on any terminal request
 * (DONE, FAILED, CANCELLED) it releases everything the server keeps for it,
 * and the id is no longer valid afterwards; a FAILED request returns the
 * status it failed with (LBM_ERR_UNSTABLE after a health check, LBM_ERR_ARG
 * for a bad flag field or too many slots, LBM_ERR_OOM for a footprint above
 * the budget, LBM_ERR_CUDA) and a CANCELLED one LBM_ERR_STATE, with the
 * reason in lbm_server_last_error.
 * Errors: LBM_ERR_STATE if still queued or running (the request is kept). */
lbm_status lbm_server_result(lbm_server *s, int64_t id, double *rho, double *u);

/* Cancel a queued or running request (its memory is freed at the next tick). */
lbm_status lbm_server_cancel(lbm_server *s, int64_t id);

/* Counters: out[0] cell updates done, out[1] ticks, out[2] device bytes held
 * now, out[3] peak device bytes, out[4] graph launches, out[5] graph
 * captures, out[6] requests finished, out[7] requests queued. */
lbm_status lbm_server_info(lbm_server *s, double out[8]);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
