/*
 * lbgm.h -- lattice Boltzmann for generalized metrics on one NVIDIA GB300.
 *
 * C ABI of liblbgm.so: the per-time-step fused collide-and-stream update of
 * the lattice Boltzmann (LB) model in curvilinear coordinates of
 *   J.-D. Debus, M. Mendoza, H. J. Herrmann, "Dean Instability in
 *   Double-Curved Channels" (arXiv:1411.3133),
 * Sec. II (method), Sec. III (cylindrical channel), Sec. IV (double-curved
 * channel in ellipsoidal coordinates).
 *
 * Conventions for every entry point
 *   - Every call returns lb_status and never aborts the process. On failure
 *     lb_last_error(ctx) (or lb_last_error(NULL) for calls without a context)
 *     returns a message.
 *   - After a CUDA error or a detected non-finite state the context is
 *     poisoned: lb_step, lb_macros and lb_diagnostics return LB_ERR_STATE
 *     until lb_init, lb_init_fields, lb_set_populations or lb_set_state
 *     succeeds.
 *   - The library owns the device memory of a context (allocated at
 *     lb_create_geometry, through the caller's lb_allocator if one is given);
 *     callers own every output buffer they pass in.
 *   - Work is enqueued on the context's CUDA stream. Calls returning host data
 *     synchronise that stream. Calls on one context are not thread-safe.
 *   - Field layout (lb_macros, lb_init_fields): for instance b and node
 *     (i_r, i_theta, i_3) the linear index is
 *       b * N + (i_r * ntheta + i_theta) * n3 + i_3,   N = nr * ntheta * n3.
 *     Vector fields add the component as the slowest axis inside an instance:
 *       u[(b * 3 + i) * N + cell], i = 0 (r), 1 (theta), 2 (x3).
 *   - Population layout (lb_get_populations, lb_set_populations):
 *       f[(b * LB_Q + l) * N + cell], l in the order of lb_velocity_set().
 *   - Units are lattice units: time step 1, lattice spacing h = (r_outer -
 *     r_inner) / nr on every axis (Sec. III: Delta r = Delta theta = Delta z
 *     = Delta t), velocities per step in coordinate components.
 */
#ifndef LBGM_H
#define LBGM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LB_Q 41            /* D3Q41, Table I */
#define LB_GEO_STRIDE 44   /* doubles per row of lb_geometry_eval */

typedef struct lb_ctx lb_ctx;

typedef enum {
  LB_OK = 0,
  LB_ERR_ARG = 1,        /* invalid argument; nothing was changed */
  LB_ERR_CUDA = 2,       /* a CUDA call failed; context poisoned */
  LB_ERR_NONFINITE = 3,  /* the state holds NaN/Inf (divergence); poisoned */
  LB_ERR_TIMEOUT = 4,    /* a bounded device wait gave up */
  LB_ERR_STATE = 5       /* context poisoned or not initialised */
} lb_status;

typedef enum {
  LB_METRIC_FLAT = 0,         /* Cartesian channel, walls normal to x^1 */
  LB_METRIC_CYLINDRICAL = 1,  /* (r, theta, z), Sec. III */
  LB_METRIC_ELLIPSOIDAL = 2,  /* (r, theta, phi), a = c = 1, Sec. IV */
  LB_METRIC_ELLIPSOIDAL_THETA = 3  /* the same coordinates with the metric of
                                      each theta node (theta-resolved; see
                                      lb_geometry_desc); FP64 and FP32
                                      storage, the plain step kernel, no
                                      lb_batch membership */
} lb_metric;

typedef enum {
  LB_FP64 = 0,          /* populations and arithmetic in FP64 */
  LB_FP32 = 1,          /* populations and arithmetic in FP32 */
  LB_FP16_SHIFTED = 2,  /* populations stored in FP16 as the scaled deviation
                           (f_l - r_l) / w_l from a reference population r_l
                           per geometry row (LB_OPT_STORAGE_REFERENCE: the
                           initial rows' equilibria, or w_l); FP32
                           arithmetic */
  LB_BF16_SHIFTED = 3   /* the same deviation stored in BF16; FP32 arithmetic */
} lb_precision;

/* Wall condition of the walled axes (r, and x3 when periodic3 == 0). */
typedef enum {
  LB_WALL_BOUNCEBACK = 0,  /* walls halfway outside the first and last node;
                              populations reflected along their one-step
                              path (full bounce-back) */
  LB_WALL_EQUILIBRIUM = 1  /* the paper's Dirichlet walls (Sec. III: zero
                              wall velocity imposed through the
                              equilibrium on both walls at every step):
                              the first and last node lie on the
                              walls and leave every step as f^eq(rho', 0)
                              of their own density; a population whose
                              source lies beyond a wall is read from the
                              wall node of the same line. First-order
                              accurate; mass is not conserved exactly. */
} lb_wall;

/* Channel geometry (Sec. III lattice map; Sec. IV lattice map and the
 * rescaled spacings of Sec. IV.B).
 *   LB_WALL_BOUNCEBACK: nodes at r = r_inner + (i_r + 1/2) h, i_r = 0..nr-1,
 *   h = (r_outer - r_inner)/nr, so that the walls are halfway outside the
 *   first and last node, exactly at r_inner and r_outer. The third axis is
 *   centred: x3 = (i_3 + 1/2 - n3/2) h * d3_scale.
 *   LB_WALL_EQUILIBRIUM: nodes at r = r_inner + i_r h, h = (r_outer -
 *   r_inner)/(nr - 1) (wall nodes at both ends); a walled third axis
 *   x3 = (i_3 - (n3 - 1)/2) h * d3_scale, a periodic one as above.
 *   The metric is evaluated at theta = 0 for every theta node (quasi-2-D
 *   channel, periodic in theta); the Christoffel symbols of both coordinate
 *   systems do not depend on theta. LB_METRIC_ELLIPSOIDAL_THETA evaluates
 *   the printed Sec. IV metric at each theta node instead, theta =
 *   (i_theta + 1/2 - ntheta/2) h * dtheta_scale (centred on theta = 0), the
 *   theta axis still periodic: off theta = 0 with b != 1 every off-diagonal
 *   metric component is present (full Delta^ij, body force g^{i theta} G
 *   with r and phi components). */
typedef struct {
  double r_inner, r_outer;  /* wall positions, 0 < r_inner < r_outer
                               (any r_inner < r_outer for FLAT) */
  double b;                 /* ellipsoid semi-axis b > 0; ignored otherwise */
  int nr, ntheta, n3;       /* nodes per axis: nr >= 7, ntheta >= 1, n3 >= 1
                               (n3 >= 7 when periodic3 == 0) with
                               bounce-back walls */
  int periodic3;            /* 1: periodic third axis; 0: walls there too */
  double dtheta_scale;      /* Delta theta / h (> 0; 1 unless rescaled) */
  double d3_scale;          /* Delta x3 / h (> 0; 1 unless rescaled) */
  int wall;                 /* lb_wall (nr >= 3 and walled n3 >= 3 suffice
                               for LB_WALL_EQUILIBRIUM) */
} lb_geometry_desc;

/* Per-instance run parameters (Sec. II; Sec. III for the driving force). */
typedef struct {
  double tau;               /* BGK relaxation time in steps, > 1/2;
                               nu = (tau - 1/2) cs^2 (Eq. viscosity) */
  double force_G;           /* constant covariant streamwise force per step:
                               F^i_ext = g^{i theta} * force_G */
  int old_forcing;          /* 0: improved forcing a2 = a2^eq - sigma (Sec. II);
                               1: the earlier method, a2 = a2^eq;
                               2: improved forcing with the half-force
                               velocity -- not the paper's printed scheme:
                               f^eq and the forcing term take
                               u_s = u + M(u_s) / (2 rho'), M the forcing
                               term's first moment (two fixed-point
                               iterations from u = sum c f / rho'), and the
                               forcing term is scaled by 1 - 1/(2 tau).
                               FP64 and FP32 storage only; a context with
                               any such instance runs the plain step kernel
                               (LB_OPT_STEP_KERNEL is ignored) and cannot
                               join an lb_batch. lb_macros still reports
                               u = sum c f / rho'. */
  unsigned long long seed;  /* velocity noise seed (see lb_init) */
  double noise_amp;         /* noise amplitude (lattice velocity units) */
  int init_base_flow;       /* 1: start from the laminar profile for force_G
                               (FLAT and CYLINDRICAL with dtheta_scale == 1) */
} lb_params;

/* Observables of one instance (Sec. III Eq. dean-number and its Sec. IV
 * form, the mean streamwise velocity and the mean absolute streamwise
 * vorticity). */
typedef struct {
  double mass_rho_prime;    /* sum over nodes of rho' */
  double mass_physical;     /* sum over nodes of rho' g  (= rho sqrt g) */
  double mean_v_theta;      /* <v_theta>, area mean of sqrt(g_thth) u^theta */
  double dean;              /* <v_theta> nr / nu * sqrt(d / R); 0 for FLAT */
  double mean_vorticity;    /* <omega^theta> */
  double vortex_amp;        /* rms of u^r over all nodes */
  double vortex_amp_x3;     /* rms of u^r minus its mean along x3 */
  double max_speed;         /* largest Euclidean norm of u (coordinates) */
  long long nonfinite;      /* nodes with a non-finite rho' or u */
  long long step;           /* time steps since initialisation */
} lb_diag;

/* Optional device allocator (e.g. a framework's caching allocator). alloc
 * returns a device pointer aligned to 256 bytes or NULL; free releases it. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* user);
  void (*free)(void* ptr, size_t bytes, void* stream, void* user);
  void* user;
} lb_allocator;

typedef enum {
  LB_OPT_CHECK_EVERY = 0,   /* lb_step checks for non-finite values every k
                               steps (k >= 0; 0: never; default 0) */
  LB_OPT_BLOCK_THREADS = 1, /* threads per block of the step kernel
                               (64..256, multiple of 32; default 128). The
                               one-node-per-thread kernel with FP32
                               arithmetic runs at most 128 per block (its
                               register cap); larger values run as 128 */
  LB_OPT_USE_GRAPH = 2,     /* 1: lb_step replays a captured CUDA graph of
                               pairs of steps (default 0) */
  LB_OPT_STEP_KERNEL = 3,   /* 0: automatic (default): FP64 arithmetic 1,
                               else 4 where x3 is periodic with bounce-back
                               walls, else 5;
                               1: the one-node-per-thread kernel, gathering
                               from global memory; 2: the TMA-pipelined
                               kernel (FP32, bounce-back walls and n3 in
                               {128, 256} only);
                               4: the region split (periodic x3 and
                               bounce-back walls only): one
                               kernel for the 3 node layers next to each
                               r-wall, one for the interior without any
                               wall code; 5: tiled: runs of interior nodes
                               and the wall nodes in two kernels (the
                               lb_batch work-list kernels over this context
                               alone), for any geometry. With instances
                               of the half-force velocity variant
                               (lb_params.old_forcing 2) the context runs
                               kernel 1 whatever is set here.
                               Unsupported choices return LB_ERR_ARG. All
                               give bitwise identical states. */
  LB_OPT_SCHEDULE = 4,      /* batches only (lb_batch_set_option): 0: one
                               block per tile of block_threads nodes
                               (default); 1: a persistent grid of (resident
                               blocks per SM) x (SMs) blocks that walks the
                               tile list. Both give bitwise identical
                               states. */
  LB_OPT_TILE_BLOCKS = 5,   /* batches only (lb_batch_set_option): nodes per
                               work-list tile, in blocks' worth: 1
                               (default), 2 or 4; each thread of a tile's
                               block takes every blockDim-th node of it.
                               Bitwise neutral. */
  LB_OPT_STORAGE_REFERENCE = 6 /* FP16/BF16 storage only: the reference
                               r_l of the stored deviation (f_l - r_l)/w_l.
                               0: r_l = w_l (the rest state of unit
                               density); 1 (default): the equilibrium of
                               each geometry row's initial state -- lb_init:
                               rho' = 1/sqrt(g) and the laminar profile where
                               init_base_flow is set, rest otherwise;
                               lb_init_fields: the row means of the given
                               fields. The
                               small perturbations of an instability are
                               then stored as small numbers. Changing it
                               requires lb_init again (LB_ERR_STATE until
                               then); state bytes (lb_get_state) are
                               deviations from the reference of the last
                               initialisation or lb_capture_reference. */
} lb_option;

/* One configuration measured by lb_autotune / lb_batch_autotune. */
typedef struct {
  int block_threads;   /* LB_OPT_BLOCK_THREADS */
  int schedule;        /* contexts: LB_OPT_STEP_KERNEL (1, 2, 4 or 5);
                          batches: LB_OPT_SCHEDULE (0 or 1) */
  int tile_nodes;      /* batches: nodes per work-list tile (block_threads x
                          LB_OPT_TILE_BLOCKS); contexts: 0 */
  double ms_per_step;  /* measured with CUDA events on the stream */
} lb_tune;

/* --------------------------------------------------------------------- */

/* Library's D3Q41 velocities c[l*3 + i] and weights w[l] (Table I) in the
 * order used by lb_get_populations. Either pointer may be NULL. Returns
 * LB_Q. Host only. */
int lb_velocity_set(int* c, double* w);

/* Host-only geometry evaluation (Sec. III metric and symbols; Sec. IV metric
 * and symbols; Sec. IV.B rescaling; lattice Christoffels h * Gamma). Writes
 * nr * n3 rows (row = i_r * n3 + i_3; LB_METRIC_ELLIPSOIDAL_THETA: nr *
 * ntheta * n3 rows, row = (i_r * ntheta + i_theta) * n3 + i_3) of
 * LB_GEO_STRIDE doubles:
 *   [0..8]   Delta^ij = g^ij - delta^ij   (row-major 3x3, scaled metric)
 *   [9..35]  h * Gamma^i_jk               (index (i*3 + j)*3 + k)
 *   [36..38] g^{i theta}                  (body force per unit force_G)
 *   [39] sqrt(det g)   [40] sqrt(g_thth)  [41] area weight of the (r, x3)
 *   cross-section (physical metric)       [42] sqrt(g_thth) physical
 *   [43] physical radius r of the node.
 * out_len is the capacity of out in doubles. Needs no GPU. */
lb_status lb_geometry_eval(lb_metric metric, const lb_geometry_desc* geom,
                           double* out, size_t out_len);

/* Force per step giving Dean number De in the laminar state (Sec. III Eq.
 * dean-number with the curved channel Poiseuille profile v = A r ln r + B r
 * + C / r, A = -G / (2 nu h^2), averaged over the nodes). CYLINDRICAL with
 * dtheta_scale == 1 only (LB_ERR_ARG otherwise). Needs no GPU. */
lb_status lb_force_for_dean(lb_metric metric, const lb_geometry_desc* geom,
                            double tau, double De, double* G_out);

/* Create a context holding `batch` independent instances of one channel
 * geometry (each with its own lb_params), in precision `prec`, working on
 * `cuda_stream` (a cudaStream_t; NULL: the library creates its own stream).
 * Evaluates the geometry on the host in FP64 (lb_geometry_eval) and uploads
 * it. `alloc` may be NULL (cudaMalloc). On success *out owns its memory
 * until lb_destroy. Limits (LB_ERR_ARG beyond them): batch <= 65535,
 * batch * nodes < 2^32, and one instance's populations (41 * nodes * bytes
 * per population) below 4 GiB. */
lb_status lb_create_geometry(lb_metric metric, const lb_geometry_desc* geom,
                             int batch, lb_precision prec, void* cuda_stream,
                             const lb_allocator* alloc, lb_ctx** out);

/* Initial state (end of Sec. II: f = f^eq(rho', u) from initial fields) for
 * every instance b from params[b]: rho' = 1/sqrt(g) (uniform rho = rho' sqrt g
 * = 1, Sec. IV) and u = base flow (init_base_flow) plus noise
 *   u^i += noise_amp * (2 U - 1),  U = (s >> 11) * 2^-53,
 * where s is output number k = 3 * cell + i (cell within the instance,
 * counting from 0) of the SplitMix64 generator seeded with params[b].seed.
 * Resets the step counter. */
lb_status lb_init(lb_ctx* ctx, const lb_params* params);

/* Initial state f = f^eq(rho', u) from caller fields rho[batch * N] and
 * u[batch * 3 * N] (host pointers if on_device == 0, else device pointers on
 * the context's device), with params[b] for tau and the force. */
lb_status lb_init_fields(lb_ctx* ctx, const lb_params* params, const double* rho,
                         const double* u, int on_device);

/* n >= 0 time steps (Eq. LB): pull streaming with full bounce-back at the
 * walls, moments, f^eq, non-equilibrium stress, forcing term with the
 * Christoffel symbols and the body force, BGK collision. Asynchronous unless
 * LB_OPT_CHECK_EVERY is set; then returns LB_ERR_NONFINITE when a check
 * finds a non-finite density. */
lb_status lb_step(lb_ctx* ctx, long long n);

/* rho' and u of the current state (moments of the streamed populations,
 * Sec. II) into rho[batch * N], u[batch * 3 * N] (either may be NULL). */
lb_status lb_macros(lb_ctx* ctx, double* rho, double* u, int on_device);

/* Observables of every instance into out[batch] (host). Synchronises. */
lb_status lb_diagnostics(lb_ctx* ctx, lb_diag* out);

/* Populations of the state as FP64 in the documented layout, f[batch * LB_Q
 * * N]. The conversion is exact both ways for LB_FP32; for the reduced-
 * precision formats a state read out and written back is unchanged (the
 * stored deviations round-trip). */
lb_status lb_get_populations(lb_ctx* ctx, double* f, int on_device);

/* Convergence monitor: per instance b, change[b] = max over nodes and
 * components of |u - u_prev| and umax[b] (may be NULL) = max |u|, with u
 * the velocity of lb_macros; then u_prev = u. u_prev is a caller-owned
 * DEVICE array [batch * 3 * N] in the field layout (start it from
 * lb_macros(..., on_device = 1)); change, umax are host arrays [batch]. A run
 * stepped K times between two calls has converged to a per-step residual r
 * when change[b] <= r * K * umax[b]. Synchronises the stream. */
lb_status lb_velocity_change(lb_ctx* ctx, double* u_prev, double* change, double* umax);

/* FP16/BF16 storage only: make the current state the reference of the stored
 * deviations. The reference population of every geometry row becomes the
 * mean of that population over the row's nodes (all theta and x3 of a layer
 * for the cylinder and flat channel; all theta of an (r, x3) row for the
 * ellipsoid), and the state is re-encoded against it. Called once a laminar
 * state has developed, its non-equilibrium part moves into the FP32 table
 * and only departures from it -- the perturbations of an instability -- are
 * rounded to 2 bytes. The populations do not change beyond one rounding of
 * the new encoding. Synchronises the stream; LB_ERR_ARG for other precisions. */
lb_status lb_capture_reference(lb_ctx* ctx);
lb_status lb_set_populations(lb_ctx* ctx, const double* f, int on_device);

/* Raw state for checkpointing (private layout, native precision) plus the
 * step counter. lb_state_bytes gives the size. */
size_t lb_state_bytes(const lb_ctx* ctx);
lb_status lb_get_state(lb_ctx* ctx, void* buf, size_t bytes, int on_device);
lb_status lb_set_state(lb_ctx* ctx, const void* buf, size_t bytes, int on_device);

/* Set a context option (lb_option). */
lb_status lb_set_option(lb_ctx* ctx, int option, long long value);

/* Time steps taken since initialisation. */
long long lb_step_count(const lb_ctx* ctx);

/* Observables of `batch` instances from fields the caller already holds on
 * the device, for callers that cannot call cudaMalloc -- e.g. a program whose
 * device memory is all owned by another allocator, or a loop that must not
 * allocate after start-up. The paper has no counterpart; this is a way to
 * run lb_diagnostics' reduction without a context.
 *   metric, geom  the channel (as for lb_create_geometry)
 *   batch         1..LB_NOALLOC_MAX_BATCH instances
 *   tau           host array [batch] (for the Dean number)
 *   rho, u        device arrays [batch * N] and [batch * 3 * N] in the field
 *                 layout above (e.g. written by lb_macros with on_device = 1)
 *   cuda_stream   cudaStream_t to work on (NULL: the legacy default stream)
 *   out           host array [batch]; out[b].step is -1
 * Allocates no device memory: its working memory is one file-scope device
 * array of LB_NOALLOC_SCRATCH_BYTES bytes, held by every GPU that loads the
 * library until the process exits. Sizes needing more return LB_ERR_ARG.
 * Every call looks the array's address up on the current device (the one
 * rho and u live on). All calls share the array, so calls that overlap on
 * the GPU race. Synchronises cuda_stream. LB_METRIC_ELLIPSOIDAL_THETA (whose
 * weights differ per node) returns LB_ERR_ARG. Errors are reported through
 * lb_last_error(NULL). */
#define LB_NOALLOC_SCRATCH_BYTES (4u << 20)
#define LB_NOALLOC_MAX_BATCH 64
lb_status lb_diagnostics_noalloc(lb_metric metric, const lb_geometry_desc* geom, int batch,
                                 const double* tau, const double* rho, const double* u,
                                 void* cuda_stream, lb_diag* out);

/* Measured fused multiply-add peak of the current CUDA device, in flop/s
 * (2 flops per FMA): the ALU roof against which the FP64 step, bound by the
 * FP64 units rather than by HBM, is reported. Not part of the paper's
 * method; a measurement aid.
 *   precision    LB_FP64 or LB_FP32 (others: LB_ERR_ARG)
 *   cuda_stream  cudaStream_t to run on (NULL: the legacy default stream)
 *   flops_per_s  host output; best of five timed launches of a kernel in
 *                which every thread runs eight independent FMA chains
 *                (eight 256-thread blocks per SM), each lasting >= 50 ms
 *                after a warm-up launch
 * Allocates and frees a few bytes of device memory; synchronises
 * cuda_stream. Errors are reported through lb_last_error(NULL). */
lb_status lb_fma_peak(lb_precision precision, void* cuda_stream, double* flops_per_s);

/* Autotuner of the step launch. Runs steps_per_trial (>= 1) time steps in
 * each configuration -- block_threads in {64, 96, 128} (FP64: {64, 128, 192,
 * 256}) with the plain step kernel, {64, 96, 128} with the region split
 * where x3 is periodic and with the tiled step, and the TMA kernel where the
 * context supports it -- timed with
 * CUDA events on the context's stream, then keeps the fastest. Every
 * configuration computes bitwise the same states, so the trial steps are
 * real time steps: they advance the simulation and the step count. best
 * (may be NULL) receives the chosen configuration; trials (may be NULL,
 * capacity max_trials) every measured one, *n_trials their number.
 * Synchronises the stream. */
lb_status lb_autotune(lb_ctx* ctx, int steps_per_trial, lb_tune* best, lb_tune* trials, int max_trials,
                      int* n_trials);

/* Release everything the context owns. NULL is allowed. */
void lb_destroy(lb_ctx* ctx);

/* Message of the last failure on ctx (NULL: of the calling thread's last
 * call without a context). Never NULL. */
const char* lb_last_error(const lb_ctx* ctx);

/* --------------------------------------------------------------------- */
/* Batches of contexts of different geometry.
 *
 * A sweep over Dean numbers, radii and grid sizes (Sec. III and IV vary
 * the driving force, the radii ratio and the cross-section) has instances
 * of different metric kind and size. lb_batch_step advances every instance
 * of every member context by one time step per step with two launches of a
 * work-list kernel per metric kind present: one over tiles of up to
 * block_threads consecutive interior nodes (instance, first node, count),
 * one over tiles of the nodes within three nodes of a wall (instance, first
 * index into a list of wall nodes, count), so instances of any size share
 * the grid. All these launches run concurrently on forked streams (they
 * read one buffer and write disjoint nodes). The update is the one of
 * lb_step (Eq. LB), node for node, and the resulting states are bitwise
 * those of lb_step on each member.
 *
 * Members stay owned by the caller and usable with every lb_* call
 * (lb_init, lb_diagnostics, lb_get_state, ...) between batch steps; they
 * must outlive the batch, share one precision, device and stream, and
 * appear once. The batch reads each member's buffer parity before every
 * lb_batch_step call, so stepping members on their own in between is
 * allowed. */
typedef struct lb_batch lb_batch;

/* members: host array [count] of initialised or not-yet-initialised
 * contexts. No device work; the work list is built on the first step. */
lb_status lb_batch_create(lb_ctx* const* members, int count, lb_batch** out);

/* n >= 0 time steps of every member (each must be initialised). Options:
 * LB_OPT_CHECK_EVERY, LB_OPT_BLOCK_THREADS, LB_OPT_USE_GRAPH (a captured
 * graph of two batch steps), LB_OPT_SCHEDULE, LB_OPT_TILE_BLOCKS. A
 * non-finite density found by
 * a check poisons that member and returns LB_ERR_NONFINITE. */
lb_status lb_batch_step(lb_batch* batch, long long n);
lb_status lb_batch_set_option(lb_batch* batch, int option, long long value);

/* As lb_autotune over block_threads in {64, 96, 128} (FP64: {64, 96, 128,
 * 192, 256}) x LB_OPT_SCHEDULE in {0, 1} x LB_OPT_TILE_BLOCKS in {1, 2, 4}
 * (the tile length: nodes per work-list item); the trial steps are real batch
 * steps. With FP32 arithmetic the work-list kernel runs at most 128 threads
 * per block (LB_OPT_BLOCK_THREADS above that runs as 128). */
lb_status lb_batch_autotune(lb_batch* batch, int steps_per_trial, lb_tune* best, lb_tune* trials,
                            int max_trials, int* n_trials);

/* Nodes of all instances of all members (one batch step updates them all). */
long long lb_batch_nodes(const lb_batch* batch);

/* Batch steps taken since creation. */
long long lb_batch_step_count(const lb_batch* batch);

/* Release the batch's work list, streams and graph (not the members). */
void lb_batch_destroy(lb_batch* batch);

/* Message of the last failure on the batch (NULL: as lb_last_error(NULL)). */
const char* lb_batch_last_error(const lb_batch* batch);

/* --------------------------------------------------------------------- */
/* Surrogate of developed channel flow, for warm starts (no counterpart in
 * the paper). A multilayer perceptron maps an input row x = (p_1 .. p_P, z)
 * -- n_plain = P channel parameters and coordinates, each scaled by the
 * caller (typically De / 100, a curvature ratio, (r - r_i)/d), then x3 / L_3
 * in [0, 1) -- to the node's fields y = (rho', u^r, u^theta, u^3) of a
 * converged LB run. Features (p_1 .. p_P, sin(2 pi k z), cos(2 pi k z), k =
 * 1..n_fourier) feed depth - 1 hidden layers of `width` SiLU units and a
 * linear layer of 4 outputs, which predicts (y - mean)/std per field
 * (lb_mlp_set_output_scale). Weights: FP32 master copy and Adam moments,
 * BF16 in every product, FP32 accumulation; He-uniform initial weights from
 * a SplitMix64 stream seeded with `seed`, zero biases. Parameters are laid
 * out layer by layer as W (fan_out x fan_in, row-major) then b. All x, y
 * arrays are device FP32, row-major ([n][n_plain + 1], [n][4]); calls are
 * ordered on `cuda_stream` (NULL: legacy default stream). */
typedef struct lb_mlp lb_mlp;
lb_status lb_mlp_create(int n_plain, int n_fourier, int width, int depth, int max_batch, unsigned long long seed,
                        void* cuda_stream, lb_mlp** out);
size_t lb_mlp_param_count(const lb_mlp* net);
/* host arrays mean[4], std[4] (std > 0) */
lb_status lb_mlp_set_output_scale(lb_mlp* net, const float* mean, const float* std);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, learning rate lr) on the mean
 * squared error of the normalised outputs over n <= max_batch samples;
 * *loss (host, may be NULL: then no synchronisation) receives that error
 * before the step. */
lb_status lb_mlp_train_step(lb_mlp* net, const float* x, const float* y, int n, float lr, float* loss);
/* y = the network's fields at n <= max_batch inputs (asynchronous). */
lb_status lb_mlp_predict(lb_mlp* net, const float* x, int n, float* y);
/* FP32 master parameters / gradients of the last train step, host arrays of
 * lb_mlp_param_count floats; set_params also resets the Adam state. */
lb_status lb_mlp_get_params(lb_mlp* net, float* host, size_t count);
lb_status lb_mlp_set_params(lb_mlp* net, const float* host, size_t count);
lb_status lb_mlp_get_grads(lb_mlp* net, float* host, size_t count);
void lb_mlp_destroy(lb_mlp* net);
/* Message of the last failure (NULL: of the calling thread's last
 * lb_mlp_create). */
const char* lb_mlp_last_error(const lb_mlp* net);

#ifdef __cplusplus
}
#endif
#endif /* LBGM_H */
