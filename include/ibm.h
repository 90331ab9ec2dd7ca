/*
 * ibm.h -- C ABI of the GB300 (sm_103a) distribution-function-correction
 * immersed-boundary lattice Boltzmann library (arXiv 1803.09380).
 *
 * The library advances a D2Q9 BGK lattice (section 2.1, Eqs. 1, 3, 4, 7)
 * whose no-slip boundaries are immersed Lagrangian markers enforced by the
 * paper's iterative distribution-function correction (section 2.3,
 * Eqs. 22-28, with the 4-point delta function of Eq. 15c), sums the
 * corrections into body force and torque (Eq. 29, Eqs. 37-38) and moves
 * free bodies with an FP64 Newton-Euler update (Eqs. 39-42).
 *
 * Conventions for every entry point:
 *   - All arrays passed in or out are HOST memory, FP64, caller-owned; the
 *     library copies inputs before returning.  Device memory is owned by the
 *     library (plain cudaMalloc, or the allocator installed with
 *     ibm_set_allocator) and released by ibm_destroy.
 *   - Work is enqueued on the CUDA stream named in the lattice descriptor
 *     (the correction loop forks onto a private high-priority stream and
 *     joins back within each step).  ibm_step returns once the work is
 *     enqueued; ibm_read_fields synchronises the stream, so asynchronous
 *     device errors surface there (and in ibm_destroy / ibm_sync).
 *   - No exception crosses the ABI.  Every call returns an ibm_status;
 *     ibm_last_error(h) gives a message for the last failure on that handle
 *     (ibm_last_error(NULL) for a failed ibm_create_lattice).
 *   - A handle is not thread-safe: use one handle per host thread / stream.
 *   - Lattice units throughout: dx = dt = 1, c_s^2 = 1/3.  Node (x, y) sits
 *     at integer coordinates 0 <= x < nx, 0 <= y < ny.  Half-way walls sit
 *     at x = -1/2, nx - 1/2, y = -1/2, ny - 1/2.
 *   - Field arrays are row-major [ny][nx] (x fastest); populations are
 *     [9][ny][nx] in the order e0=(0,0) e1=(1,0) e2=(0,1) e3=(-1,0)
 *     e4=(0,-1) e5=(1,1) e6=(-1,1) e7=(-1,-1) e8=(1,-1) (the rows of the
 *     transform matrix of Eq. 5).
 */
#ifndef IBM_H_
#define IBM_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IBM_ABI_VERSION 5

typedef struct ibm_ctx *ibm_handle; /* opaque, library-owned */

typedef enum {
  IBM_OK = 0,
  IBM_ERR_INVALID = 1,        /* bad argument or unsupported combination */
  IBM_ERR_NOMEM = 2,          /* device or host allocation failed */
  IBM_ERR_CUDA = 3,           /* a CUDA call failed (message has details) */
  IBM_ERR_BOUNDS = 4,         /* a device-side capacity or bounds check tripped */
  IBM_ERR_DIVERGED = 5,       /* NaN/Inf found by the watchdog */
  IBM_ERR_TIMEOUT = 6,        /* a bounded device wait ran out */
  IBM_WARN_NOT_CONVERGED = 7  /* corr_tol > 0 and the residual stayed above it */
} ibm_status;

/* Storage / arithmetic precision of the populations.  FP64: stored and
 * computed in double.  FP32: stored and computed in float.  FP16_DEV and
 * BF16_DEV: f_i - w_i stored in 16 bits, arithmetic in float.  Body force,
 * torque and the Newton-Euler update are FP64 in every mode. */
typedef enum { IBM_FP64 = 0, IBM_FP32 = 1, IBM_FP16_DEV = 2, IBM_BF16_DEV = 3 } ibm_precision;

/* Rule at each domain side.  PERIODIC must be paired on opposite sides.
 * INLET_EQ is supported on the -x side only (column 0 held at
 * f^eq(rho0, inlet_u)); OUTLET_ZEROGRAD on the +x side only (populations
 * entering column nx-1 from outside copied from column nx-2). */
typedef enum {
  IBM_BC_PERIODIC = 0,
  IBM_BC_BOUNCEBACK = 1,      /* half-way bounce-back, optional wall velocity */
  IBM_BC_FREESLIP = 2,        /* specular reflection */
  IBM_BC_INLET_EQ = 3,
  IBM_BC_OUTLET_ZEROGRAD = 4,
  IBM_BC_INLET_NEE = 5,       /* -x side only: velocity inlet by non-equilibrium
                                 extrapolation (the scheme of section 3.2):
                                 column 0 is rebuilt every step as
                                 f^eq(rho(1), inlet_u) + f(1) - f^eq(rho(1), u(1)) */
  IBM_BC_OUTLET_NEE = 6       /* +x side only: pressure outlet by the same
                                 extrapolation, column nx-1 rebuilt as
                                 f^eq(rho0, u(nx-2)) + f(nx-2) - f^eq(nx-2);
                                 marker supports must stay off the two
                                 columns next to an extrapolation side */
} ibm_bc;

/* Collision operator.  BGK: Omega_i = -(f_i - f_i^eq)/tau.  MRT: Eq. 2
 * with the transform matrix of Eq. 5 and the diagonal relaxation matrix of
 * Eq. 6; with every rate equal to 1/tau it is BGK. */
typedef enum { IBM_COLL_BGK = 0, IBM_COLL_MRT = 1 } ibm_collision;

enum { IBM_SIDE_XMIN = 0, IBM_SIDE_XMAX = 1, IBM_SIDE_YMIN = 2, IBM_SIDE_YMAX = 3 };

typedef struct {
  int nx, ny;                 /* lattice size, 4 <= nx, ny; nx*ny < 2^31 */
  double tau;                 /* BGK relaxation time, > 0.5 (nu = (tau - 1/2)/3, Eq. 8) */
  double rho0;                /* reference density: initial state, inlet, walls */
  int prec;                   /* ibm_precision */
  int bc[4];                  /* ibm_bc per side, indexed by IBM_SIDE_* */
  double wall_u[4][2];        /* velocity of each bounce-back side */
  double inlet_u[2];          /* inlet velocity */
  int n_corr;                 /* correction iterations N per step (paper: about 10) */
  double corr_tol;            /* 0: always N iterations; > 0: report
                                 IBM_WARN_NOT_CONVERGED when r^N > corr_tol */
  int delta_points;           /* delta function of Eq. 15: 2 (15a), 3 (15b) or
                                 4 (15c, the paper's choice); 0 means 4.  A
                                 marker's 4 x 4 node window must stay inside
                                 a non-periodic domain for every choice */
  void *cuda_stream;          /* cudaStream_t to enqueue on; NULL: the library
                                 creates its own stream, which synchronises
                                 with the legacy default stream */
  int device;                 /* CUDA device ordinal */
  int collision;              /* ibm_collision; 0 (zero-initialised) is BGK */
  double mrt_s[3];            /* MRT rates s_e, s_eps, s_q of Eq. 6 for the
                                 energy, energy-square and energy-flux
                                 moments, each in (0, 2); 0 takes the
                                 values of section 3 (1.1, 1.25, 1.8).  The
                                 stress moments relax at 1/tau (Eq. 8);
                                 ignored for BGK */
} ibm_lattice_desc;

typedef enum { IBM_BODY_FIXED = 0, IBM_BODY_PRESCRIBED = 1, IBM_BODY_FREE = 2 } ibm_body_kind;

/* A rigid body carrying markers.  FIXED: markers never move; their velocity
 * is u + omega x (X - xc) (e.g. a cylinder spinning in place).
 * PRESCRIBED: markers move rigidly with the constant (u, omega).
 * FREE: (u, omega) evolve by Eqs. 37-42 with the force and torque summed
 * from the corrections (Eq. 29), the internal-mass terms, the collision
 * force of Eq. 39 and the net weight M (1 - rho_f/rho_s) g. */
typedef struct {
  int kind;                   /* ibm_body_kind */
  double xc[2];               /* mass centre */
  double u[2];                /* translational velocity */
  double omega;               /* angular velocity (counter-clockwise) */
  double theta;               /* orientation angle */
  double rho_s, rho_f;        /* solid and fluid densities */
  double volume, inertia;     /* area V_s and moment of inertia I_s (2-D) */
  double radius;              /* collision radius for Eq. 39 */
  double gravity[2];          /* gravitational acceleration vector */
} ibm_body_desc;

/* Field selectors for ibm_read_fields / ibm_write_fields. */
enum {
  IBM_FIELD_RHO = 1,          /* [ny][nx] density of the last corrected state */
  IBM_FIELD_UX = 2,           /* [ny][nx] velocity x of the last corrected state */
  IBM_FIELD_UY = 3,           /* [ny][nx] velocity y of the last corrected state */
  IBM_FIELD_F = 4,            /* [9][ny][nx] post-stream populations (read/write) */
  IBM_FIELD_BODIES = 5,       /* [nbodies][9]: xc, yc, ux, uy, omega, theta, Fx, Fy, T */
  IBM_FIELD_RESIDUAL = 6,     /* [n_corr + 1]: r^0..r^N of the last step */
  IBM_FIELD_MARKERS = 7,      /* [nmarkers][2]: current marker positions */
  IBM_FIELD_MACRO_INIT = 8,   /* write only, [3][ny][nx] rho, ux, uy: f := f^eq(rho, u) */
  IBM_FIELD_BODY_STATE = 9    /* read/write, [nbodies][9]: xc, yc, ux, uy, omega, theta of the
                                 body (Eqs. 40-42) and its ux, uy, omega of the step before,
                                 which the internal-mass terms of Eqs. 37-38 use.  Writing it
                                 moves the body's markers rigidly to the new pose (marker
                                 velocities u + omega x r) and rebuilds the band before the
                                 next step; IBM_FIELD_F plus IBM_FIELD_BODY_STATE are a
                                 complete checkpoint: a lattice created with the same
                                 parameters and bodies and given both continues bit for bit
                                 with FP64 and FP32 storage (16-bit storage: to the storage
                                 rounding of the populations) */
};

/* Flags for ibm_step. */
enum {
  IBM_STEP_DEFAULT = 0,
  IBM_STEP_NO_GRAPH = 1,      /* launch kernel by kernel instead of replaying a CUDA graph */
  IBM_STEP_TIME_KERNELS = 2,  /* bracket each collide+stream launch with CUDA events */
  IBM_STEP_NO_MACRO = 4       /* do not write rho, u on the last step of the call */
};

/* Creates a lattice in the rest equilibrium f_i = w_i rho0 (Eq. 3 with
 * u = 0) on desc->device.  Returns IBM_ERR_INVALID for nx or ny < 4, tau
 * <= 0.5 or not finite, an unpaired periodic side, an inlet/outlet on an
 * unsupported side, n_corr < 0 or delta_points not 0, 2, 3, 4; IBM_ERR_NOMEM or
 * IBM_ERR_CUDA when device set-up fails.  *out is NULL on failure. */
ibm_status ibm_create_lattice(const ibm_lattice_desc *desc, ibm_handle *out);

/* Adds one rigid body and its n markers (section 2.2: the boundary is
 * discretised into Lagrangian points).  xy: 2n doubles, interleaved
 * (X0, Y0, X1, Y1, ...).  ds: n arc lengths per marker (Eq. 26), or NULL
 * for an equal share of the polygon perimeter through the markers.
 * body: its description; *body_id_out (optional) receives its index.
 * Markers whose 4 x 4 delta-function support leaves a non-periodic side,
 * or touches an inlet/outlet column, give IBM_ERR_INVALID. */
ibm_status ibm_add_markers(ibm_handle h, const double *xy, const double *ds,
                           int n, const ibm_body_desc *body, int *body_id_out);

/* Advances nsteps time steps.  One step: the N-iteration correction loop on
 * the post-stream state (Eqs. 22-28; residuals r^0..r^N recorded), body
 * force and torque (Eq. 29), the body update (Eqs. 37-42) and marker motion,
 * then the fused BGK collide + AA-pattern stream over every node.  Returns
 * once the steps are enqueued, except with corr_tol > 0: then it waits for
 * them and returns IBM_WARN_NOT_CONVERGED if any step since the last
 * synchronising call ended with r^N > corr_tol (or the error of a failed
 * step).  IBM_ERR_INVALID after a failed ibm_add_markers (destroy the
 * lattice). */
ibm_status ibm_step(ibm_handle h, int nsteps, unsigned flags);

/* Copies a field into host_dst (n_elems doubles, which must equal the
 * field's size) after synchronising the handle's stream.  The fields are the
 * moments of Eq. 7 of the last corrected pre-collision state (RHO, UX, UY),
 * the post-stream populations of Eq. 1 (F), the body state of Eqs. 41-42
 * with the force and torque of Eq. 29 and Eq. 38 of the last step (BODIES),
 * the no-slip residuals r^0..r^N of the correction loop of section 2.3
 * (RESIDUAL; returns IBM_WARN_NOT_CONVERGED when corr_tol > 0 and r^N is
 * above it), the marker positions X_l (MARKERS) and the body state needed to
 * resume a run (BODY_STATE).  Errors: IBM_ERR_INVALID
 * for an unknown field or a wrong n_elems, and the device errors of
 * ibm_sync. */
ibm_status ibm_read_fields(ibm_handle h, int field, double *host_dst, size_t n_elems);

/* Writes IBM_FIELD_F (raw post-stream populations of Eq. 1),
 * IBM_FIELD_MACRO_INIT (the equilibrium of Eq. 3 at the given rho, u) or
 * IBM_FIELD_BODY_STATE (the pose and velocities of Eqs. 40-42, see the field
 * list) from host_src, n_elems doubles, and synchronises the handle's
 * stream.  Errors: IBM_ERR_INVALID for a field that cannot be written, a
 * wrong n_elems or a non-finite value (and a density <= 0 for
 * MACRO_INIT), and the device errors of ibm_sync. */
ibm_status ibm_write_fields(ibm_handle h, int field, const double *host_src, size_t n_elems);

/* Blocks until the handle's queued work is done; reports device errors:
 * IBM_ERR_BOUNDS (a capacity check tripped: markers too dense),
 * IBM_ERR_TIMEOUT (a bounded grid-barrier wait ran out), IBM_ERR_DIVERGED
 * (a non-finite residual, or a NaN/Inf found by the watchdog), and the
 * warning IBM_WARN_NOT_CONVERGED (corr_tol > 0 and some step since the last
 * report ended with r^N above it; reported once). */
ibm_status ibm_sync(ibm_handle h);

/* Device time of the collide+stream launches bracketed since the last call
 * (IBM_STEP_TIME_KERNELS), in milliseconds, and their count; resets the
 * accumulators.  With markers the bracketed launch covers the band-free row
 * segments (see ibm_get_sizes).  Synchronises the stream. */
ibm_status ibm_kernel_times(ibm_handle h, double *ms_total, int *launches);

/* Sizes of the current state: nodes, markers, bodies, band nodes (distinct
 * nodes inside some marker support) and band segments (32-node row segments
 * holding a band node, which the correction kernel streams itself); any
 * pointer may be NULL. */
ibm_status ibm_get_sizes(ibm_handle h, long long *nodes, int *markers, int *bodies,
                         int *band_nodes, int *band_segments);

/* Counters since creation: CUDA kernels the library enqueued for ibm_step
 * (a CUDA-graph replay counts the kernels it contains) and time steps taken.
 * Either pointer may be NULL. */
ibm_status ibm_get_counters(ibm_handle h, long long *kernel_launches, long long *steps);

/* Prescribes the velocity U_l of Eq. 24 marker by marker: uv holds (u_x, u_y)
 * interleaved for all n markers of h (n must equal the marker count), in
 * the order they were added.  It applies to markers of FIXED bodies from
 * the next step on and stays until the next call -- a time-dependent
 * boundary (e.g. the Taylor-Green case of section 3.1.1, Eq. 30) calls it
 * before every step.  Markers of moving bodies keep taking their velocity
 * from the body motion; adding markers resets every marker to its body's
 * u + omega x (X - xc).  The array is copied before the call returns.
 * Errors: IBM_ERR_INVALID for NULL, a wrong n or a non-finite value. */
ibm_status ibm_set_marker_velocities(ibm_handle h, const double *uv, int n);

/* Tuning options for ibm_set_option. */
enum {
  IBM_OPT_IB_CTAS = 1,  /* CTAs of the correction kernel: 0 (default) = one CTA for up to 512
                           markers, 3 per 4 SMs above that; n > 0 = min(n, SMs).  2..16 CTAs
                           run as one thread-block cluster when the device can schedule it.
                           Results do not depend on it. */
  IBM_OPT_IB_THREADS = 2, /* threads per correction-kernel CTA: 256 (default), 512 or 1024 */
  IBM_OPT_WATCHDOG_STEPS = 3, /* K > 0: after every K steps (at the next 8-step block boundary)
                           scan every stored population for NaN/Inf; a hit makes the next
                           synchronising call return IBM_ERR_DIVERGED.  0 (default): no scan.
                           Independently of it, a non-finite no-slip residual r^N is
                           detected by the correction kernel every step. */
  IBM_OPT_BARRIER_LIMIT_US = 4, /* wait limit of the correction kernel's global-memory grid
                           barrier in microseconds, [100, 6e7] (default 2 s); a wait that runs
                           out makes the next synchronising call return IBM_ERR_TIMEOUT */
  IBM_OPT_IB_PHASES = 6,     /* how the correction loop of section 2.3 is launched.  0 (default):
                           one persistent kernel with a grid barrier between phases.  1: a chain
                           of short kernels, one per phase (band gather, interpolation, each
                           Jacobi iteration, final residual and history, second moments),
                           ordered by the stream; their CTAs leave the SMs as soon as their
                           share is done.  2: gather and interpolation in one persistent kernel,
                           the Jacobi iterations in one thread-block cluster (up to 16 CTAs)
                           holding A^n in distributed shared memory, history and moments in a
                           second persistent kernel; boundaries of at most 512 markers, or a
                           device that cannot schedule the cluster, keep mode 0.  Results do
                           not depend on it (bit for bit). */
  IBM_OPT_TEST_DROP_ARRIVAL = 5 /* testing the timeout path only: 1 makes the last CTA of the
                           correction kernel skip its arrival at the first grid barrier of each
                           step, so the other CTAs' waits run out (bounded by
                           IBM_OPT_BARRIER_LIMIT_US).  Only grids that wait at the
                           global-memory barrier (more than 16 CTAs) are affected.  The
                           lattice's results are then wrong; destroy it afterwards. */
};

/* Chooses the correction kernel's CTA count by measurement: for each of the
 * n candidates (CTA counts as for IBM_OPT_IB_CTAS; NULL or n == 0: a default
 * set around the SM count) the lattice takes steps_each ordinary time steps,
 * timed with CUDA events on its stream; the fastest count is then set and
 * written to *best (optional), its time per step to *best_us (optional).
 * The steps are real steps of the simulation (n * steps_each of them;
 * results do not depend on the CTA count, so the trajectory is the one any
 * single setting would give).  Synchronises the lattice's stream.  No
 * counterpart in the paper: it is a deployment aid.  Errors: IBM_ERR_INVALID
 * for steps_each < 2 or a negative candidate. */
ibm_status ibm_autotune_ib(ibm_handle h, const int *candidates, int n, int steps_each, int *best,
                           double *best_us);

/* Sets a tuning option of h (takes effect at the next step).  Concurrency
 * note: a correction kernel of more than 16 CTAs (the default for more than
 * 512 markers) waits at a grid barrier in global memory and needs all its
 * CTAs resident at once; step at most two such lattices at once on one GPU
 * (the server below keeps a budget).  Grids of 2..16 CTAs run as one
 * thread-block cluster, which the hardware schedules as a whole. */
ibm_status ibm_set_option(ibm_handle h, int option, long long value);

/* Frees every device and host resource of h (NULL is a no-op): the
 * populations of Eq. 1, the marker and band arrays of the correction loop
 * (section 2.3) and the body records of Eqs. 37-42.  Synchronises the
 * handle's stream first; returns IBM_ERR_CUDA when that reports an error
 * (the resources are freed all the same). */
ibm_status ibm_destroy(ibm_handle h);

/* Message for the last failure on h (thread-local for h == NULL). */
const char *ibm_last_error(ibm_handle h);

/* Optional process-wide device allocator used for every later allocation:
 * alloc(bytes, device, stream, ctx) returns a device pointer or NULL;
 * release(ptr, device, stream, ctx) frees it.  Pass NULLs to go back to
 * cudaMalloc / cudaFree.  Not thread-safe with concurrent handle creation. */
typedef void *(*ibm_alloc_fn)(size_t bytes, int device, void *stream, void *ctx);
typedef void (*ibm_free_fn)(void *ptr, int device, void *stream, void *ctx);
ibm_status ibm_set_allocator(ibm_alloc_fn alloc, ibm_free_fn release, void *ctx);

/* ------------------------------------------------------------------ serving
 * A server keeps many independent cases resident on one GPU and runs them
 * concurrently (continuous batching; the paper has no counterpart, this is
 * the deployment layer around ibm_step).  Submitted cases wait in a FIFO
 * and are admitted while the device-memory budget, the slot count and the
 * correction-kernel CTA budget allow; each admitted case gets its own
 * lattice and stream and is advanced in chunks of steps (CUDA-graph
 * replays), so kernels of different cases overlap on the device.  When a
 * case has taken its steps, its requested outputs are copied to host
 * memory, its device memory is released and the next waiting case is
 * admitted.  A case's results do not depend on what else runs with it. */
typedef struct ibm_server_s *ibm_server;

typedef struct {
  int device;
  double max_device_bytes;    /* budget for resident cases; <= 0: 80% of free memory */
  int max_active;             /* resident cases at once (slots), >= 1 */
  int steps_per_launch;       /* steps enqueued per case per round, >= 1 */
  int ib_cta_budget;          /* sum of the CTAs of resident cases whose correction
                                 kernel waits at a global-memory grid barrier (a
                                 grid the device cannot schedule as one cluster);
                                 <= 0: 2 per SM */
  int ib_markers_per_cta;     /* a case with M markers runs its correction loop on
                                 ceil(M / this) CTAs, at most 16 (one thread-block
                                 cluster; one CTA when M <= this); <= 0: 512 */
  int batched;                /* 0: each resident case is stepped by its own graph
                                 launches on its own stream; 1: one persistent kernel per
                                 round of steps_per_launch steps advances every resident
                                 case (FP32 and 16-bit storage; FP64 cases are refused):
                                 its CTAs take each step's correction tasks and
                                 collide+stream tiles of all cases from one work queue */
  int tile_nodes;             /* batched: lattice nodes per collide+stream tile (whole
                                 rows, at least one); <= 0: 32768 */
  int corr_first;             /* batched: order of a step's tasks in the queue.  1 or <= 0
                                 (default): the correction tasks of every case, then all
                                 tiles; 2: case by case, its correction tasks then its tiles */
} ibm_server_desc;

enum { IBM_OUT_MACRO = 1, IBM_OUT_BODIES = 2, IBM_OUT_RESIDUAL = 4 };

typedef struct {
  ibm_lattice_desc lattice;   /* cuda_stream and device are set by the server */
  int nbodies;
  const ibm_body_desc *bodies;
  const int *nmarkers;        /* markers per body */
  const double *xy;           /* all markers, interleaved, body after body */
  const double *ds;           /* arc lengths of all markers, or NULL */
  int nsteps;                 /* time steps of the case */
  unsigned outputs;           /* IBM_OUT_* */
} ibm_case_desc;

typedef struct {
  long long submitted, completed, active, pending, failed;
  double p50_ms, p95_ms, p99_ms, mean_ms;  /* time to solution: submission to results in host memory */
  double solves_per_s;        /* completed / (last completion - first submission) */
  double mlups;               /* lattice updates of completed cases over the same interval */
  double device_bytes;        /* estimated device memory of resident cases */
  double host_admit_s;        /* host seconds spent admitting cases (lattice set-up) */
  double host_launch_s;       /* host seconds spent enqueuing chunks */
  double host_harvest_s;      /* host seconds spent copying results out */
} ibm_server_stats;

ibm_status ibm_server_create(const ibm_server_desc *desc, ibm_server *out);
/* Copies the case; *case_id receives its id.  Never blocks on the GPU. */
ibm_status ibm_server_submit(ibm_server s, const ibm_case_desc *c, long long *case_id);
/* Harvests finished chunks, launches next chunks, admits waiting cases;
 * *completed (optional) receives the number of cases finished by this call.
 * Never blocks on the GPU. */
ibm_status ibm_server_progress(ibm_server s, int *completed);
/* Runs progress until the case (case_id >= 0) or every case (case_id < 0)
 * is finished. */
ibm_status ibm_server_wait(ibm_server s, long long case_id);
/* Outputs of a finished case: IBM_FIELD_RHO / UX / UY ([ny][nx]),
 * IBM_FIELD_BODIES ([nbodies][9]) or IBM_FIELD_RESIDUAL ([n_corr + 1]) of its
 * last step, if requested at submission.  Returns the case's own failure
 * status if it failed. */
ibm_status ibm_server_result(ibm_server s, long long case_id, int field, double *host_dst, size_t n_elems);
ibm_status ibm_server_release(ibm_server s, long long case_id);   /* drops stored results */
ibm_status ibm_server_get_stats(ibm_server s, ibm_server_stats *out);
/* Batched mode's autotuner (no counterpart in the paper): on an idle server,
 * runs the n sample cases for every combination of the candidate tile sizes
 * (nodes per collide+stream tile), markers per correction CTA and task
 * orders (1 and 2, see corr_first), times each run (all samples submitted
 * at once, wall clock to the last result), keeps the fastest setting and
 * returns it.  The sample runs do not enter the server's statistics.  NULL
 * or empty candidate lists take defaults (tiles 8192, 16384, 32768, 65536;
 * markers per CTA 256, 512, 1024).  Errors: IBM_ERR_INVALID when the server
 * is not batched or not idle, or a sample is invalid; a failed sample run's
 * status otherwise. */
ibm_status ibm_server_autotune(ibm_server s, const ibm_case_desc *samples, int n, const int *tile_nodes,
                               int n_tiles, const int *markers_per_cta, int n_mpc, int *best_tile_nodes,
                               int *best_markers_per_cta, int *best_corr_first, double *best_seconds);
ibm_status ibm_server_destroy(ibm_server s);
const char *ibm_server_last_error(ibm_server s);

/* The correction loop of one step for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is a deployment variant of the
 * correction loop that ibm_step runs.  It is meant for code that may not call
 * cudaMalloc -- code running inside another framework's memory pool or
 * under a fixed device-memory budget, plug-ins that may only use the buffers
 * handed to them, or paths where an allocation could fail or block at a
 * point where the caller cannot recover.
 *
 * The caller passes every input and output as device memory it owns:
 *   f          [9][ny][nx] post-stream populations (double for IBM_FP64,
 *              float for IBM_FP32), corrected in place by the N-iteration
 *              correction loop of ibm_step (no collision, no streaming); the
 *              lattice is periodic in x and y;
 *   xy, ds     2n interleaved marker positions and n arc lengths (double);
 *   uvel       2n interleaved marker velocities (double);
 *   resid_out  n_corr + 1 doubles, the residuals r^0 .. r^N (may be NULL);
 *   force_out  2 doubles, the force on all markers together (may be NULL).
 * The work runs on cuda_stream (NULL: the legacy default stream) on the
 * current device as one CTA per kernel, and the call returns after
 * synchronising that stream, so it cannot be captured into a CUDA graph.  On entry it clears the calling thread's
 * pending CUDA launch error (left by earlier work), so that it reports only
 * errors of its own work.  When the call fails, the contents of f, resid_out
 * and force_out are undefined.
 *
 * Nothing is allocated: every intermediate array lives in one fixed 8 MiB
 * device array that the library reserves when it is loaded and that every
 * GPU using the library keeps until the process exits.  Limits:
 * nx * ny <= 262144, 1 <= n <= 512 markers, 0 <= n_corr <= 64; larger
 * requests return IBM_ERR_INVALID with a message in ibm_last_error(NULL).
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress).  All calls share the array and it keeps the last call's contents
 * (the call clears what must start empty); calls that overlap on the GPU --
 * from several host threads or streams at once -- race and give wrong
 * results. */
ibm_status ibm_ib_correct_noalloc(int nx, int ny, int prec, void *f, int n_markers, const double *xy,
                                  const double *ds, const double *uvel, int n_corr, double *resid_out,
                                  double *force_out, void *cuda_stream);

/* ABI version the library was built with (IBM_ABI_VERSION). */
int ibm_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* IBM_H_ */
