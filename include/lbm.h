/*
 * lbm.h -- C ABI of the GB300 two-phase colour-gradient lattice Boltzmann library.
 *
 * The library advances D2Q9 two-phase colour-gradient LBM simulations
 * (arXiv 1903.01168, Sec. 2) on one NVIDIA GB300 (sm_103a) with hand-written
 * CUDA kernels.  One time step applies, per node and per colour k in {red,
 * blue}:
 *   1. collision, Eq. (eq:singleCollision) (BGK) or Eq. (eq:singleCollisionMRT)
 *      (MRT), towards Eq. (eq:equilibrium) or the Hermite equilibrium
 *      Eq. (eq:equilibrium_hermite) (+ the source U^k = M^-1 C^k under MRT),
 *      with the interpolated relaxation rate omega_eff(psi) of Sec. 2.1 and a
 *      Guo body force F^k = rho_k g;
 *   2. the surface-tension perturbation, Eq. (eq:perturbation), driven by the
 *      S2I4 colour gradient F of Eq. (eq:colorGradient), A = 9 sigma omega_eff / 4
 *      (Eq. (eq:sigmaIsoAllen));
 *   3. recolouring, Eq. (eq:recoloringOperator);
 *   4. streaming, Eq. (eq:subop4), with periodic ends, halfway bounce-back
 *      walls and the two-phase Zou-He velocity inlet / pressure outlet of
 *      Sec. 2.5 (rotated to a west inlet and an east outlet).
 *
 * Conventions
 *   - Lattice nx * ny nodes; host field arrays are double, nx*ny values,
 *     x fastest (index y*nx + x).
 *   - Colour red (k = 0) is the heavy phase with reference density
 *     rho_r^0 = gamma, blue (k = 1) the light one with rho_b^0 = 1; the colour
 *     field psi is +1 in pure red, -1 in pure blue (Eq. (eq:color_field)).
 *   - Velocities u include the Guo half-force shift: u = (sum N c + rho g/2)/rho.
 *   - Pressure p = sum_k rho_k (c_s^k)^2 with (c_s^k)^2 = 3 (1 - alpha_k)/5
 *     (Eq. (eq:pressureRelation)).
 *   - Every call returns an lbm_status; nothing throws across the ABI.  On
 *     failure lbm_last_error() returns a message for that simulation.
 *   - One simulation is driven by one host thread at a time.  lbm_step and
 *     lbm_batch_step are asynchronous on the simulation's CUDA stream; the
 *     read / diagnostic / state calls synchronise that stream.
 *   - Device memory is owned by the library (lbm_create) or by the caller
 *     (lbm_create_ex, e.g. a torch tensor), who must keep it alive until
 *     lbm_destroy.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = -1,     /* invalid argument or parameter combination */
    LBM_ENOMEM = -2,     /* device or host allocation failed / buffer too small */
    LBM_ECUDA = -3,      /* a CUDA runtime or driver call failed */
    LBM_EUNSTABLE = -4,  /* non-finite values found by lbm_diagnostics */
    LBM_ETIMEOUT = -5,   /* a bounded device-side wait gave up */
    LBM_EBUDGET = -6     /* request exceeds a memory budget */
} lbm_status;

typedef enum { LBM_BGK = 0, LBM_MRT = 1 } lbm_collision;
typedef enum { LBM_EQ_STD = 0, LBM_EQ_HERMITE = 1 } lbm_equilibrium;
/* Population storage (arithmetic is FP32 in every case).  The state holds per
 * node the colour densities rho_r, rho_b (FP32) and the deviations
 * d^k_i = N^k_i - phi^k_i rho_k of the post-collision populations from the rest
 * state of the node's own colour densities (i = 1..8).
 *   F32     deviations in FP32: 144 bytes read + written per node update.
 *   F16DEV  deviations in FP16 and BF16DEV in BF16, in a split form.  The
 *   BF16DEV recolouring shift and flux that dominate d^k_i at an interface
 *           (Eq. (eq:recoloringOperator)) are rebuilt from three FP32 node
 *           scalars (rho_r rho_b / rho and the flux vector), and only the small
 *           colour-blind remainder is rounded to 16 bits: 104 bytes per update. */
typedef enum { LBM_F32 = 0, LBM_F16DEV = 1, LBM_BF16DEV = 2 } lbm_storage;
/* bc_x: PERIODIC or INOUT; bc_y: PERIODIC or WALL. */
typedef enum { LBM_BC_PERIODIC = 0, LBM_BC_WALL = 1, LBM_BC_INOUT = 2 } lbm_bc;
typedef enum { LBM_INLET_ALTERNATE = 0, LBM_INLET_LAYERED = 1 } lbm_inlet_mode;
/* Kernel choice: the fused single-pass kernel (default) or the two-pass
 * reference kernel pair (moments pass + collide pass, with a scratch field). */
typedef enum { LBM_KERNEL_AUTO = 0, LBM_KERNEL_FUSED = 1, LBM_KERNEL_TWOPASS = 2 } lbm_kernel;

/* How the strip rows of a launch are shared among thread blocks.  Every plan
 * gives the same results; only the speed differs. */
typedef enum {
    LBM_PLAN_AUTO = 0,      /* SPLIT when there are no more 128-column strips than
                               resident blocks, else BALANCED (the default) */
    LBM_PLAN_BALANCED = 1,  /* equal shares of row cost; a block may march over
                               several segments */
    LBM_PLAN_SPLIT = 2      /* one segment per block, the costliest segment as cheap
                               as the block count allows */
} lbm_plan_kind;

typedef struct {
    double gamma;        /* density ratio rho_r^0 / rho_b^0 >= 1 (Eq. (eq:gammaAlphaBeta)) */
    double alpha_b;      /* rest fraction of blue, 0 < alpha_b < 1 (paper: 0.2); alpha_r =
                            1 - (1 - alpha_b)/gamma */
    double tau_r, tau_b; /* relaxation times, omega_k = 1/tau_k; kinematic viscosity
                            nu_k = (tau_k - 1/2)/3 with the standard equilibrium (Sec. 2.1),
                            nu_k = (c_s^k)^2 (tau_k - 1/2) with the Hermite one */
    double delta;        /* omega_eff interpolation half-width (paper: 0.1) */
    double sigma;        /* surface tension (lattice units) */
    double beta;         /* recolouring parameter in [0, 1] (paper default 0.99) */
    double gx, gy;       /* body acceleration g (Guo forcing, F^k = rho_k g) */
    int collision;       /* lbm_collision */
    int equilibrium;     /* lbm_equilibrium; HERMITE adds U^k when collision == MRT */
    double mrt_lambda;   /* s_0..s_6 = lambda omega_eff, s_7 = s_8 = omega_eff (paper: 4/5) */
    double c7_sign;      /* sign of the d_y Q_y term of C^k_7: -1 (default) from the
                            Chapman-Enskog expansion, +1 as the paper prints it */
    double c7_factor;    /* factor of C^k_7: 1 (default) from the expansion, 3 as printed.
                            C^k_7 = c7_factor (1 - omega_eff/2)(d_x Q_x + c7_sign d_y Q_y)
                            (Sec. 2.1, "Proper recovery of Navier-Stokes equations") */
    int bc_x;            /* LBM_BC_PERIODIC or LBM_BC_INOUT */
    int bc_y;            /* LBM_BC_PERIODIC or LBM_BC_WALL */
    int storage;         /* lbm_storage */
    double u_in_r, u_in_b; /* inlet speed of the red / blue phase (bc_x == INOUT) */
    double p_out;        /* outlet pressure (bc_x == INOUT) */
    int inlet_mode;      /* lbm_inlet_mode */
    int inlet_period_r, inlet_period_b; /* ALTERNATE: steps of red, then blue injection */
    int inlet_layer;     /* LAYERED: rows y < inlet_layer inject red, the rest blue */
    int kernel;          /* lbm_kernel */
    int plan_rows;       /* fused kernel work plan: fewest rows of this lattice a thread
                            block marches over in one segment (0 = 8), alone or in a
                            batch; larger values trade parallelism for less halo
                            re-reading.  Never changes results, only speed (the
                            Python autotuner picks it per lattice size class). */
    int plan;            /* lbm_plan_kind of this lattice's own launches (0 = AUTO) */
    int wall_slip;       /* walls (bc_y = WALL): 0 no slip (halfway bounce-back), 1 free
                            slip: diagonal populations travel on along the wall,
                            mirrored (Sec. 2.5 "Boundary conditions").  Free slip and a
                            contact angle (below) select the wetting variant of the step
                            kernels (fused or two-pass, alone or in a batch); the
                            no-slip variant keeps fewer registers */
    double contact_angle;/* static contact angle on the walls, radians in (0, pi), measured
                            through the blue phase; 0 = no adjustment.  On the fluid rows
                            next to a wall the colour gradient is turned to the closer of
                            the two normals at this angle from the wall normal (Sec.
                            "Adjustment of the color gradient for static contact angles") */
} lbm_params;

/* FP64 diagnostics of the state at the current time t (sums over all nodes). */
typedef struct {
    long long t;          /* time step of the state */
    double mass_r, mass_b;/* sum rho_r, sum rho_b */
    double mom_x, mom_y;  /* sum rho u */
    double max_u;         /* max |u| */
    double area_b;        /* sum (1 - psi)/2: light-phase area */
    double cx_b, cy_b;    /* light-phase centroid (area-weighted, unwrapped coordinates) */
    double ux_b, ux_r;    /* area-weighted mean x-velocity of the light / heavy phase */
    double r_eff;         /* sqrt(area_b / pi) */
    double p_in, p_out;   /* mean p over r < r_eff/2 and over r > r_eff + 8 around the
                             bubble centre given to lbm_init_bubble (else the centroid) */
    double dp;            /* p_in - p_out (Laplace pressure jump) */
    long long nonfinite;  /* nodes with a non-finite density or velocity */
} lbm_diag;

/* Geometry of a train of light bubbles moving along x (the slug measurements of
 * Sec. 5.1: bubble and slug lengths, the liquid film between a bubble and the
 * walls, the bubble nose).  Measured on the colour field psi of the state:
 *   - the centreline profile psi_c(x): psi on the middle row, or the mean of the
 *     two middle rows when ny is even, taken linear between nodes;
 *   - a bubble's tail is a centreline zero of psi_c where it goes from >= 0
 *     (heavy) to < 0 (light) in +x, its nose the next zero from < 0 to >= 0;
 *   - the light thickness of a column, g(x) = sum_y (1 - psi(x, y)) / 2, taken
 *     linear between columns; a bubble's film thickness is (ny - g(x_mid)) / 2 at
 *     its middle x_mid = (tail + nose) / 2.
 * Periodic x closes the line (a bubble may straddle x = 0); on an open x axis
 * only bubbles with both ends inside count, and a slug needs a bubble on both
 * sides. */
#define LBM_SLUG_MAX 16
typedef struct {
    long long t;          /* time step of the state */
    int n_bubbles;        /* bubbles cut by the centreline (all of them count in the
                             means; the first LBM_SLUG_MAX are listed) */
    int n_slugs;          /* liquid slugs between two counted bubbles */
    double bubble_len;    /* mean bubble length nose - tail on the centreline */
    double slug_len;      /* mean slug length (next tail - nose) on the centreline */
    double film;          /* mean film thickness at the bubbles' middles */
    double x_tail[LBM_SLUG_MAX], x_nose[LBM_SLUG_MAX]; /* in [0, nx), ordered in x by tail */
} lbm_slug;

typedef struct lbm_sim lbm_sim;
typedef struct lbm_batch lbm_batch;

/* Fill *p with the paper's defaults: gamma 1, alpha_b 0.2, tau 1, delta 0.1,
 * sigma 0.005, beta 0.99, BGK, standard equilibrium, lambda 4/5, periodic. */
lbm_status lbm_default_params(lbm_params *p);

/* Device bytes one simulation needs (both population buffers).  0 on invalid
 * arguments. */
size_t lbm_bytes_required(int nx, int ny, const lbm_params *p);

/* Create a simulation of nx * ny nodes (nx >= 8, ny >= 4) on the current CUDA
 * device, allocating its population buffers and a private stream.  The state
 * is zero until an init call. */
lbm_status lbm_create(int nx, int ny, const lbm_params *p, lbm_sim **out);

/* As lbm_create, on caller-owned device memory dev_buf of at least
 * lbm_bytes_required() bytes (256-byte aligned) and the caller's stream
 * (cudaStream_t, may be NULL for the legacy default stream). */
lbm_status lbm_create_ex(int nx, int ny, const lbm_params *p, void *dev_buf, size_t bytes,
                         void *cuda_stream, lbm_sim **out);

/* Sharp-interface static bubble at rest: light phase (rho_b = 1) where the
 * periodic distance to (cx, cy) is below R, heavy phase (rho_r = gamma)
 * elsewhere; equilibrium populations; t = 0. */
lbm_status lbm_init_bubble(lbm_sim *s, double cx, double cy, double R);

/* Periodic slug train: n_bubbles evenly spaced light stadium bubbles of length
 * bubble_len and height bubble_h centred in y, heavy liquid elsewhere; with
 * poiseuille != 0 the start velocity is u_x(y) = gx/(2 nu_r) Y (ny - Y),
 * Y = y + 1/2 (Sec. 5.1); t = 0. */
lbm_status lbm_init_slug(lbm_sim *s, int n_bubbles, double bubble_len, double bubble_h,
                         int poiseuille);

/* Equilibrium state from host fields rho_r, rho_b, ux, uy (nx*ny doubles each);
 * t = 0. */
lbm_status lbm_init_fields(lbm_sim *s, const double *rho_r, const double *rho_b,
                           const double *ux, const double *uy);

/* State from host pre-collision populations N^k_i(x, y) (Eq. (eq:evolution)):
 * 18*nx*ny doubles laid out [k = red, blue][i = 0..8][y][x], directions in the
 * order 0 rest, 1 E, 2 N, 3 W, 4 S, 5 NE, 6 NW, 7 SW, 8 SE; t = 0.  On an open
 * (inlet / outlet) column the populations entering from outside are replaced by
 * the Zou-He values when the state is first read. */
lbm_status lbm_init_populations(lbm_sim *s, const double *pops);

/* Advance n >= 0 time steps (asynchronous on the simulation's stream). */
lbm_status lbm_step(lbm_sim *s, long n);

/* Stop the simulation at time t_end (t_end >= current time; t_end < 0 removes
 * the stop): steps that would start at t >= t_end leave the state unchanged, so
 * lbm_step / lbm_batch_step may run past it and the state stays at t_end.
 * Batches created before the call keep the previous stop time.  Synchronous. */
lbm_status lbm_set_stop(lbm_sim *s, long long t_end);

/* Block until the simulation's queued work is done; reports CUDA errors. */
lbm_status lbm_synchronize(lbm_sim *s);

/* Current time step. */
long long lbm_time(const lbm_sim *s);

/* Macroscopic fields at the current time into caller-owned host arrays of
 * nx*ny doubles (x fastest); any pointer may be NULL.  Synchronous. */
lbm_status lbm_read_fields(lbm_sim *s, double *rho_r, double *rho_b, double *ux, double *uy,
                           double *p);

/* Pre-collision populations N^k_i at the current time into a caller-owned host
 * array of 18*nx*ny doubles, in the layout of lbm_init_populations (boundary
 * conditions applied).  Synchronous. */
lbm_status lbm_read_populations(lbm_sim *s, double *pops);

/* FP64 diagnostics of the current state.  Returns LBM_EUNSTABLE (with *out
 * filled) if any node is non-finite.  Synchronous. */
lbm_status lbm_diagnostics(lbm_sim *s, lbm_diag *out);

/* Slug-train geometry of the current state (lbm_slug above), computed from an
 * FP64 per-column profile that a kernel reduces on the device.  gas: NULL, or a
 * caller-owned host array of nx doubles that receives g(x) (the light thickness
 * of each column; behind a nose, g(x_nose - s) is the nose shape).  Synchronous. */
lbm_status lbm_slug_geometry(lbm_sim *s, lbm_slug *out, double *gas);

/* Raw state (both population buffers and the time step): size, save to a
 * host buffer, restore from one.  Synchronous.  A restored state continues
 * bit-identically. */
size_t lbm_state_bytes(const lbm_sim *s);
lbm_status lbm_save_state(lbm_sim *s, void *host, size_t bytes);
lbm_status lbm_load_state(lbm_sim *s, const void *host, size_t bytes);

/* Message of the last failed call on s (or of the last failed create when s is
 * NULL); never NULL. */
const char *lbm_last_error(const lbm_sim *s);

/* Free the simulation (its own buffers and stream; never caller memory). */
void lbm_destroy(lbm_sim *s);

/* ---- allocation-free stepping ---- */

/* Advance n >= 0 steps of a simulation whose state lives in caller-owned device
 * memory, allocating nothing: no cudaMalloc, cudaMallocAsync, cudaFree or
 * allocating library routine is called.  The paper has no counterpart; this is
 * for callers that cannot allocate device memory themselves at run time (an
 * embedding runtime whose allocator owns the GPU, a fixed pre-registered memory
 * pool, an allocation-free real-time loop).
 *   p, nx, ny    parameters and lattice, as for lbm_create (p->kernel is ignored:
 *                the two-pass kernels run); nx * ny <= 262144
 *   state        device buffer of lbm_bytes_required(nx, ny, p) bytes, 256-byte
 *                aligned, holding the state at time t in the layout of
 *                lbm_save_state (its bytes after the leading time stamp); it is
 *                advanced in place (the state at t + n ends in the same buffer)
 *   t            time step of the state in `state`
 *   cuda_stream  stream the kernels are queued on (asynchronous)
 * The intermediate colour-field pass uses a static scratch array of 5 MiB, and
 * the kernels read the simulation's descriptor from a static slot beside it;
 * every GPU loading the library holds both until exit.  Their device addresses
 * are looked up by the first call made on each device, with that device
 * current; make that first call before capturing any stream.  Each call copies
 * the descriptor into its slot on `cuda_stream` (no allocation).  All calls
 * share the scratch and the slot, which keep the previous call's contents:
 * calls that may overlap on the GPU (different streams, or different
 * simulations on one stream that are not ordered) race, so order them.
 * Errors (message in lbm_last_error(NULL)):
 *   LBM_EINVAL  invalid parameters, more than 262144 nodes, a state pointer that
 *               is not device (or managed) memory of the current device, or a
 *               misaligned state; LBM_ENOMEM  `bytes` too small;
 *   LBM_ECUDA   a CUDA error left pending by earlier work (reported, and cleared,
 *               before anything is queued), or a failed copy or launch. */
lbm_status lbm_step_noalloc(const lbm_params *p, int nx, int ny, void *state, size_t bytes, long long t,
                            long n, void *cuda_stream);

/* ---- batched stepping of many independent simulations ---- */

/* Group n simulations (created on the same device, any sizes and parameters,
 * FP32 or 16-bit storage) so that lbm_batch_step advances all of them with one
 * kernel launch per time step and storage / collision type (types run
 * concurrently on streams of the batch, joined into the stream of sims[0]).
 * rows_per_item > 0 cuts every strip into pieces of that many rows, one per
 * thread block; 0 shares the rows of all members among the resident thread
 * blocks (LBM_PLAN_AUTO of lbm_batch_create_ex), no segment of a member shorter
 * than its plan_rows.
 * The simulations stay owned by the caller and must outlive the batch. */
lbm_status lbm_batch_create(lbm_sim *const *sims, int n, int rows_per_item, lbm_batch **out);


/* Work-plan options of a batch. */
typedef struct {
    int rows_per_item;   /* > 0: fixed plan, as in lbm_batch_create (plan is ignored) */
    float row_overhead;  /* cost of one strip row = the warps it keeps busy (1..4) +
                            row_overhead; < 0 selects the library default (1) */
    int plan;            /* lbm_plan_kind */
    const int *member_plan_rows; /* NULL, or n values (>= 0, 0 = 8) used instead of each
                            member's own plan_rows; read during the call only */
} lbm_batch_opts;

/* lbm_batch_create with explicit plan options (opts must not be NULL).
 * LBM_EINVAL for rows_per_item < 0, row_overhead > 64, an unknown plan or a
 * member_plan_rows value out of range. */
lbm_status lbm_batch_create_ex(lbm_sim *const *sims, int n, const lbm_batch_opts *opts, lbm_batch **out);

/* Host only (no device call): the work plan a batch of n lattices of sizes
 * nx[i] x ny[i] would get with these options and max_blocks resident thread
 * blocks (the library queries that number from the device; pass any positive
 * value here).  plan_rows: NULL or the members' plan_rows (opts->member_plan_rows
 * takes precedence).  Sets *n_items and *n_blocks and writes the first
 * `capacity` items as 6 ints each: member, first column, width (<= 128), first
 * row, end row, thread block.  Items of one block are listed in the order the
 * block runs them.  LBM_EINVAL for invalid sizes or options. */
lbm_status lbm_plan_preview(const int *nx, const int *ny, const int *plan_rows, int n, const lbm_batch_opts *opts,
                            int max_blocks, int *n_items, int *n_blocks, int *items, int capacity);

/* Advance every simulation of the batch by n steps; with use_graph != 0 the
 * launches are captured once into a CUDA graph of n steps and replayed on
 * later calls with the same n. Asynchronous. */
lbm_status lbm_batch_step(lbm_batch *b, long n, int use_graph);

/* Number of work items (thread blocks) of one batched step. */
int lbm_batch_items(const lbm_batch *b);

void lbm_batch_destroy(lbm_batch *b);

#ifdef __cplusplus
}
#endif
#endif
