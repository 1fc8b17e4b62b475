/*
 * lsgg.h -- C ABI of the GB300 (sm_103a) local level-set grain-growth library.
 *
 * Method: C. Miessen, N. Velinov, G. Gottstein, L.A. Barrales-Mora, "A highly
 * efficient 3D level-set grain growth algorithm tailored for ccNUMA
 * architecture", arXiv:1701.06658.  Each grain i carries its own level-set
 * function phi_i on a local box Omega_i (its bounding box plus a halo,
 * Sec. 2.1.3, Fig. 1); one time step is Algorithm 1's loop body:
 *   predictor     phi_p = G(dt) * phi           (Eqs. (7)-(9); Eq. (10) with physics)
 *   corrector     phi_c = (phi_p - max_{j!=i} phi_p_j) / 2        (Eq. (16))
 *   re-init       taxicab signed distance to the zero level        (Sec. 2.1.6)
 *   box update    bbox{phi > 0} + halo, neighbour data              (Secs. 2.1.3, 3.1)
 *
 * Units: grid units (cell spacing h = 1, M_max * gamma_max = 1).  The domain is
 * periodic, nx * ny * nz cells, x fastest; nz == 1 is a 2D domain.
 *
 * Conventions for every function below:
 *   - return LSGG_OK (0) on success, a negative LSGG_ERR_* code otherwise;
 *     lsgg_status_string() names it.  No function throws or aborts.
 *   - host pointers are caller-owned; the library copies what it needs and
 *     keeps no host pointer after the call returns.
 *   - a context owns all of its device memory; lsgg_destroy frees it.
 *   - a context is not thread-safe; distinct contexts are independent.
 *   - every device computation runs in the library's CUDA kernels; there is
 *     no CPU fallback.  Without a usable CUDA device, calls that compute
 *     return LSGG_ERR_CUDA.
 */
#ifndef LSGG_H
#define LSGG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define LSGG_OK                 0
#define LSGG_ERR_INVALID_ARG   -1   /* a size, pointer or config field is out of range */
#define LSGG_ERR_OUT_OF_MEMORY -2   /* a device allocation failed */
#define LSGG_ERR_OVER_BUDGET   -3   /* a server admission would exceed its HBM budget */
#define LSGG_ERR_CUDA          -4   /* a CUDA runtime call failed (no device, launch error); with
                                       LSGG_TRACE_ERRORS set in the environment the runtime's
                                       message is printed on stderr */
#define LSGG_ERR_TIMEOUT       -5   /* a bounded wait expired (device queue or host wait) */
#define LSGG_ERR_NOT_READY     -6   /* a served request has not finished yet */
#define LSGG_ERR_CAPACITY      -7   /* a caller buffer (see *n_out) or a fixed library buffer is too small */
#define LSGG_ERR_UNSUPPORTED   -8   /* a requested variant is not built */

/* ---------------------------------------------------------------- config */
#define LSGG_INIT_VORONOI   0   /* Voronoi tessellation of the seeds */
#define LSGG_INIT_LAGUERRE  1   /* power diagram: seeds plus weights */
#define LSGG_INIT_LABELS    2   /* a label field: every cell's grain id (a tessellation read from a file) */

#define LSGG_PHYSICS_IDEAL          0  /* w = 1, no bulk term: phi_p = G * phi */
#define LSGG_PHYSICS_READ_SHOCKLEY  1  /* per-pair w = M* gamma*(theta), cubic disorientation (Sec. 4.3) */
#define LSGG_PHYSICS_MAGNETIC       2  /* w = 1, per-grain bulk energy (Eqs. (18)-(19)) */

#define LSGG_STORAGE_FP32  0   /* phi stored in FP32 */
#define LSGG_STORAGE_BF16  1   /* phi stored in BF16 between steps, FP32 arithmetic */

#define LSGG_EXEC_BATCHED  0   /* all boxes at once: 3D boxes by five passes over (box, plane /
                                  slab / column) work items in size tiers (x, y side <= 32, 40, 48, 64
                                  in shared memory, larger through global memory), 2D boxes by
                                  box-streaming kernels; persistent grids, one CUDA graph per step */
#define LSGG_EXEC_PLAIN    1   /* comparator: separate launches per grain per sub-step */
#define LSGG_EXEC_STREAMED 2   /* all boxes by box-streaming kernels: one CTA streams one box
                                  along z (register-ring / shared-memory rings per size class) */

#define LSGG_REDIST_TAXICAB 0  /* Sec. 2.1.6 as printed: taxicab propagation from the reference cells */
#define LSGG_REDIST_GODUNOV 1  /* the Euclidean first-order (Godunov upwind) update instead, iterated
                                  (Jacobi, 20 sweeps over the boxes); LSGG_EXEC_BATCHED, 3D only */
#define LSGG_REDIST_HARTMANN 2 /* the constrained reinitialization of Hartmann, Meinke and Schroeder
                                  (Sec. 2.1.6 names it; its first form): 20 forward-Euler steps of
                                  phi_tau + S(phi0)(|grad phi| - 1) = beta F, dtau = 1/2, beta = 1/2,
                                  Godunov upwind gradient, F pulling the cells next to the zero level
                                  towards the values that keep phi0's interpolated crossings in place;
                                  LSGG_EXEC_BATCHED, 3D only */

#define LSGG_MOBILITY_STEP  0  /* mob_low below theta_max, 1 above */
#define LSGG_MOBILITY_EQ20  1  /* Eq. (20): 1 - 0.99 exp(-5 (theta / 15 deg)^9) */

typedef struct lsgg_config {
    int32_t nx, ny, nz;        /* domain size in cells; nz == 1 selects 2D */
    int32_t n_grains;          /* number of seeds (grains), >= 1 */
    uint64_t seed;             /* SplitMix64 seed for generated seeds / weights / orientations */
    int32_t halo;              /* box halo in cells around the positive set (default 5) */
    int32_t radius;            /* heat-kernel half width R in cells, 1..7 (default 5) */
    float eps;                 /* band half width: phi is clamped to [-eps, eps] (default 7) */
    int32_t init_kind;         /* LSGG_INIT_* */
    int32_t physics;           /* LSGG_PHYSICS_* */
    int32_t storage;           /* LSGG_STORAGE_* */
    int32_t exec;              /* LSGG_EXEC_* */
    int32_t mobility_law;      /* LSGG_MOBILITY_* (READ_SHOCKLEY only) */
    int32_t device;            /* CUDA device ordinal */
    int32_t redist;            /* LSGG_REDIST_* re-initialisation metric (default TAXICAB) */
    int32_t reserved;          /* 0 */
    double theta_max_deg;      /* Read-Shockley / mobility cut-off angle (default 15) */
    double mob_low;            /* low-angle mobility for LSGG_MOBILITY_STEP (default 0.1) */
    double lognormal_sigma;    /* LAGUERRE: sigma of the lognormal radii (default 0.5) */
    double big_fraction;       /* LAGUERRE: fraction of enlarged grains (default 0.01) */
    double big_volume;         /* LAGUERRE: their volume factor (default 5) */
    double field_dir[3];       /* MAGNETIC: field direction (normalised by the library) */
    double energy_scale;       /* MAGNETIC: grid-unit bulk energy of cos^2 = 1, i.e.
                                  B^2 dchi h / (2 mu0 gamma_max) (Eqs. (13), (18)) */
    double arena_slack;        /* device box arena capacity / initial need (default 1.5) */
    double gb_map_tube;        /* 0 (default): Eq. (10)'s pair (i, j) per cell from the ID-field; > 0
                                  (physics other than IDEAL, batched 3D, below eps): every cell with
                                  |phi_i| < gb_map_tube takes j from the closest point of grain i's
                                  triangulated boundary (Sec. 2.1.4; lsgg_closest_gb_map) */
    const double* seeds;       /* optional n_grains x 3 (x, y, z) seed points in cells */
    const double* weights;     /* optional n_grains power weights (LAGUERRE) */
    const double* quats;       /* optional n_grains x 4 unit quaternions (w, x, y, z) */
    const double* energy;      /* optional n_grains bulk energies in grid units (MAGNETIC) */
    const int32_t* labels;     /* LABELS: nx*ny*nz grain ids in [0, n_grains), x fastest (host memory,
                                  read during creation); grain i starts on its box (per axis the
                                  shortest periodic arc of its cells grown by the halo) with the
                                  re-initialisation of +1/2 on its cells and -1/2 elsewhere; a label
                                  without a cell is an extinct grain.  Batched 3D only */
} lsgg_config;

/* Fill *cfg with the defaults above (64^3, 50 grains, seed 1, ideal, FP32, batched). */
void lsgg_config_default(lsgg_config* cfg);

/* --------------------------------------------------------------- lifecycle */
typedef struct lsgg_ctx lsgg_ctx;

/* Algorithm 1, Initialization (Sec. 2.1.3, reading of Sec. 3.1's tessellation
 * input): seeds (given, or drawn from cfg->seed by SplitMix64 as in
 * lsgg_generate_seeds) -> Voronoi / power labels on the grid (FP64, minimum
 * image, lowest id on ties) -> per grain the bbox of its cells grown by the
 * halo (an axis reaching the domain size becomes full and periodic) -> phi_i
 * = min over face-adjacent grains j of the signed distance to the (power)
 * bisector plane, clamped to [-eps, eps].  Grains with no cell start extinct.
 * `stream` is a cudaStream_t (NULL: the library creates its own).  The call
 * synchronises before returning.  On success *out owns the device state. */
int lsgg_create_microstructure(const lsgg_config* cfg, void* stream, lsgg_ctx** out);

/* n time steps of Algorithm 1 with time dt (grid units; dt = 1 gives a heat
 * kernel of variance 2 per axis).  Enqueues on the context's stream and
 * returns after enqueue; lsgg_sync waits.  dt must satisfy 0 < dt <= 4. */
int lsgg_step(lsgg_ctx* ctx, int32_t n, double dt);

/* Wait for enqueued work, at most timeout_ms (< 0: no limit).  Handles a box
 * arena that ran out of room by growing it and finishing the steps.  Returns
 * LSGG_ERR_TIMEOUT if the wait expired (the work keeps running).  A failure
 * on the device (LSGG_ERR_TIMEOUT from a bounded wait in a kernel,
 * LSGG_ERR_UNSUPPORTED from a launch that refused its input) is returned
 * once and cleared; the steps that did not complete are dropped
 * (lsgg_get_stats' steps_done counts the completed ones). */
int lsgg_sync(lsgg_ctx* ctx, int64_t timeout_ms);

/* ------------------------------------------------------------ step groups
 * Several microstructures advanced by one set of launches per step
 * (Algorithm 1's loop body over the boxes of every member at once, Sec. 3.1's
 * per-grain work spread over all of them): each pass kernel walks the
 * concatenation of the members' work items, so that many small simulations
 * share the GPU's SMs instead of each occupying it with its own launches.
 * Each member keeps its own domain, grains, arenas and field; the results of a
 * member are bit for bit those of stepping it alone with lsgg_step.
 *
 * lsgg_group_create: members = n (1 <= n <= LSGG_MAX_GROUP) contexts created on
 * the same device with exec LSGG_EXEC_BATCHED, a 3D domain, physics
 * LSGG_PHYSICS_IDEAL, redist LSGG_REDIST_TAXICAB, radius 5, no anisotropy map
 * and kernel timing off; anything else is LSGG_ERR_UNSUPPORTED, a NULL or
 * repeated member LSGG_ERR_INVALID_ARG.  The group holds the pointers, not
 * the contexts: destroy the group before any of its members.  The call
 * allocates the group's device array and streams; *out owns them. */
#define LSGG_MAX_GROUP 64
typedef struct lsgg_group lsgg_group;
int lsgg_group_create(lsgg_ctx* const* members, int32_t n, lsgg_group** out);

/* n steps with time dt of every member, enqueued on the group's stream after
 * the work already enqueued on each member's stream; each member's stream
 * then waits for them, so that its later calls (lsgg_sync, outputs) see the
 * steps.  step_limits (optional, n_members entries): member k takes part only
 * while its completed steps are below step_limits[k] (an absolute count since
 * its creation), so members needing different step counts share the chunk.
 * A member whose box arena runs out of room halts; lsgg_sync on it grows the
 * arena and finishes its steps alone.  Returns after enqueue. */
int lsgg_group_step(lsgg_group* g, int32_t n, double dt, const int64_t* step_limits);

/* Replace the group's members (same rules as lsgg_group_create) without any
 * allocation or synchronisation: the next lsgg_group_step advances the new
 * members, after the steps already enqueued for the old ones.  A server
 * changes the membership whenever a request joins or completes. */
int lsgg_group_set_members(lsgg_group* g, lsgg_ctx* const* members, int32_t n);

/* Waits for the group's work and frees the group (not its members). */
int lsgg_group_destroy(lsgg_group* g);

/* Per-grain volume V_i = sum_x H(phi_i(x)), H(phi) = clamp(phi + 1/2, 0, 1).
 * The paper does not define a grain's volume; this is a smooth cell count:
 * the zero level of phi_i smeared over one cell, so that it moves
 * continuously with the interface (the volumes the grain-size analysis of
 * Sec. 5 takes its equivalent radii from).  Computed from exact fixed-point
 * partial sums merged with FP64 compensated sums in a fixed order
 * (deterministic); index = grain id, 0 for extinct grains.  out: host array
 * of cap >= n_grains doubles; *n_out = n_grains.  Synchronises. */
int lsgg_grain_volumes(lsgg_ctx* ctx, double* out, int64_t cap, int64_t* n_out);

/* Grain statistics of the size analysis (Sec. 5), computed on the device from
 * the grain volumes: the alive grains (V > 0), their mean volume, the mean,
 * root-mean-square and largest equivalent radius R = (3 V / 4 pi)^(1/3)
 * (3D; (V / pi)^(1/2) in 2D), and the distribution of R / <R> as fractions of
 * the alive grains in n_bins equal bins over [0, r_max_rel) (hist, n_bins
 * doubles; the fraction at or above r_max_rel in overflow).  Deterministic
 * (fixed-order FP64 compensated sums, integer bin counts).  Synchronises. */
typedef struct lsgg_grain_stats {
    int64_t alive;
    double mean_volume;
    double mean_radius;
    double rms_radius;
    double max_radius;
    double overflow;
    double rho;                /* <R>^2 / <R^2> (Sec. 5) */
    double var_z;              /* Var(R / <R>) = <R^2> / <R>^2 - 1 = 1 / rho - 1 (Eq. (varianz)) */
} lsgg_grain_stats;
int lsgg_grain_statistics(lsgg_ctx* ctx, int32_t n_bins, double r_max_rel, lsgg_grain_stats* out, double* hist);

/* Texture shares (Sec. 5.3's texture components): for each class c in
 * [0, n_classes), the summed volume of the grains with grain_class[id] == c
 * over the summed volume of all grains (grains of other classes count in the
 * total only).  grain_class: host array of n_grains int32; out: host array of
 * n_classes doubles; 1 <= n_classes <= 4096.  Computed on the device from the
 * grain volumes with compensated sums in a fixed order (deterministic).
 * Synchronises. */
int lsgg_texture_shares(lsgg_ctx* ctx, const int32_t* grain_class, int32_t n_classes, double* out);

/* Size analysis of Sec. 5 on the host (no context, no device).
 * lsgg_rios_pdf: Rios' distribution of z = R / <R> (Eq. (Rios), H = 3, the
 * printed factor nu^(H0/2) read as nu^(H/2), under which it integrates to
 * 1); NaN unless 0 < nu < 4, rho > 0 and z >= 0.
 * lsgg_hillert_pdf: Hillert's distribution in z, rho P(rho z) with
 * rho = 8/9 and P(u) = (2e)^3 3u / (2 - u)^5 exp(-6 / (2 - u)) for u < 2 (the
 * nu -> 4 limit of Rios').
 * lsgg_fit_rios_nu: the nu in (0, 4) whose Rios density is closest (least
 * squares at the bin centres) to hist, fractions per bin of [0, r_max_rel)
 * as lsgg_grain_statistics gives them, for the given rho.
 * lsgg_fit_growth_exponent: the kinetic exponent n of <R> ~ t^n and k, fitted
 * as <R>^(1/n) - <R_0>^(1/n) = k t (the printed law <R>^n - <R_0>^n = k t
 * read with the reported n = 0.45-0.46 as the exponent of <R>) over n
 * samples (t increasing, <R> > 0; n >= 3), n searched in [0.05, 2].
 * The fits return LSGG_ERR_INVALID_ARG for invalid input. */
double lsgg_rios_pdf(double z, double nu, double rho);
double lsgg_hillert_pdf(double z);
int lsgg_fit_rios_nu(const double* hist, int32_t n_bins, double r_max_rel, double rho, double* nu);
int lsgg_fit_growth_exponent(const double* t, const double* mean_r, int32_t n, double* n_out, double* k_out);

/* Grid coarsening (Sec. 4.1: as the population falls the spacing grows so a
 * grain keeps about the same number of cells; each function is projected to
 * the coarser grid by trilinear interpolation).  The same periodic 3D domain
 * on nx x ny x nz cells, one spacing: nx / Nx = ny / Ny = nz / Nz, each at
 * most the current count.  Coarse cell i' of an axis sits at fine index
 * coordinate u = i' N / N' (cell 0 in place); its value interpolates the fine
 * values at floor(u), floor(u) + 1 (-eps outside the grain's box), is scaled
 * by N' / N and clamped to [-eps, eps]; then the step's re-initialisation
 * (the configured metric) and box update run on the coarse boxes; with
 * physics other than ideal growth the ID-field is rebuilt from the coarse
 * functions (argmax over the other grains).  No step is counted.  eps, the
 * halo, the kernel radius and dt stay in grid units, so one step's physical
 * time grows with the spacing squared, and volumes are in coarse cells.
 * Batched execution of a 3D domain only (else LSGG_ERR_UNSUPPORTED);
 * LSGG_ERR_INVALID_ARG for unequal ratios or a finer grid.  Waits for
 * enqueued steps first; synchronises. */
int lsgg_coarsen(lsgg_ctx* ctx, int32_t nx, int32_t ny, int32_t nz);

/* Voxel owner map: owner(x) = argmax_i phi_i(x) over the boxes covering x --
 * the grain whose function is largest at x, i.e. the grain the comparison
 * step of Eq. (16) leaves positive there and the voxel ID-field of Sec. 3.1
 * records -- lowest id on ties, -1 where no box covers x; x fastest,
 * n_cells >= nx*ny*nz int32s.  Synchronises. */
int lsgg_voxel_owner(lsgg_ctx* ctx, int32_t* out, int64_t n_cells);

/* Device-pointer variants of lsgg_grain_volumes and lsgg_voxel_owner (same
 * definitions and results, bit for bit) for outputs that stay on the device,
 * e.g. in a torch tensor's data_ptr().  out_dev: DEVICE array of cap >=
 * n_grains doubles / n_cells >= nx*ny*nz int32s, owned by the caller.
 * status_dev (optional DEVICE int32, may be NULL) receives the status of the
 * steps enqueued before the call, read on the device: 0, their error code, or
 * LSGG_ERR_CAPACITY when one of them stopped on a full box arena -- then the
 * output describes the state before that step, and lsgg_sync (which grows the
 * arena and finishes the steps) followed by another call gives the result.
 * The work is enqueued on `stream` (a cudaStream_t; NULL = the context's
 * stream) after the context's enqueued work, and the context's later work
 * waits for it; the calls do not synchronise and allocate nothing.  The owner
 * map takes the context's neighbour-max field as scratch, so
 * lsgg_grain_neighbours needs another step afterwards. */
int lsgg_grain_volumes_device(lsgg_ctx* ctx, double* out_dev, int64_t cap, int32_t* status_dev, void* stream);
int lsgg_voxel_owner_device(lsgg_ctx* ctx, int32_t* out_dev, int64_t n_cells, int32_t* status_dev, void* stream);

/* Free all device memory of the context (after finishing its work). */
int lsgg_destroy(lsgg_ctx* ctx);

const char* lsgg_status_string(int status);

/* The context's CUDA stream (a cudaStream_t) so callers can order their own
 * work and time the library's kernels with events on it. */
void* lsgg_get_stream(lsgg_ctx* ctx);

/* sizeof(lsgg_config) as compiled into the library: bindings check their
 * struct layout against it before calling lsgg_create_microstructure. */
size_t lsgg_abi_config_size(void);

/* ------------------------------------------------------------- inspection */
#define LSGG_PASS_TIERS 5      /* pass-path tiers: boxes of x, y side <= 32, <= 40, <= 48, <= 64, larger */
typedef struct lsgg_stats {
    int64_t steps_done;        /* steps completed since creation */
    int64_t cell_updates;      /* box cells advanced, summed over completed steps */
    int64_t alive;             /* grains with a positive cell */
    int64_t box_cells;         /* sum over alive grains of box volume (cells) */
    int64_t arena_capacity;    /* device arena capacity per buffer (elements) */
    double superimposition;    /* box_cells / (nx*ny*nz) (Sec. 5.2.3) */
    int64_t device_bytes;      /* device memory held by the context */
    int32_t n_classes;         /* box-size classes of the batched path */
    int32_t class_count[8];    /* boxes per class at the last box update */
    int64_t pass_cells[LSGG_PASS_TIERS];  /* box cells on the pass path per tier (x, y side
                                  <= 32, <= 40, <= 48, <= 64, larger) at the last box update; 0 off the
                                  pass path */
} lsgg_stats;

int lsgg_get_stats(lsgg_ctx* ctx, lsgg_stats* out);

/* Kernel timing with CUDA events on the context's stream.  While enabled,
 * lsgg_step launches eagerly (no graph) and records events between the
 * kernel groups of every step, and runs the kernels of a step one after
 * another on the context's stream (unprofiled steps run size classes and
 * tiers concurrently), so each kernel's time is its own.
 * lsgg_kernel_times synchronises and writes,
 * for groups 0 = neighbour-max field clear (pass path: tile binning),
 * 1 = predictor (k_predict; pass path: p_conv_xy, p_conv_z, p_field),
 * 2 = corrector + re-initialisation (k_correct; pass path: p_redist_xy,
 * p_redist_z), 3 = box update
 * (k_box_update): out_ms[g] = summed device milliseconds and out_count[g] =
 * kernel launches of the library in that group (any pointer may be NULL),
 * over the steps since the previous call; then resets the sums. */
int lsgg_profile(lsgg_ctx* ctx, int32_t enable);

/* Tile autotuner of the batched path.  On the pass path (3D boxes) it runs
 * four trials of steps_per_trial profiled steps each -- every persistent grid
 * at the CTAs per SM that fit, every grid at half of that, and slab items of
 * 4 and 16 planes for the re-initialisation's plane pass instead of 8 -- and
 * keeps per tier and pass the faster grid and the slab with the least plane
 * pass time (read back with lsgg_pass_tuning); chosen (optional, 2 x 8
 * int32) is then all -1.  Otherwise, for every box-size class served by the
 * register-ring kernels, it runs steps_per_trial real steps with each tile
 * variant (cells per thread, threads per CTA), times each class's kernels
 * with CUDA events on its stream, and keeps the fastest variant per class
 * and kernel; chosen: variant per kernel (predictor, corrector) and class,
 * -1 for classes not served by these kernels.  Every setting gives
 * bit-identical steps, so the tuning steps are ordinary steps of the
 * simulation (4 x steps_per_trial on the pass path, 3 x steps_per_trial
 * otherwise, time dt).  Synchronises. */
int lsgg_autotune(lsgg_ctx* ctx, int32_t steps_per_trial, double dt, int32_t* chosen);

/* The pass path's current tuning: ctas_per_sm (optional, 4 * LSGG_PASS_TIERS
 * int32) the CTAs per SM of the persistent grids of p_conv_xy, p_conv_z,
 * p_redist_xy and p_redist_z of each tier, slab (optional) the planes per slab
 * item of p_redist_xy; -1 off the pass path. */
int lsgg_pass_tuning(lsgg_ctx* ctx, int32_t* ctas_per_sm, int32_t* slab);
int lsgg_kernel_times(lsgg_ctx* ctx, double* out_ms, int64_t* out_count);

/* Per-pass timing of the pass path (LSGG_EXEC_BATCHED, 3D), from the same
 * profiled steps as lsgg_kernel_times (arrays of 4 * LSGG_PASS_TIERS + 2;
 * NULL allowed): out_ms[t * 4 + k] / out_count[t * 4 + k] for tier t = 0
 * (boxes of x, y side <= 32), 1 (<= 40), 2 (<= 48), 3 (<= 64), 4 (larger:
 * plane passes through global memory) and pass k = 0 p_conv_xy,
 * 1 p_conv_z, 2 p_redist_xy, 3 p_redist_z; [4 * LSGG_PASS_TIERS] the tile
 * binning (k_bin), [4 * LSGG_PASS_TIERS + 1] the field pass (p_field, all
 * boxes).  In lsgg_kernel_times the binning is group 0 and the field
 * pass belongs to group 1.  Synchronises, then resets the sums. */
int lsgg_pass_times(lsgg_ctx* ctx, double* out_ms, int64_t* out_count);

/* Contact neighbours of every grain after the last completed step (Sec. 3.1's
 * neighbourhood from the points of contact): the distinct grains j != i that
 * are the largest other function somewhere in grain i's box with a value above
 * -eps -- the ids of its ID-field.  counts[i] = number of neighbours (at most
 * cap_per_grain are stored, ascending, at ids[i * cap_per_grain ...]; a count
 * above cap_per_grain means the list was cut).  Reads the neighbour-max field
 * of the last step, which the pass path stores only while lsgg_keep_field is
 * on: needs such a step since creation or lsgg_set_state (else
 * LSGG_ERR_NOT_READY).  Synchronises. */
int lsgg_grain_neighbours(lsgg_ctx* ctx, int32_t* counts, int32_t* ids, int32_t cap_per_grain);

/* The pass path's field pass consumes each domain cell's two largest
 * (phi_p, grain) pairs (the neighbour-max field of Eq. (16)) in registers;
 * with on != 0 it also stores them (16 bytes per domain cell and step) for
 * lsgg_grain_neighbours.  Off by default.  The box-streaming and plain modes
 * always build the field in device memory. */
int lsgg_keep_field(lsgg_ctx* ctx, int32_t on);

/* Boxes of all grains: out[7*i .. 7*i+6] = alive, ox, oy, oz, nx, ny, nz
 * (origin in [0, N) per axis).  cap in int32s, >= 7 * n_grains.  Synchronises. */
int lsgg_get_boxes(lsgg_ctx* ctx, int32_t* out, int64_t cap);

/* phi of all alive grains, packed in grain-id order, each box x fastest with
 * no padding (sum of nx*ny*nz over alive grains floats).  *n_out = that
 * count; LSGG_ERR_CAPACITY if cap is smaller.  Synchronises. */
int lsgg_get_phi(lsgg_ctx* ctx, float* out, int64_t cap, int64_t* n_out);

/* Replace the state: boxes as in lsgg_get_boxes (7 int32 per grain), phi
 * packed as in lsgg_get_phi, idf (optional, may be NULL) the ID-field packed
 * the same way (-1 = no neighbour).  Grows the arena if needed.  Synchronises. */
int lsgg_set_state(lsgg_ctx* ctx, const int32_t* boxes, const float* phi, const int32_t* idf);

/* One step like lsgg_step(ctx, 1, dt) that also copies the step's
 * intermediate fields to host arrays (each packed like lsgg_get_phi in the
 * boxes the step ran on, i.e. lsgg_get_boxes before the call; any pointer may
 * be NULL): phip = predictor output, m = max_{j != i} phi_p_j, idm = its
 * argmax (-1 when no other grain exceeds -eps), phic = comparison output,
 * phin = re-initialised phi before the box update.  Synchronises. */
int lsgg_debug_step(lsgg_ctx* ctx, double dt, float* phip, float* m, int32_t* idm,
                    float* phic, float* phin);

/* ------------------------------------------------------------- serving */
/* A server runs independent simulations on one GPU with continuous batching
 * (the paper has no serving layer; this is a request loop around Algorithm 1).
 * Requests wait in FIFO order; a scheduler thread admits the head request when
 * a slot is free and the HBM estimates of the running requests plus its own
 * fit in budget_bytes and creates its microstructure (boxes resident on the
 * device).  With shared launches (LSGG_SERVE_SHARED, the default of
 * lsgg_server_create) the running requests of at most 128^3 domain cells that
 * a step group accepts (lsgg_group_create: batched 3D, ideal growth, taxicab,
 * radius 5) and share one dt advance together: one group over all of them (up
 * to LSGG_MAX_GROUP) takes chunks of steps_per_round steps, each request
 * stopping at its own step count; the group's members are replaced whenever a
 * request joins or completes, with at most two chunks queued ahead.  Larger
 * requests fill the GPU with their own launches.  Other requests, and every
 * request with LSGG_SERVE_PER_CONTEXT, get their own stream fed with chunks of
 * their own steps, so that requests overlap on the device.  Finished requests
 * keep their grain volumes on the host and release their device memory.
 * Results are those of lsgg_create_microstructure + lsgg_step(n_steps, dt) +
 * lsgg_grain_volumes run alone.  Times are seconds since lsgg_server_create. */
typedef struct lsgg_server lsgg_server;
#define LSGG_SERVE_PER_CONTEXT 0
#define LSGG_SERVE_SHARED 1

typedef struct lsgg_request_info {
    int32_t state;             /* 0 queued, 1 running, 2 done, < 0 failed with that status */
    double t_submit, t_admit, t_done;
    int64_t cell_updates;      /* box cell-updates of the request's steps */
    int64_t device_bytes;      /* device memory its context held after creation */
    int64_t estimate_bytes;    /* the admission estimate */
} lsgg_request_info;

typedef struct lsgg_server_stats {
    int64_t queued, active, completed;
    int64_t used_bytes, peak_bytes;   /* admission estimates in use / at most */
    int64_t cell_updates;             /* summed over completed requests */
} lsgg_server_stats;

int lsgg_server_create(int64_t budget_bytes, int32_t max_active, int32_t steps_per_round, int32_t device,
                       lsgg_server** out);
/* lsgg_server_create with the scheduling mode: LSGG_SERVE_SHARED or
 * LSGG_SERVE_PER_CONTEXT (anything else: LSGG_ERR_INVALID_ARG). */
int lsgg_server_create_mode(int64_t budget_bytes, int32_t max_active, int32_t steps_per_round, int32_t device,
                            int32_t mode, lsgg_server** out);
/* Queue a request; cfg and its arrays (seeds, weights, quats, energy, labels)
 * are copied before the call returns.  *ticket identifies it.
 * A request whose estimate exceeds the whole budget fails with
 * LSGG_ERR_OVER_BUDGET when it reaches the head of the queue. */
int lsgg_server_submit(lsgg_server* s, const lsgg_config* cfg, int32_t n_steps, double dt, int64_t* ticket);
/* LSGG_OK when done, LSGG_ERR_NOT_READY while queued or running, the failure status otherwise. */
int lsgg_server_poll(lsgg_server* s, int64_t ticket, lsgg_request_info* info);
/* Block until done (timeout_ms < 0: no limit; LSGG_ERR_TIMEOUT on expiry). */
int lsgg_server_wait(lsgg_server* s, int64_t ticket, int64_t timeout_ms, lsgg_request_info* info);
/* Grain volumes of a finished request (cap >= n_grains doubles). */
int lsgg_server_volumes(lsgg_server* s, int64_t ticket, double* out, int64_t cap, int64_t* n_out);
/* Forget a finished request's record. */
int lsgg_server_release(lsgg_server* s, int64_t ticket);
int lsgg_server_get_stats(lsgg_server* s, lsgg_server_stats* out);
/* Stop the scheduler; running requests are abandoned and their memory freed. */
int lsgg_server_destroy(lsgg_server* s);

/* -------------------------------------------------- stateless device ops */
/* A box of the packed layout used by the stateless ops: origin in [0, N) per
 * axis, dims 1..N per axis (nx <= 0: an unused entry), and the element offset
 * of the box's first cell in the packed per-cell arrays (x fastest, then y,
 * then z, no padding). */
typedef struct lsgg_box {
    int32_t ox, oy, oz;
    int32_t nx, ny, nz;
    int64_t offset;
} lsgg_box;

/* Corrector, first part (Eq. (16), max over all other grains; Sec. 3.1
 * ID-field): for every cell c of every box i,
 *   m[c]  = max over boxes j != i that cover c's domain cell of phip_j there,
 *           -eps where no other box covers it (outside its box a grain's
 *           function is -eps),
 *   id[c] = that j (lowest index on ties), -1 where m[c] == -eps.
 * The domain is periodic, nx*ny*nz cells.  All array pointers are DEVICE
 * pointers: boxes_dev (n_boxes entries), phip_dev / m_dev / id_dev (n_elems
 * entries each, indexed by the boxes' offsets), scratch_dev (16 * nx*ny*nz
 * bytes, 16-byte aligned, overwritten: the per-cell top-2 field).  Boxes
 * with an origin or dims out of range, or reaching past n_elems, are skipped
 * and their outputs left untouched.  Enqueued on `stream` (a cudaStream_t,
 * NULL = legacy default stream); returns after enqueue. */
int lsgg_neighbour_max(const lsgg_box* boxes_dev, int32_t n_boxes, const float* phip_dev, int64_t n_elems,
                       int32_t nx, int32_t ny, int32_t nz, float eps, void* scratch_dev,
                       float* m_dev, int32_t* id_dev, void* stream);

/* Largest domain (nx*ny*nz cells) lsgg_neighbour_max_noalloc accepts: its
 * top-2 field is a fixed 16 * 2^20 bytes = 16 MiB of static device memory. */
#define LSGG_NOALLOC_MAX_CELLS (1 << 20)

/* lsgg_neighbour_max for callers that cannot allocate device memory.  The
 * paper has no counterpart: this is an interface for hosts that own all
 * device memory themselves (a server that hands its whole budget to its own
 * pool, a plug-in inside a framework that exposes no allocator) or that keep
 * cudaMalloc / cudaFree out of latency-critical loops (cudaFree synchronises
 * the device, cudaMalloc can wait on other work).  Same arguments, result
 * and rules as lsgg_neighbour_max, without scratch_dev: the scratch field is
 * a file-scope static device array of LSGG_NOALLOC_MAX_CELLS cells that
 * every GPU on which the library's ops module is loaded keeps until the
 * process exits.  The call allocates nothing (no cudaMalloc, no cudaFree,
 * no allocating library routine).  Domains above LSGG_NOALLOC_MAX_CELLS
 * cells return LSGG_ERR_CAPACITY without touching the device.  Every call
 * looks up the array's device address in the current device's context
 * (cudaGetSymbolAddress, which allocates nothing), so a context torn down and
 * recreated in the same process is followed; the first lookup on a device
 * loads the library's ops module there, so make the first call on a device
 * before any stream capture.  Every call shares the one array and leaves the
 * last call's field in it (each call clears it first), so calls whose work
 * overlaps on the GPU (different streams, different host threads) race and
 * must be ordered by the caller. */
int lsgg_neighbour_max_noalloc(const lsgg_box* boxes_dev, int32_t n_boxes, const float* phip_dev,
                               int64_t n_elems, int32_t nx, int32_t ny, int32_t nz, float eps,
                               float* m_dev, int32_t* id_dev, void* stream);

/* Anisotropy map (Sec. 2.1.4: a grid point takes w and M of the closest
 * point on the grain boundary, found on a marching-cubes triangulation; Sec.
 * 4.1 accelerates that search).  For every box i of the packed set, its
 * boundary is the zero level of phi_i on the box's own cells (box-local: a
 * full periodic axis is not wrapped), triangulated by marching tetrahedra:
 * each cell cube split into the six tetrahedra around its main diagonal (one
 * per order of the axes z, y, x), the level linearly interpolated on the edges
 * between corners of opposite sign (phi > 0 inside); a quad (two positive
 * corners a < b, two others c < d, in the tetrahedron's corner order: the
 * cube corner, then one, two and three unit steps) is split along the
 * diagonal from the point on edge (a, c) to the point on edge (b, d).
 * A triangle faces the grain most frequent in idf among its tetrahedron's
 * corners with phi <= 0 (lowest id on ties, -1 without any).  Then for every
 * cell c of the box:
 *   out[c] = the grain of the triangle at the smallest (squared Euclidean
 *            distance from c, grain) when |phi[c]| < tube and the box has a
 *            triangle,
 *   out[c] = idf[c] otherwise (a box with an axis of one cell has none).
 * The result replaces the per-cell ID-field in Eq. (10)'s pair weights.
 * Distances are evaluated in FP32, so cells whose two nearest grains lie
 * within rounding of each other may take either.  All array pointers are
 * DEVICE pointers: boxes_dev (n_boxes entries, the origin is ignored),
 * phi_dev (float), idf_dev and out_dev (int32), each of n_elems entries
 * indexed by the boxes' offsets; out_dev must not overlap phi_dev or idf_dev.
 * Boxes with dims below 1 or reaching past n_elems are skipped and their
 * outputs left untouched.  0 < tube <= 16, else LSGG_ERR_INVALID_ARG.  The
 * search per cell covers the triangles of the cubes within ceil(tube) + 1
 * cells and, where the best distance there does not prove it the box's
 * minimum (a function far from a distance function, or a tube wider than
 * the function's band, which makes every cell a band cell), every triangle
 * of the box: the work is bounded by band cells x the box's triangles.
 * Allocates its scratch in stream order (cudaMallocAsync / cudaFreeAsync on
 * `stream`: per CTA room for the triangles of a box of up to 2^17 cubes;
 * larger boxes rebuild their triangles per cell) and returns
 * LSGG_ERR_OUT_OF_MEMORY if that fails.  Enqueued on `stream` (a
 * cudaStream_t, NULL = legacy default stream); returns after enqueue. */
int lsgg_closest_gb_map(const lsgg_box* boxes_dev, int32_t n_boxes, const float* phi_dev, const int32_t* idf_dev,
                        int64_t n_elems, float tube, int32_t* out_dev, void* stream);

/* Test hook: reallocate the context's box arenas to exactly `capacity`
 * elements (at least what the current state needs), so that a later box update
 * overflows and exercises the growth path of lsgg_sync.  Synchronises. */
int lsgg_debug_set_capacity(lsgg_ctx* ctx, int64_t capacity);

/* Test hook of the bounded device waits: one CTA initialises an mbarrier that
 * nothing will complete and waits on it for at most `iterations` polls, the
 * way the step kernels wait for their bulk copies; *timed_out = 1 when the
 * wait gave up (the kernel then returns normally).  Synchronises. */
int lsgg_debug_wait_timeout(int32_t device, int32_t iterations, int32_t* timed_out);

/* Test hook of the anisotropy map (contexts created with gb_map_tube > 0):
 * the pairs the next step's Eq. (10) blend will use.  idf_out = the ID-field
 * of the last step resampled onto the current boxes (-1 outside the previous
 * box), map_out = the map computed from it and the state on those boxes
 * (lsgg_closest_gb_map's definition, box-local to the current box); both
 * packed like lsgg_get_phi, cap >= that count.  LSGG_ERR_UNSUPPORTED without
 * the map.  Synchronises. */
int lsgg_debug_pair_ids(lsgg_ctx* ctx, int32_t* idf_out, int32_t* map_out, int64_t cap);

/* Test hook of the step's own bounded waits: the pass kernels poll the
 * mbarrier of each bulk copy at most `polls` times (polls < 0 restores the
 * default of 2^22) before they give up: the CTA records LSGG_ERR_TIMEOUT,
 * halts the step (the step's remaining launches return at once), waits with
 * the default bound for its copies in flight and returns.  With polls = 0 the
 * first plane pass of the next step gives up at its first wait, before any
 * kernel writes the state, so the state stays that of the last completed
 * step.  Waits for enqueued work first; the next step is captured anew. */
int lsgg_debug_set_wait_limit(lsgg_ctx* ctx, int32_t polls);

/* SplitMix64 seed points (host only, no device needed): out[3*i + a] =
 * u01(seed, 3*i + a) * N_a for a = x, y, z with
 * u01(s, k) = (mix(s + (k + 1) * 0x9E3779B97F4A7C15) >> 11) * 2^-53 and
 * mix the SplitMix64 finaliser; z = 0 in 2D.  out holds 3 * n doubles. */
int lsgg_generate_seeds(uint64_t seed, int32_t n, int32_t nx, int32_t ny, int32_t nz, double* out);

#ifdef __cplusplus
}
#endif

#endif /* LSGG_H */
