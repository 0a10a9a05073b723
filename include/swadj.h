/*
 * swadj.h -- C ABI of libswadj.so: the data-parallel hot path of adjoint-guided
 * refinement for tsunami modelling (Davis & LeVeque, arXiv 1605.05320) on one
 * NVIDIA GB300 (sm_103a).
 *
 * Conventions for every entry point
 * ---------------------------------
 *  - Arrays are cell-centred, row-major with x fastest: index j*nx + i.
 *  - "_host" pointers are host memory, "_dev" pointers are device memory of
 *    the current CUDA device.  Where an argument takes either, `where` says
 *    which (SWA_HOST / SWA_DEVICE).
 *  - The library never allocates device memory.  Each object has a
 *    *_workspace_bytes() query; the caller allocates that many bytes of
 *    device memory (256-byte aligned) and passes it to *_create(); the object
 *    carves its arrays out of it.  The caller keeps the workspace alive until
 *    the object is destroyed and frees it afterwards.  Handles themselves are
 *    small host structs owned by the library (freed by swa_destroy_*).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Device work
 *    is enqueued on it and the call returns without waiting, except where a
 *    function says it synchronises.  Forward and adjoint stepping keep time,
 *    time step and buffer parity on the device, so a sequence of calls can be
 *    captured into a CUDA graph and replayed.
 *  - Every function returns an int status (SWA_OK = 0 or a negative code).
 *    swa_last_error() gives a message for the calling thread.  No C++
 *    exception crosses the ABI.  Device-side problems (non-finite state,
 *    non-positive depth) set a device error word that swa_sync_status()
 *    reports.
 */
#ifndef SWADJ_H
#define SWADJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SWA_OK 0
#define SWA_EINVAL (-1)    /* bad argument */
#define SWA_ENOMEM (-2)    /* workspace too small / capacity exceeded */
#define SWA_ECUDA (-3)     /* a CUDA runtime call failed */
#define SWA_ESTATE (-4)    /* call not valid in the object's state */
#define SWA_EUNSTABLE (-5) /* device saw a non-finite value or depth <= 0 */
#define SWA_ETIMEOUT (-6)  /* reserved: a bounded device wait expired */

/* ---- enums ---- */
#define SWA_FP64 0      /* state (h, hu, hv) and bathymetry B in double     */
#define SWA_FP32 1      /* perturbation form: (eta, hu, hv) and hbar = -B in
                           float; the time step is still reduced in double  */
#define SWA_BC_EXTRAP 0 /* ghost cells copy the nearest interior cell        */
#define SWA_BC_WALL 1   /* ghost cells mirror, normal momentum negated       */
#define SWA_FLAG_INTERP 0  /* Eq. (ip_timerange), adjoint linear in time      */
#define SWA_FLAG_BRACKET 1 /* max over bracketing snapshots, Eq. (ip_timepoint)
                              when t_s = t_f                                  */
#define SWA_HOST 0
#define SWA_DEVICE 1

/*
 * Grid descriptor.  ndim = 1 (ny must be 1) or 2.  x_lo/y_lo: lower-left
 * corner; dx/dy: cell size.  bc[] = {x_lo, x_hi, y_lo, y_hi}.  g: gravity
 * (9.81); cfl: Courant number (0.75); dry_tol: depth at or below which a
 * cell is dry (1e-3 m).  order: 1 (Godunov) or 2 (MC-limited corrections).
 */
typedef struct swa_grid_desc {
    int ndim, nx, ny;
    double x_lo, y_lo, dx, dy;
    int precision;
    int order;
    int bc[4];
    double g, cfl, dry_tol;
} swa_grid_desc;

typedef struct swa_grid swa_grid;
typedef struct swa_adjoint swa_adjoint;
typedef struct swa_snapstore swa_snapstore;

const char *swa_version(void);
/* Message of the last failing call on this thread ("" if none). */
const char *swa_last_error(void);

/*
 * Synchronise `stream`, then read and clear the device error word shared by
 * all objects on the current device.  Returns SWA_OK, SWA_EUNSTABLE, or
 * SWA_ESTATE after an AMR step whose levels fell short of its end time.
 */
int swa_sync_status(void *stream);

/* =========================== forward grid ================================
 * The nonlinear shallow water equations with bathymetry, Eq. (swe_1d) in 1D
 * and Eq. (swe) in 2D (Sec. 3, Sec. 5), solved by a Godunov-type finite
 * volume method with a Roe-type Riemann solver per edge (Sec. 6).
 */
size_t swa_grid_workspace_bytes(const swa_grid_desc *desc);

/*
 * Create a forward grid in `ws` (ws_bytes >= swa_grid_workspace_bytes).
 * bathy_host: nx*ny bottom elevations B (host, FP64, copied).  The state is
 * the ocean at rest (eta = 0) until swa_set_state.
 */
int swa_create_grid(const swa_grid_desc *desc, const double *bathy_host,
                    void *ws, size_t ws_bytes, void *stream, swa_grid **out);
int swa_destroy_grid(swa_grid *grid);

/*
 * Set the state from surface elevation eta = h + B and momenta (FP64, n
 * values each; hv may be NULL for ndim = 1), at time t.  Also computes the
 * first time step from the CFL condition on the device.
 */
int swa_set_state(swa_grid *grid, const double *eta, const double *hu,
                  const double *hv, double t, int where, void *stream);

/*
 * Read the state as FP64 arrays of n values: any of h, hu, hv, eta may be
 * NULL.  where = SWA_HOST synchronises the stream.
 */
int swa_get_state(swa_grid *grid, double *h, double *hu, double *hv,
                  double *eta, int where, void *stream);

/*
 * Take up to max_steps explicit steps, stopping at t_end: each step uses
 * dt = min(cfl / s_max(Q^n), t_end - t_n), s_max = max over cells of
 * max((|u|+c)/dx, (|v|+c)/dy), c = sqrt(g h).  The update applies, at every
 * edge, the f-wave Roe solution with the bathymetry source folded into the
 * momentum jump (the ocean at rest is exact), the fluctuations of the cell's
 * edges and, for order 2, MC-limited corrections; in 2D the step is
 * dimensionally split (an x-sweep of every row, then a y-sweep of the
 * x-swept state).  The CFL maximum for the next step is reduced in the same
 * kernel.  Steps past t_end are no-ops on the device.
 */
int swa_step_forward(swa_grid *grid, int max_steps, double t_end, void *stream);

/* Synchronises; any pointer may be NULL. */
int swa_get_time(swa_grid *grid, double *t, double *dt_next,
                 long long *nsteps, void *stream);

/*
 * Launch shape of the FP32 2D step kernel: the height in rows of the strip a
 * warp walks, 16, 32 or 64 (0 restores the default, 32).  Results do not
 * depend on it; throughput does (the autotuner picks it per grid size).
 * FP64 and 1D grids ignore it.
 */
#define SWA_MIN_STRIP_ROWS 16
int swa_grid_set_strip_rows(swa_grid *grid, int rows);

/*
 * FP32 2D grids: on = 1 (the default) lets the step skip the wave arithmetic
 * of rows that are exactly at rest (eta = hu = hv = 0 across a warp's strip
 * row), where every wave is zero and the exact result is known, and write a
 * strip unit whose whole stencil window is at rest straight back at rest
 * (its CFL terms from a table of the bathymetry's rest terms, formed when
 * the grid is created); on = 0 computes them in full.  Both give the same
 * state and time step (up to the sign of an exact zero); the switch exists
 * to show that and to time the step without the shortcut.  SWA_EINVAL for a
 * null grid or on not 0 or 1.
 */
int swa_grid_set_rest_skip(swa_grid *g, int on);
/*
 * The 2D update that swa_step_forward applies.  The paper defers the theory
 * of its finite volume methods to LeVeque (2002) (Sec. 6); both are that
 * book's wave-propagation methods:
 *   SWA_SCHEME_SPLIT (default): dimensionally split, as described above.
 *   SWA_SCHEME_CTU: unsplit.  Every x- and y-edge Riemann problem is solved
 *     from Q^n; each cell takes the fluctuations and the limited-correction
 *     flux differences of its four edges, where an edge's flux also carries,
 *     with weight -dt / (2 d_other), the transverse parts of the four
 *     fluctuations of the other direction that enter the cells beside the
 *     edge and move towards it (split by the tangential flux Jacobian at
 *     their own edge's Roe state).  Second-order accurate for smooth flow
 *     and stable for Courant numbers up to 1 in each direction.
 * The CFL rule, the clock and gauges are the same for both.  1D grids accept
 * either (the updates coincide there); patch sets always use the split step.
 * Returns SWA_EINVAL for another value.  The FP64 unsplit step rounds like
 * the FP64 reference of the same scheme; FP32 grids keep the perturbation
 * form (eta, hu, hv).
 */
#define SWA_SCHEME_SPLIT 0
#define SWA_SCHEME_CTU 1
int swa_grid_set_scheme(swa_grid *grid, int scheme);

/*
 * Wet/dry option of the split step (on = 1; 0, the default, requires h > 0
 * everywhere).  Sec. 6's solver reduces to the Roe solver away from the
 * shore and handles inundation; the reading built here: at an edge with a
 * dry cell (h <= desc.dry_tol) or a transonic rarefaction (u - c or u + c
 * rising through zero from the left cell to the right one) the fluctuations
 * come from the hydrostatic reconstruction of Audusse et al. (2004) with an
 * HLL flux (speeds min/max of u -+ c over the reconstructed states), first
 * order; every other edge keeps the Roe f-waves and their limited
 * corrections.  After each sweep a cell at or below dry_tol keeps no
 * momentum and no negative depth, and dry cells carry no waves in the CFL
 * number.  Land is a cell with h = 0 (eta = B): set the state accordingly
 * after turning the option on; a negative depth in the state set is
 * reported as SWA_EUNSTABLE by the next swa_sync_status.  The ocean at rest
 * against dry land stays exactly at rest, and the mass is conserved between
 * walls as long as no depth goes negative, which the reconstruction
 * guarantees for cfl <= 1/2 (above it a cell that would go negative is set
 * dry, adding its deficit).  The option runs the tiled split kernel (FP64:
 * the reference's rounding; FP32: the perturbation form), not the FP32
 * strip kernel; with SWA_SCHEME_CTU a step returns SWA_EINVAL.  Host state
 * only.
 */
int swa_grid_set_wetdry(swa_grid *grid, int on);

/*
 * Device pointers of the current state arrays (read-only use), for gauge or
 * diagnostic kernels of the caller.  Synchronises (the current buffer is
 * device-resident).  precision tells the element type (double or float).
 */
int swa_grid_arrays(swa_grid *grid, const void **q0, const void **q1,
                    const void **q2, const void **bath, void *stream);

/* ============================== adjoint ==================================
 * The time-reversed adjoint of Sec. 4: q~(x,t) = q^(x, t_f - t) solves
 * q~_t - (A^T q~)_x [- (A_2^T q~)_y] = 0 forward in t with q~(0) = phi,
 * A, A_2 from the linearisation about the ocean at rest (Sec. 3, Sec. 5),
 * zero normal velocity at wet/dry edges (Sec. 5).  Fixed time step
 * dt = t_f / N, N = ceil(t_f * max(c/dx, c/dy) / cfl), c = sqrt(g hbar).
 * In 2D a step is a y-sweep then an x-sweep (the reverse of the forward
 * order, so that with walls it is the transpose of a linear forward step).
 */
size_t swa_adjoint_workspace_bytes(const swa_grid_desc *desc);

/*
 * bathy_host: adjoint-grid B (FP64, copied); phi_host: (ndim+1) x n values
 * of phi = q^(t_f) (component-major).  Synchronises once (to size N).
 */
int swa_create_adjoint(const swa_grid_desc *desc, const double *bathy_host,
                       const double *phi_host, double t_f, void *ws,
                       size_t ws_bytes, void *stream, swa_adjoint **out);
int swa_destroy_adjoint(swa_adjoint *adj);
/* N, dt and the number of steps taken so far. */
int swa_adjoint_info(const swa_adjoint *adj, long long *n_steps, double *dt,
                     long long *steps_done);
/* Take nsteps adjoint steps (clamped to the remaining N - steps_done). */
int swa_step_adjoint(swa_adjoint *adj, int nsteps, void *stream);
/*
 * Temporal blocking of the fixed-dt adjoint (a 2D FP32 adjoint only): k = 2
 * lets swa_step_adjoint and swa_run_adjoint take two steps per launch
 * wherever no snapshot falls on the step between them (one pass over the
 * state instead of two: each warp loads its strip once, with 4 halo rows and
 * columns, and writes only the second step's state).  The states and
 * snapshots are bit-identical to k = 1 (the default).  SWA_EINVAL for a
 * null adjoint, k not 1 or 2, or k = 2 on an FP64 or 1D adjoint.
 */
int swa_adjoint_set_steps_per_pass(swa_adjoint *adj, int k);
/* Read the adjoint state (FP64, (ndim+1) x n, component-major). */
int swa_get_adjoint_state(swa_adjoint *adj, double *q, int where, void *stream);
/*
 * Restart the adjoint from new data phi = q^(t_f) ((ndim+1) x n FP64,
 * component-major, host or device): steps_done returns to 0, N and dt are
 * kept (they depend only on the bathymetry).
 */
int swa_set_adjoint_state(swa_adjoint *adj, const double *phi, int where,
                          void *stream);

/* ============================= snapshots =================================
 * Snapshots of the adjoint at regular times (Sec. 4), device resident:
 * snapshot k holds q^(tau_k) = q~(t_f - tau_k), tau strictly decreasing.
 * precision: SWA_FP64 or SWA_FP32 storage.  FP32 stores of a 2D grid with
 * nx % 4 == 0 also keep an envelope (not in the paper; an exact pruning aid
 * of the flag pass): per group of 8 consecutive snapshots and per quad of 4
 * consecutive cells, the maximum |component| of each component, updated on
 * every store; it adds 3 * (n / 4) floats per group to the workspace.
 */
size_t swa_snapstore_workspace_bytes(const swa_grid_desc *adj_desc,
                                     int max_snaps, int precision);
int swa_create_snapstore(const swa_adjoint *adj, int max_snaps, int precision,
                         void *ws, size_t ws_bytes, swa_snapstore **out);
int swa_destroy_snapstore(swa_snapstore *store);
/* Append the current adjoint state with tau = t_f - steps_done * dt. */
int swa_store_snapshot(swa_adjoint *adj, swa_snapstore *store, void *stream);
/*
 * Whole adjoint solve: snapshot at tau = t_f, then N steps with a snapshot
 * every `every` steps and after the last; the snapshot copy is fused into
 * the step that produces it.  Fails with SWA_ENOMEM before enqueuing
 * anything if the store cannot hold them all.
 */
int swa_run_adjoint(swa_adjoint *adj, swa_snapstore *store, int every,
                    void *stream);
/* Forget all snapshots (the workspace is reused by the next ones). */
int swa_snapstore_clear(swa_snapstore *store);
/* Number of snapshots and (optionally) a host copy of their tau values. */
int swa_snapstore_info(const swa_snapstore *store, int *count, double *tau_host,
                       int tau_cap);

/* =============================== flagging ================================
 * Adjoint-weighted flagging (Sec. 4.1, 4.2, Sec. 6).  For the forward state
 * at its device time t and q = (eta, hu, hv):
 *   m(x) = max over tau in [t, T] of |q^(x, tau) . q(x, t)|,
 *   T = min(t + (t_f - t_s), t_f), the window clipped to the stored taus;
 * INTERP takes q^ piecewise linear in tau; BRACKET takes every snapshot from
 * the latest at or before t to the earliest at or after T.  q^ is bilinearly
 * interpolated from the adjoint grid's cell centres (clamped at the edge),
 * component by component.  m = 0 where the forward cell is dry or an adjoint
 * cell with positive weight is dry.  flags_dev[i] = (m >= tol); maxip_dev
 * (nullable, float) receives m; *count_dev (device int64, overwritten)
 * receives the number of flags.  t > t_f gives no flags.
 * When maxip_dev is null and the store has an envelope (FP32 forward grid
 * and FP32 snapshots of a 2D adjoint grid, the same grid or another one), a
 * snapshot group is read for a cell only if its envelope bound on
 * |q^ . q| reaches tol (1 - 1e-5) there (on another grid: the largest
 * envelope entry over the quads of the cell's bilinear stencil);
 * the flags and the count are identical to the full pass (every product the
 * pruned pass forms is the one the full pass forms; skipped products are
 * provably below tol), so only the optional m output needs the full pass.
 */
int swa_flag_cells(const swa_grid *grid, const swa_snapstore *store,
                   double t_s, double t_f, double tol, int mode,
                   uint8_t *flags_dev, float *maxip_dev, long long *count_dev,
                   void *stream);

/*
 * Surface flagging, the default criterion the paper compares adjoint
 * flagging against (Sec. 6): flags_dev[i] = 1 where the cell is wet and its
 * surface elevation relative to sea level exceeds tol, |eta| > tol.
 * *count_dev (device int64, overwritten) receives the number of flags.
 */
int swa_flag_surface(const swa_grid *grid, double tol, uint8_t *flags_dev,
                     long long *count_dev, void *stream);

/* ================================ gauges =================================
 * Surface elevation eta = h + B at n points xy_dev[2k], xy_dev[2k+1]
 * (device, FP64) by bilinear interpolation of cell centres, clamped to the
 * outermost centres (Sec. 6 gauges); written to eta_dev[0..n).
 */
int swa_gauge_sample(const swa_grid *grid, int n, const double *xy_dev,
                     double *eta_dev, void *stream);

/*
 * Gauge recording fused into the forward step.  Every step of
 * swa_step_forward that advances the grid (no-op steps past t_end record
 * nothing) samples eta at the n points xy_dev (device FP64, [n][2], as
 * swa_gauge_sample) from the state the step starts from, with one block
 * working beside the step's own, and writes row r of series_dev (device
 * FP64, [capacity][n], row-major) and, if times_dev (device FP64,
 * [capacity]) is not NULL, that state's time to times_dev[r]; r counts the
 * recorded steps from 0 and is reset to 0 by this call (stream-ordered).
 * So after k steps rows 0..k-1 hold the states at t_0 .. t_{k-1}; sample
 * the final state with swa_gauge_sample.  Rows past capacity are not
 * written.  The arrays are the caller's and must stay valid while
 * recording is on; n = 0 or capacity = 0 turns recording off.  Replaces one
 * gauge launch per step; values equal swa_gauge_sample's bit for bit.
 */
int swa_grid_record_gauges(swa_grid *grid, int n, const double *xy_dev,
                           double *series_dev, double *times_dev,
                           long long capacity, void *stream);
/* Rows recorded since the last swa_grid_record_gauges (synchronises). */
int swa_grid_gauge_rows(const swa_grid *grid, long long *rows, void *stream);

/* ======================= batched uneven patches ===========================
 * Many independent patches of refinement levels 1..SWA_MAX_LEVELS stepped
 * together (the AMR hierarchy of Sec. 1 and Sec. 6 holds patches on levels
 * with refinement ratios; here each patch is self-contained, with ghost
 * cells from its own boundary conditions and no exchange between patches).
 * FP32 perturbation form only.  One swa_step_level call enqueues one
 * kernel launch per step whose resident warps walk the strips (28 columns x
 * 16 or 32 rows) of every patch of that level; results do not depend on the
 * strip height.  All patches of a level share one time step, reduced on the
 * device from their CFL maxima (dt_l = cfl / max over the level's cells),
 * so a loop of level steps can be captured in a CUDA graph.
 */
#define SWA_MAX_LEVELS 8

typedef struct swa_patch_desc {
    int level;              /* 1 .. SWA_MAX_LEVELS                          */
    int nx, ny;             /* cells, each >= 2                              */
    double x_lo, y_lo;      /* lower-left corner                             */
    double dx, dy;          /* cell size; equal for all patches of a level   */
} swa_patch_desc;

typedef struct swa_patchset swa_patchset;

/* common: g, cfl, dry_tol, order, bc of every patch (ndim, nx, ny, x_lo,
 * y_lo, dx, dy and precision of `common` are ignored). */
size_t swa_patches_workspace_bytes(int n, const swa_patch_desc *patches,
                                   const swa_grid_desc *common);
/* bathy_host[k]: nx*ny bottom elevations of patch k (host FP64, copied).
 * The state starts as the ocean at rest. */
int swa_create_patches(int n, const swa_patch_desc *patches,
                       const double *const *bathy_host, const swa_grid_desc *common,
                       void *ws, size_t ws_bytes, void *stream, swa_patchset **out);
int swa_destroy_patches(swa_patchset *ps);
/* Set patch k from FP64 eta, hu, hv (host or device). */
int swa_patches_set_state(swa_patchset *ps, int k, const double *eta,
                          const double *hu, const double *hv, int where,
                          void *stream);
/* Restart the clock of `level` at time t, its first step from the CFL
 * condition of the level's current state (call after setting its patches). */
int swa_patches_start_level(swa_patchset *ps, int level, double t, void *stream);
/* Read patch k as FP64 (any pointer may be NULL); where = SWA_HOST syncs. */
int swa_patches_get_state(swa_patchset *ps, int k, double *h, double *hu,
                          double *hv, double *eta, int where, void *stream);
/* nsteps level steps, each stopping at t_end (steps past it are no-ops). */
int swa_step_level(swa_patchset *ps, int level, int nsteps, double t_end,
                   void *stream);
/* Synchronises; any pointer may be NULL. */
int swa_patches_get_time(swa_patchset *ps, int level, double *t, double *dt_next,
                         long long *nsteps, void *stream);
/* Number of patches, strips (work units of one warp, at the level's current
 * strip height) and cells of a level (host bookkeeping). */
int swa_patches_level_info(const swa_patchset *ps, int level, int *npatches,
                           int *ntiles, long long *ncells);
/* Strip height of the level's kernel in rows: 16 or 32 (0 = default: 16
 * when the level's 16-row strips are no more than the warps the launch keeps
 * resident, else 32).  Results do not depend on it; throughput does (the
 * autotuner picks it). */
int swa_patches_set_tile_rows(swa_patchset *ps, int level, int rows);

/* ============================== AMR glue ===================================
 * One coarse grid (FP32, 2D) and L nested levels of fine patches of a patch
 * set, level l refined from level l - 1 by an integer ratio r_l in space and
 * in time: the AMR hierarchy the paper's runs use (Sec. 1, Sec. 6; four
 * levels in its Crescent City run).
 *
 * Patches carry a 2-cell ring: a level-l patch whose interior is mx x my
 * level-(l - 1) cells with lower-left level-(l - 1) cell (i0, j0) (counted on
 * the uniform level-(l - 1) grid over the whole domain) is described with
 * nx = mx r_l + 4, ny = my r_l + 4, dx = dx_(l - 1) / r_l, dy likewise,
 * x_lo = coarse x_lo + i0 dx_(l - 1) - 2 dx, y_lo likewise.  Level-1 rings
 * must lie inside the coarse domain; every cell of a level-l patch (ring
 * included) must lie inside the interior of some level-(l - 1) patch for
 * l >= 2 (proper nesting).  The level step updates ring cells like any
 * other (they enter the level's CFL maximum); the fill before each launch
 * overwrites them.  The patch set's boundary conditions act only beyond the
 * ring, on ring cells: create it with SWA_BC_EXTRAP, the rule the hierarchy
 * is defined with.  Set every patch's state (ring included) and start every
 * level at the coarse grid's time before the first step.
 *
 * swa_amr_step(amr, t_n, dt_c, m, stream), all stream-ordered, no host sync
 * (Berger-Oliger subcycling):
 *   1. the coarse grid steps to t_n + dt_c (dt_c must not exceed its CFL
 *      step, so that it takes exactly one);
 *   2. run(1) over the coarse step, where run(l) over a parent step [t_p,
 *      t_p + dt_p] takes r_l substeps, the k-th ending at t_p + dt_p k /
 *      r_l, with one launch each for a level with children (its CFL step
 *      must cover the substep) and m launches each for the finest level
 *      (launches past the substep's end are no-ops).  Before every launch
 *      each ring cell is filled: from the lowest-index other patch of its
 *      level whose interior holds it, else from its parent (the coarse grid
 *      at level 1, else the lowest-index level-(l - 1) patch whose interior
 *      holds it), linearly in time between the parent's states at t_p and
 *      t_p + dt_p (alpha = (t - t_p) / dt_p in [0, 1], eta and both
 *      momenta), then piecewise linearly in space within the parent cell
 *      holding it, with minmod slopes from the parent's array (zero where a
 *      neighbour lies outside it: the domain edge of the coarse grid).
 *      After each substep of a level with children: run(l + 1) over it, then
 *      steps 3 and 4 for level l + 1;
 *   3. every copy of a level-(l - 1) cell under a level-l interior (the
 *      coarse cell, or its cell in each level-(l - 1) patch whose interior
 *      holds it) takes the mean of the r_l x r_l cells of the lowest-index
 *      level-l patch over it (eta and both momenta);
 *   4. refluxing (on unless swa_amr_set_reflux turned it off): every copy of
 *      an uncovered level-(l - 1) cell U beside a covered cell V takes, for
 *      each such edge, the mass its own updates moved through the edge minus
 *      the mass level l moved through it over the parent step (the cells of
 *      V's lowest-index level-l patch along the edge, weighted 1 / r_l):
 *        eta_U += sum dt_p / d phi_U - sum_launches dt_l / (d r_l) sum phi_l
 *      with phi the mass flux of the split step's update (x-edges from the
 *      state, y-edges from the x-swept state; the normal momentum of the
 *      cell below the edge plus the net the update gives it), signed into
 *      V, and d the level-(l - 1) cell width across the edge.  The fluxes
 *      are recomputed before each launch by the step's own edge arithmetic,
 *      summed in FP64 per edge and added to eta_U in FP32 after step 3.
 *      With every level's bottoms the means of the bottoms under them, the
 *      hierarchy then keeps its mass (the coarse grid's, whose covered cells
 *      hold the means of the levels below) to rounding, as conservative
 *      refinement requires (Sec. 6 runs GeoClaw's conservative AMR).  Only
 *      the mass is corrected.
 * If a level starts the step away from t_n or ends a parent step short of
 * its end (a CFL step below its substep, or m launches that did not reach a
 * substep's end), the next swa_sync_status returns SWA_ESTATE.
 */
typedef struct swa_amr swa_amr;
/* Device workspace for the maps and the refluxing slots (per level: 20
 * bytes per ring cell, 4 per patch of the patch set, 16 per covered parent
 * cell, 20 + 8 (1 + r) per coarse-fine edge, 16 per uncovered parent cell
 * beside the level, plus padding); 0 if the geometry is invalid (the reason is in swa_last_error).
 * levels[l - 1]: the patch-set level of hierarchy level l (1 .. nlevels);
 * ratios[l - 1]: r_l in [1, 64]. */
size_t swa_amr_levels_workspace_bytes(const swa_grid *coarse, const swa_patchset *fine,
                                      int nlevels, const int *levels, const int *ratios);
/*
 * coarse: a 2D FP32 grid; fine: a patch set whose patches of the listed
 * levels form the hierarchy (other levels are ignored); nlevels in
 * [1, SWA_MAX_LEVELS], no patch-set level listed twice.  ws: device buffer
 * of at least swa_amr_levels_workspace_bytes, 256-byte aligned, owned by
 * the caller for the hierarchy's lifetime; coarse and fine must outlive it
 * too.  Checks the geometry (SWA_EINVAL: level without patches, cell size
 * not the parent's / r, interior not on whole parent cells, ring outside the
 * domain, a patch not nested in its parent level, a patch set without
 * SWA_BC_EXTRAP), uploads the maps and clears the slots on `stream`, and
 * synchronises it.  SWA_ENOMEM if ws_bytes is too small.
 */
int swa_create_amr_levels(swa_grid *coarse, swa_patchset *fine, int nlevels, const int *levels,
                          const int *ratios, void *ws, size_t ws_bytes, void *stream,
                          swa_amr **out);
/* The two-level hierarchy: swa_amr_levels_workspace_bytes and
 * swa_create_amr_levels with nlevels = 1, levels = {level}, ratios =
 * {ratio}. */
size_t swa_amr_workspace_bytes(const swa_grid *coarse, const swa_patchset *fine, int level,
                               int ratio);
int swa_create_amr(swa_grid *coarse, swa_patchset *fine, int level, int ratio, void *ws,
                   size_t ws_bytes, void *stream, swa_amr **out);
/* Host bookkeeping only; the workspace stays the caller's. */
int swa_destroy_amr(swa_amr *amr);
/*
 * One coarse step of dt_c from t_n (the time every level must be at) with
 * the subcycled levels below it, max_launches launches per substep of the
 * finest level, enqueued on `stream`.  SWA_EINVAL: null hierarchy, dt_c <=
 * 0, max_launches < 1, refluxing on with the coarse grid on the unsplit
 * scheme (the recomputed fluxes are the split step's); SWA_ESTATE: coarse
 * state not set or a level not started; SWA_ECUDA: a launch failed.  Levels
 * off their times show up as SWA_ESTATE at the next swa_sync_status.
 */
int swa_amr_step(swa_amr *amr, double t_n, double dt_c, int max_launches, void *stream);
/* Refluxing (step 4 above) on (on != 0, the default) or off.  Host state
 * only; takes effect at the next swa_amr_step. */
int swa_amr_set_reflux(swa_amr *amr, int on);
/* Where the ring fills of step 2 run (results are the same bit for bit):
 * SWA_AMR_FILL_KERNEL (the default) in a kernel of its own before each
 * launch, one thread per ring cell; SWA_AMR_FILL_FUSED in the level launch
 * itself: each strip first writes the ring cells inside its own stencil
 * window (strips sharing a ring cell write the same value), and the
 * launch's refluxing fluxes form the ring cells they read from the fill map.
 * The fused form saves the kernel but puts the fills on the critical path
 * of the strips at patch edges; on levels with about one strip per resident
 * warp (latency-bound launches) it is slower.  Host state only. */
#define SWA_AMR_FILL_FUSED 0
#define SWA_AMR_FILL_KERNEL 1
int swa_amr_set_fill_mode(swa_amr *amr, int mode);
/* Sizes of hierarchy level `level`'s maps (1 .. nlevels): ring cells filled
 * per launch, covered parent cell copies averaged, coarse-fine edges
 * refluxed (any pointer may be null). */
int swa_amr_info(const swa_amr *amr, int level, int *nfill, int *navg, int *nedges);

/*
 * FP64 audit of the conserved mass of the grid's current state: writes
 * M = sum over interior cells of h dx dy (1D: h dx) to the device double
 * *mass_dev, summed in double whatever the storage precision (FP32:
 * h = (double) eta + (double) hbar), in a fixed order, so the same state
 * always gives the same bits.  Between walls the conservative update keeps
 * M constant (Eq. swe in conservation form); its drift measures the
 * rounding of the step.  Asynchronous on `stream`; it uses the grid's
 * reduction scratch, so issue it on the stream that steps the grid.
 * SWA_EINVAL for a null argument, SWA_ESTATE before the state is set,
 * SWA_ECUDA if a launch fails.
 */
int swa_grid_mass(const swa_grid *g, double *mass_dev, void *stream);

/* ============================ ALU peak probes =============================
 * Measurement aid (no counterpart in the paper): throughput probes of the
 * arithmetic units that bound the step kernels, so that the FP64 and FP32
 * rooflines are stated against peaks measured on the device at hand.
 *
 * swa_alu_probe launches `blocks` x `threads` threads (threads a multiple of
 * 32 in [32, 256]), each running 8 independent chains of `iters` operations
 * of one kind, on `stream`; sink_dev is a device float array of `blocks`
 * entries that is written only if a chain takes an impossible value (it
 * keeps the work from being optimised away).  Time the launch with CUDA
 * events and divide swa_alu_probe_ops(kind, blocks, threads, iters), the
 * operation count (flops for the FMA kinds: 2 per FMA, 4 per packed FMA;
 * 1 per reciprocal square root), by it.  SWA_EINVAL for a bad shape, a null
 * sink or an unknown kind; SWA_ECUDA if the launch fails.
 */
#define SWA_PROBE_FFMA64 0   /* fma.rn.f64 */
#define SWA_PROBE_FFMA32 1   /* fma.rn.f32 */
#define SWA_PROBE_FFMA32X2 2 /* fma.rn.f32x2 (packed pair) */
#define SWA_PROBE_RSQRT32 3  /* rsqrt.approx.ftz.f32 (special-function unit) */
double swa_alu_probe_ops(int kind, int blocks, int threads, int iters);
int swa_alu_probe(int kind, int blocks, int threads, int iters, float *sink_dev, void *stream);

/* ======================= allocation-free forward step =====================
 * The paper has no counterpart to this entry point; it is an integration aid.
 *
 * One forward step, as in swa_step_forward, for callers that cannot allocate
 * device memory: code whose device memory belongs to a host framework that
 * hands out only the arrays to work on, or that runs where cudaMalloc is not
 * allowed (a fixed memory budget, a region that must not synchronise the
 * device).  Such a caller cannot provide the per-block reduction scratch that
 * a grid workspace holds, so this call takes it from a fixed static device
 * array of SWA_STATIC_SCRATCH_BYTES inside the library (every GPU that loads
 * the library holds it until the process exits).  It allocates nothing.
 *
 * desc       grid descriptor (precision selects the storage layout below).
 * q_in[3]    current state, device, n values each, storage precision:
 *            SWA_FP64: (h, hu, hv) double; SWA_FP32: (eta, hu, hv) float.
 *            q_in[2] may be NULL for ndim = 1.
 * q_out[3]   new state after one step, same layout; must not alias q_in.
 * bath       device, n values: B (double) for SWA_FP64, hbar = -B (float)
 *            for SWA_FP32.
 * dt         the step (the caller chooses it, e.g. cfl / s_max).
 * smax_out_dev  optional device double receiving s_max of the new state,
 *            max over cells of max((|u|+c)/dx, (|v|+c)/dy) (the split
 *            step's CFL rule, as in swa_step_forward), for the next dt.
 * Errors: SWA_EINVAL for bad arguments; SWA_ENOMEM when the grid needs more
 * reduction slots than the static array holds (SWA_STATIC_MAX_BLOCKS blocks;
 * 2048 x 2048 fits in both precisions); SWA_ECUDA for a runtime failure.
 * All calls share the static array and it keeps the last call's contents;
 * each call resets what must start at zero with a one-thread kernel on
 * `stream` before its step kernel runs (no host memory is read, nothing
 * synchronises).  Calls whose kernels overlap on the GPU race on the array:
 * issue them on one stream.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) and caches it; make that first call
 * before any stream capture.  The cached address is not refreshed after a
 * cudaDeviceReset: do not reset a device while the library is in use.
 */
#define SWA_STATIC_MAX_BLOCKS 32768
#define SWA_STATIC_SCRATCH_BYTES (256 + 8 * SWA_STATIC_MAX_BLOCKS)
int swa_step_forward_static(const swa_grid_desc *desc, const void *const q_in[3],
                            void *const q_out[3], const void *bath, double dt,
                            double *smax_out_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SWADJ_H */
