/*
 * hlbm.h - C ABI of the GB300 hybrid lattice Boltzmann (HLBM) library.
 *
 * The library advances the coupled grid system of Di Ilio, Chiappini,
 * Ubertini, Bella and Succi ("Fluid flow around NACA 0012 airfoil at
 * low-Reynolds numbers with hybrid lattice Boltzmann method") on one GPU:
 *   - D2Q9 BGK lattice on nested Cartesian levels refined by a factor of two
 *     (Eq. 1, Eq. 2; Section 4 for the refinement boxes and outer conditions),
 *   - cell-vertex finite-volume LBE on a body-fitted triangular mesh with the
 *     airfoil wall condition (Eq. 3; Section 4),
 *   - the overlap interpolation between the two grids (Eq. 4-9),
 *   - the drag and lift coefficients (Eq. 10-11).
 *
 * Conventions used by every entry point:
 *   - All functions return an int status (HLBM_OK = 0, negative on error);
 *     hlbm_last_error(ctx) gives a message for the last failing call on ctx.
 *   - Pointers are plain host pointers unless stated otherwise; the library
 *     copies every input it needs, so the caller may free them on return.
 *   - Lengths are finest-level lattice units: the finest level has unit
 *     spacing and unit time step.  Flow enters along +x.
 *   - A context is not thread-safe; separate contexts are independent.
 */
#ifndef HLBM_H
#define HLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HLBM_OK 0
#define HLBM_EINVAL (-1)    /* invalid argument or geometry                    */
#define HLBM_ENOMEM (-2)    /* device or host allocation failed                */
#define HLBM_ECUDA (-3)     /* CUDA runtime error                              */
#define HLBM_EUNSTABLE (-4) /* NaN in the force reduction (simulation unstable) */
#define HLBM_ETIMEOUT (-5)  /* a device-side wait gave up                      */
#define HLBM_ESTATE (-6)    /* call not valid in the context's current state   */
#define HLBM_ENOTIMPL (-7)  /* feature not available in this build             */

#define HLBM_FP64 0 /* populations and arithmetic in double precision          */
#define HLBM_FP32 1 /* populations stored as f - w_i in float, float arithmetic */
#define HLBM_FP16S 2 /* lattice populations stored as 16-bit floats of (f - f^eq(1, u0)) / w_i
                        (shifted by the free stream), mesh state and arithmetic in float */

/* Node kinds of the triangular mesh. */
#define HLBM_NODE_FLUID 0
#define HLBM_NODE_WALL 1 /* airfoil surface: no-slip wall rule, force nodes      */
#define HLBM_NODE_RING 2 /* outer ring: unstructured interpolation node (Eq. 5)  */

/* One Cartesian level (Section 4: nested rectangular boxes, spacing halved
 * per level).  Level 0 is the coarsest and has ox = oy = 0.  Level l > 0 has
 * odd nx, ny; its node (i, j) sits at (ox + i/2, oy + j/2) in level l-1 node
 * units and the box lies at least two parent nodes inside its parent. */
typedef struct {
    int32_t nx, ny;
    int32_t ox, oy;
} hlbm_level;

/* The body-fitted triangular mesh (Section 4), in finest-level units and in
 * the zero-incidence pose.  xy: [n_nodes][2]; tri: [n_tri][3] counter-
 * clockwise node indices; kind: [n_nodes] HLBM_NODE_*.  pivot: rotation
 * centre (quarter chord).  hole: inner interface ellipse (cx, cy, a, b), axis
 * aligned in the zero-incidence pose; finest-level nodes inside it are not
 * computed.  n_nodes == 0 gives a plain channel (lattice only); chord is
 * always the length scale of Re and must be positive. */
typedef struct {
    int32_t n_nodes;
    const double *xy;
    int32_t n_tri;
    const int32_t *tri;
    const uint8_t *kind;
    double chord;
    double pivot[2];
    double hole[4];
} hlbm_mesh;

/* Options.  precision: HLBM_FP64 or HLBM_FP32.  n_sub: finite-volume
 * sub-steps per finest lattice step (Section 6.3 uses 10); 0 selects the
 * library's stability bound.  seed, perturb: initial density 1 + perturb*xi
 * with xi uniform in [-1, 1) from splitmix64(seed ^ (grid << 40) ^ node)
 * (grid = level index, 63 for the mesh).  force_cap: length of the device
 * ring buffer of force samples (one sample per coarse step; 0 -> 4096).
 * check_every: hlbm_step synchronises and reads the health flag every
 * check_every coarse steps (0 -> only at the end of each call).
 * stream: cudaStream_t to run on (NULL: the legacy default stream).
 * alloc/free/alloc_ctx: optional device allocator (e.g. PyTorch's caching
 * allocator); NULL alloc means cudaMalloc/cudaFree.  use_graphs: capture one
 * coarse step as a CUDA graph (1, default when the struct is zeroed is 0).
 * wall_stats: 1 adds to every coarse step the accumulation of the wall
 * coefficients read by hlbm_wall_stats (one small kernel over the wall
 * nodes); 0 leaves the step as it is.  fv_variant: variant of the FP32
 * finite-volume kernel: 0 times them on this mesh at create and keeps the
 * fastest (the autotuner: the four on 128-row tiles and, where those tiles
 * need more than two waves of 8 resident blocks per SM, the four on 256-row
 * tiles); 1-4 on tiles of 128 rows: 1 registers bounded
 * for 7 resident blocks per SM, 2 for 8, 3 and 4 the same with an L2
 * prefetch, by every block, of the entries and halo states of the tile that
 * starts about when it ends; 5-8 the same four on tiles of 256 rows (3 and 4
 * resident blocks per SM; HLBM_ECUDA if such a tile's staging does not fit in
 * shared memory).  Variants of one tile size give the same results; the two
 * tile sizes order each row's operator entries differently (FP32 rounding).
 * FP64 has one unbounded kernel on 128-row tiles and reports 1.
 * fv_filter: strength sigma in [0, 1] of an odd-even filter of the mesh state
 * applied once per finest step after the Eq. 3 sub-steps (an addition to the
 * paper's method, 0 = off, the default of a zeroed struct): with the graph
 * Laplacian of the Eq. 3 collision weights, (L g)_i(P) = sum_{k != P} C_Pk
 * [g_i(P_k) - g_i(P)], every fluid node takes g <- g - sigma L d with d = L g
 * on fluid nodes and 0 on wall and ring nodes, which keep their state.  On
 * smooth fields this is a hyper-diffusion of about (7/54)^2 sigma h^4 k^4 per
 * finest step (h the mesh spacing); it damps the node-to-node oscillations
 * that the central Eq. 3 fluxes neither advect nor damp and that otherwise
 * grow in long runs at Re 1000 (factor 1 - sigma (14/27)^2 per step on a
 * regular triangulation).
 * The adjoint entry points refuse contexts with fv_filter > 0. */
typedef struct {
    int32_t precision;
    int32_t n_sub;
    uint64_t seed;
    double perturb;
    int32_t force_cap;
    int32_t check_every;
    void *stream;
    void *(*alloc)(size_t bytes, void *alloc_ctx);
    void (*free)(void *ptr, void *alloc_ctx);
    void *alloc_ctx;
    int32_t use_graphs;
    int32_t wall_stats;
    int32_t fv_variant;
    double fv_filter;
} hlbm_options;

typedef struct hlbm_ctx hlbm_ctx;

/* Create a simulation.  lv: [n_levels] levels (1 <= n_levels <= 8); m: the
 * mesh (may have n_nodes == 0); Re = u0 C / nu with u0 = Ma c_s, c_s^2 = 1/3;
 * aoa_deg: angle of attack, applied as a rotation of mesh and hole by -aoa
 * about the pivot (positive = nose up).  Copies every input, computes all
 * set-up tables on the host (Eq. 3 operators, Eq. 8 and Eq. 9 stencils,
 * refinement maps), uploads them and initialises the state.  On error *out is
 * NULL and the message is available via hlbm_last_error(NULL). */
int hlbm_create(const hlbm_level *lv, int n_levels, const hlbm_mesh *m, double Re, double Ma,
                double aoa_deg, const hlbm_options *opt, hlbm_ctx **out);

/* Advance n_coarse coarse (level-0) steps, asynchronously on the context's
 * stream.  One coarse step runs 2^l steps of level l and, per finest step,
 * n_sub finite-volume sub-steps; one force sample is recorded per coarse
 * step.  Every check_every coarse steps (option) it reads the health flag
 * and the total mass of level 0 (FP64 reduction, outside the step graph):
 * HLBM_ETIMEOUT if a bounded device-side wait gave up, HLBM_EUNSTABLE if the
 * forces held a NaN or the mass moved by more than 1e-2 of its value at
 * create (the open boundaries let it change a little in a healthy run). */
int hlbm_step(hlbm_ctx *ctx, int n_coarse);

/* Copy the force samples recorded since the previous call (oldest first, at
 * most cap of them, FP64) into host arrays cd[], cl[] (Eq. 10-11: force over
 * 1/2 rho0 u0^2 C).  *n_written receives the count.  Samples older than
 * force_cap coarse steps are lost.  Synchronises the stream. */
int hlbm_forces(hlbm_ctx *ctx, double *cd, double *cl, int cap, int *n_written);

/* Density and velocity of one grid into host FP64 arrays of cap entries:
 * grid = -1 for the mesh (n_nodes entries, input node order) or a level
 * index (nx*ny entries, x fastest).  Nodes that are not computed (inside the
 * hole) get NaN.  Synchronises the stream. */
int hlbm_fields(hlbm_ctx *ctx, int grid, double *rho, double *ux, double *uy, size_t cap);

/* Populations f_i (not deviations) of one grid into a host FP64 array of
 * cap entries, node-major: out[9 * node + i], D2Q9 order
 * (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1). */
int hlbm_populations(hlbm_ctx *ctx, int grid, double *out, size_t cap);

/* Scalar information: "n_sub", "n_levels", "tau_u", "tau0".."tau7", "steps",
 * "n_interp" (structured interpolation nodes), "n_ring", "n_wall_edges",
 * "nnz" (Eq. 3 operator entries, self entries included),
 * "lattice_updates" (computed lattice node updates per coarse step),
 * "fv_updates" (finite-volume node updates per coarse step),
 * "launches_per_step" (kernels in one coarse step), "fv_bytes" (algorithmic
 * bytes of one finite-volume sub-step), "collide_bytes<l>" (algorithmic bytes
 * of one lattice step of level l), "fv_tiles" (blocks of one finite-volume
 * sub-step), "fv_tile_rows" (rows per tile, 128 or 256), "fv_smem" (their
 * dynamic shared memory, bytes), "fv_variant" (the variant in use, 1-8, see
 * options), "fv_tune_us1" .. "fv_tune_us8" (the autotuner's launch times of
 * the eight variants, 0 if it did not run or a tile size was not built),
 * "create_ms_setup", "create_ms_device", "create_ms_capture" (wall time of
 * hlbm_create's host set-up tables, device build with uploads, initial
 * state and autotuning, and graph capture, in ms; the device build splits
 * into "create_ms_upload", device tables and copies, and "create_ms_init",
 * initial state and autotuner),
 * "mass" (total mass of level 0 now, sum of rho over its computed nodes,
 * FP64), "mass_drift" (its relative change since create); these two
 * synchronise the stream.  "bounds_violations", "bounds_sites": in a library
 * built with index bounds checks (HLBM_DEBUG), the number of out-of-range
 * indices the kernels met so far in this process and the bit mask of where
 * (1 lattice level, 2 mesh state, 4 a tile's staged nodes, 8 operator
 * entries, 16 a band snapshot); the access went to index 0 instead.  -1 in a
 * build without checks; these two synchronise the device. */
int hlbm_info(const hlbm_ctx *ctx, const char *key, double *value);

/* Measurement hook: runs one kernel of the step `reps` times back to back on
 * the context's stream (kernel = "fv" for the Eq. 3 sub-step, "collide<l>" for
 * the Eq. 1 step of level l) and returns the mean duration from CUDA events.
 * The kernels really update the state, so afterwards the context only serves
 * readback and hlbm_destroy (hlbm_step returns HLBM_ESTATE). */
int hlbm_time_kernel(hlbm_ctx *ctx, const char *kernel, int reps, double *avg_ms);

/* Host-only set-up (no GPU needed): runs the same set-up as hlbm_create and
 * copies the named table into out (cap doubles); *n receives its length.
 * Tables: "rowptr", "col", "sx", "sy", "cc" (Eq. 3 operators, CSR over the
 * input node order, columns ascending), "area", "xy" (rotated),
 * "is_node", "is_don", "is_w" (Eq. 8 stencils), "ring", "ring_don",
 * "ring_w" (Eq. 9 stencils), "wall_edges", "n_sub", "inactive<l>" (1 for
 * nodes of level l that are not computed), "perm" (input node of each device
 * row), "wall_geo" ([n_wall][7]: x/C, side, |N_P|, n_x, n_y, s_x, s_y of the
 * wall nodes, see hlbm_wall_stats).  out == NULL queries n. */
int hlbm_inspect(const hlbm_level *lv, int n_levels, const hlbm_mesh *m, double Re, double Ma,
                 double aoa_deg, const hlbm_options *opt, const char *table, double *out,
                 size_t cap, size_t *n);

/* Drag and lift coefficients of one mesh state held by the caller, computed
 * without allocating any device memory.  The paper has no counterpart: this
 * is for callers that cannot call cudaMalloc (their device memory belongs to
 * another framework's pool, or they evaluate forces inside loops that must not
 * allocate); the force reduction's per-block partial sums live in a fixed
 * file-scope device array instead.
 * All pointers are device pointers: f [n_nodes][9] FP64 populations (D2Q9
 * order of hlbm_populations), xy [n_nodes][2] node coordinates (finest-level
 * units, the pose the forces refer to), edge_a/edge_b [n_edges] wall edges
 * a -> b with the fluid on their left (indices in [0, n_nodes)), out [2]
 * receives (C_D, C_L) = F / qdyn with qdyn = rho0 u0^2 C / 2 (Eq. 10-11).
 * Runs asynchronously on `stream` (cudaStream_t, NULL = legacy default).
 * Limits: n_edges <= 131072, else HLBM_EINVAL (message via
 * hlbm_last_error(NULL)).  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) for that device, so make that first
 * call before any stream capture; the address is kept for the life of the
 * process, so it does not survive cudaDeviceReset (do not call this entry
 * point on a device after resetting it).  Every call shares the array and it
 * keeps the last call's partial sums; each call writes every slot it reads,
 * but calls that overlap on the GPU race and must be ordered.  An edge whose
 * end point lies outside [0, n_nodes) is skipped without reading f or xy, and
 * the call then writes NaN to both outputs (it still returns HLBM_OK: the
 * indices live on the device and are checked there). */
int hlbm_wall_forces_static(const double *f, int n_nodes, const double *xy, const int32_t *edge_a,
                            const int32_t *edge_b, int n_edges, double qdyn, double *out, void *stream);

/* Mean pressure and skin-friction coefficients along the wall (Eq. 12-13:
 * C_p = (p - p0) / (rho0 u0^2 / 2), C_f = tau_w / (rho0 u0^2 / 2), with
 * p = rho / 3, p0 = 1/3, rho0 = 1), averaged over the coarse steps since
 * hlbm_create or hlbm_wall_stats_reset (one sample at the end of each coarse
 * step; needs options.wall_stats = 1, else HLBM_ESTATE).  Wall node P
 * carries N_P = half the sum of its wall edges' normals times length (into the
 * fluid), so that the force of Eq. 10-11 is exactly sum_P [-(p - p0) N_P -
 * Pi^neq N_P]; with n = N_P / |N_P| and s the unit tangent pointing
 * downstream along the chord, the viscous traction -Pi^neq n = c_n n +
 * tau_w s.  out receives, per wall node in ascending input index, 10 doubles
 * (x/C from the leading edge in the body frame, side (+1 upper, -1 lower
 * surface), mean C_p, mean C_f, mean C_n = c_n / q, |N_P|, n_x, n_y, s_x,
 * s_y), so sum_P |N_P| [(-C_p + C_n) n + C_f s] / C is the mean (C_D, C_L).
 * cap is the capacity of out in doubles; *n_wall receives the wall node
 * count and *n_samples the number of coarse steps averaged.  out == NULL
 * queries the sizes.  Accumulation is FP64 in every precision. */
int hlbm_wall_stats(hlbm_ctx *ctx, double *out, size_t cap, int *n_wall, long *n_samples);
/* Restart the averages of hlbm_wall_stats from the next coarse step. */
int hlbm_wall_stats_reset(hlbm_ctx *ctx);

/* Discrete adjoint of the finite-volume part of the step (Eq. 3 sub-steps,
 * the wall rule, Eq. 10-11), FP64 contexts only.
 *
 * The window: starting from the context's current mesh state, n_window
 * consecutive sub-steps (1 <= n_window <= n_sub) of a finest step, each the
 * Eq. 3 update of every mesh node followed by the wall rule, with the
 * interface rows set after each sub-step but the last of a finest step from
 * the current Eq. 9 interface data (the lattice state now, held fixed), then
 *   J = (wd F_x + wl F_y) / (1/2 rho0 u0^2 C)
 * of the final mesh state, i.e. wd C_D + wl C_L of Eq. 10-11.  The window is
 * run on scratch buffers: the context's state and force series do not change.
 *
 * Outputs: *J; if grad_g is not NULL, dJ/dg of the window's initial mesh
 * state in populations, [n_nodes][9] in input node order and D2Q9 order
 * (cap_g >= 9 n_nodes); if grad_coef is not NULL, dJ/d(s_x, s_y, C) of every
 * Eq. 3 operator entry, [nnz][3] in the order of the "rowptr" / "col" tables
 * of hlbm_inspect (cap_coef >= 3 nnz).  Self entries (P, P) get 0: their
 * streaming coefficient is eliminated by the closed control volume
 * (sum_k s_Pk = 0) and C_PP = 11/18 is fixed.  If grad_xy is not NULL,
 * dJ/dx of the mesh node coordinates, [n_nodes][2] in input node order and
 * in the input frame (the pose before the rotation by the angle of attack),
 * through the Eq. 3 operators (their closed-form assembly from the
 * triangles) and the wall-edge normals of Eq. 10-11, the state and the
 * interface data held (cap_xy >= 2 n_nodes); if dJ_daoa is not NULL, dJ/d
 * (angle of attack) per degree through the same pose change.  Scratch:
 * (n_window + 3) x 9 x n_nodes doubles and a few per-node arrays, allocated
 * and freed by the call through the context's allocator.  Synchronises the
 * context's stream.  Errors: HLBM_ENOTIMPL (not FP64), HLBM_EINVAL (no
 * mesh, n_window out of range, capacities), HLBM_ESTATE, HLBM_ENOMEM,
 * HLBM_ECUDA. */
/* Discrete adjoint of n_steps whole coarse steps (FP64 contexts with a
 * mesh): on every level the Eq. 1 collide-stream, the outer conditions
 * (level 0), the band snapshots, the prolongation with its time and space
 * interpolation and the restriction of the refinement interfaces; on the
 * finest level the Eq. 4 + 8 hole nodes, the Eq. 9 interface data with the
 * Eq. 5-7 interface rows at their sub-step times, the Eq. 3 sub-steps with
 * the wall rule; and the force of every coarse step:
 *   J = 1/(n_steps - n_skip) sum_{k = n_skip .. n_steps-1} (wd C_D(k) + wl C_L(k)),
 * the mean of the last n_steps - n_skip of the n_steps force samples that
 * hlbm_step would record from the current state (0 <= n_skip < n_steps; the
 * first n_skip steps are differentiated through, their forces not averaged).  The forward steps run on scratch copies (the context's
 * state and force series do not change).  Recomputation checkpointing: the
 * state at every ceil(sqrt(n_steps))-th step start is kept, each segment is
 * re-run once keeping its step starts, and each step once more while its
 * level steps' states are recorded for the reverse sweep.  Outputs: *J; if
 * grad_lattice is not NULL, dJ/d(lattice populations) of the current state,
 * level after level, each [ny][nx][9] (cap_lat >= 9 sum_l nx_l ny_l; 0 on
 * nodes that are not computed); if grad_mesh is not NULL, dJ/d(mesh
 * populations), [n_nodes][9] in input node order (cap_mesh >= 9 n_nodes; 0
 * on interface rows, which are overwritten before they are read); if
 * grad_xy is not NULL, dJ/dx of the mesh node coordinates, [n_nodes][2] in
 * input node order and frame (cap_xy >= 2 n_nodes), and if dJ_daoa is not
 * NULL, dJ/d(angle of attack) per degree: through the Eq. 3 operators, the
 * wall normals, the Eq. 8 weights (donor positions) and the Eq. 9 weights
 * (interface node positions), with the initial state held, the discrete
 * choices (containing triangles, donor blocks, hole nodes) held and the
 * lattice fixed in space.  Scratch:
 * about 2 sqrt(n_steps) + 2 copies of the whole state plus one coarse step's
 * records, allocated and freed through the context's allocator.
 * Synchronises the context's stream.  Errors: HLBM_ENOTIMPL (not FP64),
 * HLBM_EINVAL (no mesh, n_steps < 1, capacities), HLBM_EUNSTABLE (NaN in a
 * forward force), HLBM_ESTATE, HLBM_ENOMEM, HLBM_ECUDA. */
int hlbm_adjoint(hlbm_ctx *ctx, int n_steps, int n_skip, double wd, double wl, double *J, double *grad_lattice,
                 size_t cap_lat, double *grad_mesh, size_t cap_mesh, double *grad_xy, size_t cap_xy, double *dJ_daoa);

int hlbm_fv_adjoint(hlbm_ctx *ctx, int n_window, double wd, double wl, double *J, double *grad_g, size_t cap_g,
                    double *grad_coef, size_t cap_coef, double *grad_xy, size_t cap_xy, double *dJ_daoa);

/* Batched ensemble: many independent cases (angles of attack, Reynolds
 * numbers, mesh sizes) advanced together.  The paper runs its angle-of-attack
 * and Reynolds sweeps (Section 5) as separate simulations; a batch runs them
 * side by side on one GPU.  hlbm_batch_create takes n contexts made by
 * hlbm_create with use_graphs = 1 on the current device (the batch keeps
 * pointers to them: they must outlive it) and builds two CUDA graphs, one per
 * step parity, in which each context's coarse-step graph is a child graph on
 * its own branch, with no dependency between cases; hlbm_batch_step then
 * advances every case by one coarse step per graph launch, on `stream` (NULL:
 * a stream of the batch's own), and the GPU runs the cases' kernels
 * concurrently.  Each case's results are bitwise those of hlbm_step on it
 * alone (the same kernels in the same order).  The batch stream first waits
 * for the contexts' own streams, and the contexts' streams then wait for the
 * batch, so readback with hlbm_fields / hlbm_forces orders after it.  A
 * context stepped on its own after hlbm_batch_create (or consumed by
 * hlbm_time_kernel) makes hlbm_batch_step return HLBM_ESTATE.  If any context
 * has check_every > 0, hlbm_batch_step synchronises at the end and returns
 * HLBM_ETIMEOUT / HLBM_EUNSTABLE if a case's health flag is set (the message
 * names the case).  Errors: HLBM_EINVAL (no contexts, a NULL or repeated
 * context, a context without graphs), HLBM_ECUDA. */
typedef struct hlbm_batch hlbm_batch;
int hlbm_batch_create(hlbm_ctx *const *ctxs, int n, void *stream, hlbm_batch **out);
int hlbm_batch_step(hlbm_batch *b, int n_coarse);
int hlbm_batch_sync(hlbm_batch *b);
/* Message of the batch's last error (b == NULL: the last failing create). */
const char *hlbm_batch_last_error(const hlbm_batch *b);
/* Releases the batch (not its contexts). */
int hlbm_batch_destroy(hlbm_batch *b);

/* Checkpoint / resume.  hlbm_save writes every array that carries state from
 * one coarse step to the next (all lattice levels, the current mesh state,
 * the interface data at t and the band snapshots, the force samples and
 * counters, the wall-statistics sums) and the step counters to `path` (a
 * magic string, a JSON header with the configuration and the buffer sizes,
 * then the raw little-endian buffers).  hlbm_load reads such a file into a
 * context created from the same inputs (levels, mesh size, precision,
 * sub-steps, force_cap, wall_stats; otherwise HLBM_EINVAL, context unchanged)
 * and stepping it on is bitwise identical to the run that was saved.  Both
 * synchronise the stream; errors: HLBM_EINVAL (path, format, mismatch),
 * HLBM_ESTATE (save after hlbm_time_kernel), HLBM_ECUDA. */
int hlbm_save(hlbm_ctx *ctx, const char *path);
int hlbm_load(hlbm_ctx *ctx, const char *path);

/* Wait for all work of the context. */
int hlbm_sync(hlbm_ctx *ctx);

/* Release the context and its device memory. */
int hlbm_destroy(hlbm_ctx *ctx);

/* Message of the last error on ctx (ctx == NULL: the last failing create or
 * inspect on this thread). */
const char *hlbm_last_error(const hlbm_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* HLBM_H */
