/*
 * apm.h -- C ABI of libapm: the adaptive particle-mesh (APM) gravity level
 * solve of Passy & Bryan, "An adaptive particle-mesh gravity solver for ENZO"
 * (arXiv:1410.0010), on NVIDIA GB300 (sm_103a).
 *
 * One APM solve over a static hierarchy of nested grids runs, level by level
 * from the root down (Sec. 2 and Sec. 2.2):
 *
 *   apm_deposit      particles drifted half a step, TSC-deposited, plus baryons,
 *                    into each grid's gravitating-mass field (GMF)
 *   apm_solve_level  per-grid FFT convolution with the APM Green's function
 *                    (periodic or isolated root, short-range on refined levels)
 *   apm_accel        finite-difference accelerations plus the potential and
 *                    acceleration carried (interpolated) from the parent grid
 *   apm_interp       TSC interpolation of the accelerations back to particles
 *
 * Conventions (all entry points):
 *  - Every array argument is a DEVICE pointer unless stated otherwise; the
 *    caller owns it.  Per-grid arguments are HOST arrays of device pointers,
 *    one entry per grid of the level, in the order the grids appear in the
 *    hierarchy passed to apm_set_hierarchy.
 *  - 3-D fields are x-fastest: cell (x, y, z) of an (nx, ny, nz) box is at
 *    x + nx * (y + ny * z).  Vector fields are 3 consecutive components
 *    (structure of arrays) in one allocation.
 *  - Floating-point fields (phi_short, phi, acc, acc_out) are float when the
 *    context's precision is APM_FP32 and double for APM_FP64.
 *  - `stream` is a cudaStream_t (NULL: the legacy default stream).  Calls are
 *    asynchronous on it; calls on one context must be ordered (one stream, or
 *    synchronised by the caller).  A context is not thread-safe.  Within a
 *    call, an FFT pass whose grids run different kernels spreads them over the
 *    context's three auxiliary streams, forked from `stream` and joined back
 *    to it with events: the work stays ordered on `stream`, and a capture of
 *    `stream` takes the branches in.
 *  - Errors detectable on the host are returned immediately and nothing is
 *    enqueued.  Errors the kernels detect (fixed-point overflow, a particle
 *    outside an isolated box, a wait that ran out) are latched in a device
 *    status word and returned by apm_sync_status.
 *  - No entry point allocates device memory after apm_set_hierarchy, and no
 *    entry point other than apm_sync_status synchronises the stream.
 */
#ifndef APM_H
#define APM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    APM_OK = 0,
    APM_E_INVALID = 1,     /* bad argument (NULL, size, level out of range) */
    APM_E_NESTING = 2,     /* hierarchy violates the nesting rules */
    APM_E_NOMEM = 3,       /* device or pinned allocation failed */
    APM_E_CUDA = 4,        /* a CUDA runtime call failed */
    APM_E_OVERFLOW = 5,    /* |m 2^F| >= 2^62 for some particle (it was skipped) */
    APM_E_OUT_OF_BOX = 6,  /* particle outside an isolated root (folded to its edge) */
    APM_E_TIMEOUT = 7,     /* a bounded device wait ran out */
    APM_E_UNSUPPORTED = 8, /* valid request the library does not implement */
    APM_E_STATE = 9,       /* call out of order (e.g. no hierarchy set) */
    APM_E_BOUNDS = 10      /* a checked device access was out of range (only in
                              libraries built with -DAPM_BOUNDS_CHECK) */
} apm_status;

typedef enum { APM_FP32 = 0, APM_FP64 = 1 } apm_precision;
typedef enum { APM_BC_ISOLATED = 0, APM_BC_PERIODIC = 1 } apm_bc;

/* Gradient operator D (Sec. 2.2: the influence function Eq. influence is built
 * for the operator the accelerations use; the paper allows a finite difference
 * or the direct Fourier-space gradient D = -ik):
 *  APM_GRAD_FD2      two-point centred difference, D_j = sin(k_j delta)/delta;
 *                    A_j(c) = -(phi(c+1) - phi(c-1)) / (2 delta)
 *  APM_GRAD_FD4      four-point difference,
 *                    D_j = (8 sin(k_j delta) - sin(2 k_j delta)) / (6 delta);
 *                    A_j(c) = -(8 (phi(c+1) - phi(c-1)) - (phi(c+2) - phi(c-2))) / (12 delta);
 *                    an isolated root then needs an even FFT length >= 2 N0 + 2,
 *                    so N0 <= 511 (APM_E_UNSUPPORTED above)
 *  APM_GRAD_SPECTRAL D_j = k_j (0 on the Nyquist mode of an even M_j); the
 *                    short-range accelerations are transformed back from
 *                    -i D_j T rho-hat, one inverse transform per component. */
typedef enum { APM_GRAD_FD2 = 0, APM_GRAD_FD4 = 1, APM_GRAD_SPECTRAL = 2 } apm_gradient;

/* Method parameters.  Defaults (apm_config_default) are the paper's:
 * a = 3.4 delta_l and R = 2 (Sec. 2.2), padding factor 0.65 (Sec. 2.2),
 * isolated root (Sec. 3), FP32 field arithmetic, 52 fraction bits. */
typedef struct {
    double box;              /* side of the cubic domain [0, box)^3 */
    double a_over_dx;        /* smoothing diameter a_l / delta_l (Sec. 2.2: 3.4) */
    int32_t refine;          /* refinement factor R between levels (Sec. 2.2: 2) */
    double pad_factor;       /* extra cells 0.65 R a/delta (Sec. 2.2): border B =
                                ceil(pad_factor * refine * a_over_dx) cells per side */
    int32_t root_bc;         /* apm_bc of the root grid */
    int32_t precision;       /* apm_precision of FFT, multiply and gradient */
    int32_t mass_frac_bits;  /* F: GMF cells hold mass * 2^F as int64, 1 <= F <= 62 */
    int32_t root_correction; /* isolated root: 1 adds the k-space optimal correction
                                to the real-space kernel (see apm_set_hierarchy) */
    int32_t device;          /* CUDA device ordinal of the context; -1: current device */
    int32_t gradient;        /* apm_gradient (default APM_GRAD_FD2) */
} apm_config;

/* One grid.  start: global level-`level` cell index of the first interior cell
 * (cell i of level l covers [i, i+1) * box / (N0 R^l)); dims: interior cells.
 * Grid 0 must be the root: level 0, parent -1, start 0, dims (N0, N0, N0). */
typedef struct {
    int32_t level;
    int32_t parent;       /* index of the parent grid in the hierarchy array */
    int64_t start[3];
    int32_t dims[3];
} apm_grid;

/* Particles: device structure of arrays of n doubles each (positions in
 * [0, box), velocities, masses).  The arrays are only read. */
typedef struct {
    int64_t n;
    const double *x, *y, *z, *vx, *vy, *vz, *m;
} apm_particles;

/* Derived sizes of one grid (apm_get_grid_info). */
typedef struct {
    int32_t level;
    int32_t border;       /* B: GMF border cells per side (0 on the root) */
    int32_t gmf[3];       /* GMF box: dims + 2B (root: dims) */
    int32_t fft[3];       /* FFT lengths M (isolated root 2 N0, or with APM_GRAD_FD4
                             the smallest even {2,3,5,7}-smooth >= 2 N0 + 2;
                             periodic root N0; refined: smallest
                             {2,3,5,7}-smooth >= dims + 4B) */
    int32_t phi_short[3]; /* dims + 2h: cells [-h, dims+h), h = 3 for APM_GRAD_FD4,
                             else 2 */
    int32_t field[3];     /* dims + 2: cells [-1, dims+1) of phi and each acc component */
    int32_t level_index;  /* position of the grid among the grids of its level */
    double delta;         /* cell size box / (N0 R^level) */
    int32_t phi_short_comps; /* components of phi_short: 1, or 4 (phi, A_x, A_y, A_z
                                short-range) for APM_GRAD_SPECTRAL */
} apm_grid_info;

typedef struct apm_ctx apm_ctx;

/* Fills the paper's defaults (see apm_config). */
void apm_config_default(apm_config* cfg);

/* Creates a context on cfg->device (or the current device).  Allocates only
 * the status word.  Returns APM_E_INVALID for out-of-range parameters,
 * APM_E_UNSUPPORTED for a refinement factor other than 2, APM_E_CUDA when no
 * usable device is present. */
apm_status apm_create(const apm_config* cfg, apm_ctx** out);

/* Sets the static hierarchy (Sec. 3: a tree of nested grids, all grids of one
 * resolution on one level) and prepares everything the solves need:
 *  - validates the tree: levels 0..L each non-empty, every child's parent on the
 *    level above, sibling interiors disjoint, and every parent cell a child
 *    reads (its GMF border, Sec. 2, and the trilinear carry of its cells
 *    [-1, dims]) inside the parent's interior; otherwise APM_E_NESTING.  On an
 *    isolated root the GMF border of a level-1 grid may extend past the box:
 *    nothing lies outside an isolated domain, so its baryons there are zero
 *    (the carry must still stay inside the root);
 *  - plans each grid's border B and FFT lengths M (FFT lengths up to 1024);
 *  - builds on the GPU, in FP64, the Green's-function table of every distinct
 *    (grid type, M) (Sec. 2.2 Eq. influence with the Brillouin sum of
 *    Eq. brillouin truncated to n in [-1,1]^3, Eq. assignment, assignment2 and
 *    reference with the TSC assignment function and the two-point FD gradient;
 *    refined levels use the short-range reference force, the periodic root
 *    sets the k = 0 mode to 0 (mean removed, Sec. 3.4), the isolated root
 *    transforms the real-space S-S pair potential on the doubled grid,
 *    Sec. 2.1, plus the optimal correction when cfg.root_correction), cached
 *    per shape (Sec. 2.2, last paragraph), with an FP32 copy;
 *  - allocates the FFT workspace and particle lookup tables.
 * grids: HOST array of n_grids descriptors.  May be called again to replace
 * the hierarchy (frees the previous one; synchronises the device). */
apm_status apm_set_hierarchy(apm_ctx* ctx, const apm_grid* grids, int32_t n_grids);

/* Checks a hierarchy against the rules of apm_set_hierarchy without touching
 * the GPU (host only): APM_OK, APM_E_INVALID (malformed descriptors or
 * config) or APM_E_NESTING. */
apm_status apm_validate_hierarchy(const apm_config* cfg, const apm_grid* grids, int32_t n_grids);

/* Derived sizes of grid `grid` (index into the hierarchy array). */
apm_status apm_get_grid_info(const apm_ctx* ctx, int32_t grid, apm_grid_info* out);

/* Number of levels of the current hierarchy (0 if none). */
int32_t apm_num_levels(const apm_ctx* ctx);

/* Gravitating-mass field of every grid of `level` (Sec. 2):
 *  gmf[c] = sum over particles of rint((m w) 2^F) + rint((rho delta^3) 2^F)
 * with w the TSC weight (27 cells, Sec. 2) of the particle position drifted by
 * x + v * half_dt (Sec. 2, time-centred density); the centre cell of each
 * particle receives rint(m 2^F) minus its other 26 charges, so integer mass is
 * conserved exactly and the sums are independent of particle order.  Every
 * particle whose cloud touches a grid's GMF box contributes (the modified
 * deposit of Sec. 2: particles of the grid, its parent and the parent's
 * siblings alike).  Cloud cells outside a refined grid's GMF box are dropped;
 * on an isolated root they fold into the edge cell; on a periodic root they
 * wrap.  Baryons: interior cells take gas[g] (density, dims^3 doubles);
 * border cells take the parent cell's density from parent_gas (the parent's
 * baryons copied onto the boundary, Sec. 2).
 *  particles : device particle arrays (all particles of the simulation)
 *  gas       : HOST array (grids of the level) of device pointers to dims^3
 *              doubles, or NULL for no baryons; entries may be NULL
 *  parent_gas: HOST array (grids of level-1) of device pointers to the parent
 *              grids' interior densities, or NULL (no baryons in the border)
 *  gmf       : HOST array (grids of the level) of device pointers to int64 GMF
 *              boxes (apm_grid_info.gmf), fully overwritten
 * Sums are exact modulo 2^64 (exact whenever each cell's true sum fits). */
apm_status apm_deposit(apm_ctx* ctx, int32_t level, const apm_particles* particles,
                       double half_dt, const double* const* gas,
                       const double* const* parent_gas, int64_t* const* gmf, void* stream);

/* apm_deposit for every level of the hierarchy at once: the baryons of each
 * level as apm_deposit (parent gas on the borders), then one pass over the
 * particles that converts each position and mass once and deposits it level
 * by level from the root down while it is a candidate of the level.  The
 * fields are bit-identical to apm_deposit level by level.  Not in the paper:
 * a batching of its per-level deposits.
 *  gas : HOST array of n_grids device pointers in hierarchy order (dims^3
 *        densities, NULL entries for no gas), or NULL for no baryons at all
 *  gmf : HOST array of n_grids device pointers in hierarchy order (the GMF
 *        box of each grid), fully overwritten */
apm_status apm_deposit_all(apm_ctx* ctx, const apm_particles* particles, double half_dt,
                           const double* const* gas, int64_t* const* gmf, void* stream);

/* Short-range (refined level) or full (root) potential of every grid of
 * `level` (Sec. 2.2, Eq. PoissonFourier with Eq. influence): the GMF cell
 * masses (gmf * 2^-F, converted in FP64) are zero-padded onto the grid's M
 * grid, transformed, multiplied by the Green's table, transformed back, and
 * the window of cells [-h, dims+h) is written:
 *  phi_short: HOST array (grids of the level) of device pointers to
 *             comps x (dims+2h)^3 floats/doubles (apm_grid_info.phi_short,
 *             phi_short_comps; h = 3 for APM_GRAD_FD4, else 2).  With
 *             APM_GRAD_SPECTRAL the components are phi_short and the
 *             short-range accelerations A_x, A_y, A_z, each the inverse
 *             transform of -i D_j T rho-hat.
 * The FFTs are hand-written mixed-radix Stockham passes (radices 2-8; the
 * FP32 path also 6, 9, 10, 12, 14, 15, 16 in registers), five launches: x
 * forward, y forward, z forward + table + z inverse, y inverse, x inverse
 * (the last three once per component). */
apm_status apm_solve_level(apm_ctx* ctx, int32_t level, const int64_t* const* gmf,
                           void* const* phi_short, void* stream);

/* Accelerations and carried potential on cells [-1, dims+1) of every grid of
 * `level` (Sec. 2.2: difference the potential, then add the parent's
 * acceleration interpolated onto the refined grid):
 *   phi      = phi_short + I(parent phi)
 *   acc_j    = -(phi_short(c + e_j) - phi_short(c - e_j)) / (2 delta) + I(parent acc_j)
 * with I the trilinear interpolation from parent cell centres, in FP64.  With
 * APM_GRAD_FD4 the difference is the four-point one, with APM_GRAD_SPECTRAL
 * the short-range term is the solve's A_j component (see apm_gradient).
 *  parent_phi, parent_acc: HOST arrays (grids of level-1) of the parent level's
 *             phi / acc outputs, or NULL at level 0 (no parent term)
 *  phi      : HOST array of device pointers to (dims+2)^3 values
 *  acc      : HOST array of device pointers to 3 (dims+2)^3 values (x, y, z) */
apm_status apm_accel(apm_ctx* ctx, int32_t level, const void* const* phi_short,
                     const void* const* parent_phi, const void* const* parent_acc,
                     void* const* phi, void* const* acc, void* stream);

/* Launch granularity of apm_solve_level and apm_accel.  batched = 1 (the
 * default): each FFT pass, and the acceleration kernel, is one launch over
 * every grid of the level.  batched = 0: one launch sequence per grid, grid
 * after grid, which is how the paper's implementation runs the level (Sec. 2.2:
 * one FFT convolution per grid); kept as the plain per-grid baseline the
 * batched launches are measured against.  Every grid runs the same kernels on
 * the same work items either way, so the results are bit-identical.
 * APM_E_INVALID for a value other than 0 or 1. */
apm_status apm_set_grid_batching(apm_ctx* ctx, int32_t batched);

/* CUDA graphs of call sequences, owned by the context.  The paper has no
 * counterpart: replaying a recorded launch sequence removes the host cost of
 * each launch, which is what lets a level of many uneven grids (one work list
 * per pass, several segments) run as one replayed sequence.
 * apm_graph_begin starts capturing the work issued to `stream` (a stream the
 * caller created; the legacy default stream cannot be captured): this
 * library's calls and anything else the caller enqueues there.
 * apm_graph_end ends the capture, instantiates it and returns its id;
 * apm_graph_launch replays it on a stream; apm_graph_destroy frees it.
 * A replay repeats every captured launch with the same arguments, on the same
 * device buffers, so their contents at replay time are what it reads.  Make
 * the sequence's calls once outside capture first (its pointer tables are then
 * uploaded), and capture no call that synchronises (apm_sync_status,
 * apm_autotune_level, apm_set_fft_shapes, apm_reserve_order): the capture
 * then fails and apm_graph_end returns APM_E_STATE.  apm_set_hierarchy and
 * apm_destroy free every graph.  APM_E_STATE from apm_graph_begin without a
 * hierarchy or while `stream` is already capturing; APM_E_INVALID for a NULL
 * stream or an unknown id. */
apm_status apm_graph_begin(apm_ctx* ctx, void* stream);
apm_status apm_graph_end(apm_ctx* ctx, void* stream, int32_t* graph_id);
apm_status apm_graph_launch(apm_ctx* ctx, int32_t graph_id, void* stream);
apm_status apm_graph_destroy(apm_ctx* ctx, int32_t graph_id);

/* Particle processing order.  The paper has no counterpart: this is a property
 * of the GPU launch, not of the method.  The interpolation kernels run one
 * thread per particle; when consecutive particles are far apart in space, a
 * warp's 27-cell gathers touch as many cache lines as it has particles.
 * apm_order_particles sorts the particle indices by a root-level bin of their
 * drifted positions (cubes of 4 or more root cells, at most 128^3 bins; a
 * counting sort: one pass computing bins and ranks with atomics, a scan of
 * the bin counts, one scatter), and every later interpolation call
 * (apm_interp, apm_interp_all) on the same number of particles visits them in
 * that order.  The deposits keep the caller's order (in bin order neighbouring
 * threads add into the same cells and their reductions serialise), unless
 * apm_set_deposit_tiles(1) gathers each CTA's charges in shared memory.  The order
 * never changes a result: each particle is interpolated on its own, so every
 * output is bit-identical with or without it, and with an order computed
 * from other positions (after a kick-drift, say) the results stay exact, only
 * less coherent in memory.
 *
 * apm_reserve_order allocates the workspace for up to n_max particles (16 bytes
 * per particle plus the bin counts; a set-up call that synchronises the
 * device), or frees it and turns the ordering off for n_max = 0.
 * apm_set_hierarchy frees it too.  APM_E_STATE without a hierarchy.
 * apm_order_particles: APM_E_INVALID when no workspace is reserved or n is
 * above n_max; asynchronous on `stream`. */
apm_status apm_reserve_order(apm_ctx* ctx, int64_t n_max);
apm_status apm_order_particles(apm_ctx* ctx, const apm_particles* particles, double half_dt, void* stream);

/* Deposit through shared-memory tiles (on = 1; default 0).  The paper has no
 * counterpart: like the order, this is a property of the GPU launch.  While a
 * current order exists (apm_order_particles for this many particles), the
 * deposits (apm_deposit, apm_deposit_all) visit the particles in bin order
 * too, and each CTA keeps the charges that fall into one grid's box around
 * its bin (the bin and the next along x, one cell of halo; on the levels
 * whose boxes together fit 2304 cells) in shared memory: each 64-bit sum as
 * two 32-bit words added with 32-bit atomics, the low word's carry into the
 * high word.  After a barrier it sends one 64-bit reduction per nonzero cell;
 * charges outside the box go straight to L2.  The field is bit-identical to
 * the direct deposit's.  It pays where many particles share cells (the
 * Plummer hierarchy's core: 0.74 -> 0.64 ms); at low density the table's
 * atomics cost more than the reductions they save (the batched level, the
 * cosmological step).  APM_E_INVALID for another value. */
apm_status apm_set_deposit_tiles(apm_ctx* ctx, int32_t on);

/* Launch shapes and plan choices of the five FFT passes of one level (x
 * forward, y forward, z with the table, y inverse, x inverse), in that order.
 *  budget[p]  the number of complex elements one shared-memory buffer of a
 *             runtime-planned pass CTA aims at: each grid batches
 *             pow2_floor(budget / M) lines per CTA (1..32 row pairs for the x
 *             passes, 4..32 kx columns for the y/z passes, 2..32 in FP64),
 *             halved while the CTA needs more than 200 KB of shared memory;
 *  threads[p] the runtime-planned pass's CTA size, 128 or 256;
 *  plan[p]    0: FP32 grids whose length has a compile-time plan (every
 *             {2,3,5,7}-smooth length from 36 to 84, and 128, 150, 256, 512)
 *             run the kernel specialised for it (16 lines per CTA); 1: every
 *             grid runs the runtime-planned kernel; 2 (x forward and x inverse only): as 0,
 *             and grids with M0 = M1 whose M x (M/2 + 1) plane fits 200 KB run
 *             the x and y transforms of a whole z plane in one kernel (the y
 *             pass then has no work for them; the inverse needs the window no
 *             taller than M1, which excludes a periodic root);
 *  max_radix  the largest stage radix of the runtime plans: 16 (FP32
 *             default; composite radices in registers) or 8 (FP64: always 8);
 *  packing    0: the grids of a level enter each work list in hierarchy order;
 *             1: largest transform first.
 * The defaults are budget 2048 (FP32) / 1024 (FP64), 256 threads, plan 0,
 * max_radix 16 (FP32) and packing 0.  budget, threads and packing only
 * regroup or reorder whole lines, so they never change a result, bit for bit;
 * plan and max_radix change the order of the butterflies' roundings (results
 * stay within the FP32 parity tolerances).  The paper has no counterpart:
 * these are properties of the GPU launch, not of the method. */
typedef struct {
    int32_t budget[5];
    int32_t threads[5];
    int32_t plan[5];
    int32_t max_radix;
    int32_t packing;
} apm_fft_shapes;

/* Autotuner: solves `level` like apm_solve_level (same arguments and outputs)
 * while timing every candidate shape of each FFT pass in turn (budgets
 * 512..8192 (FP32) or 256..4096 (FP64) by powers of two, 128 or 256 threads;
 * the fastest of five timed launches after a warm one, CUDA events on
 * `stream`), then, over the whole level's passes, each pass's plan (FP32),
 * the packing and the runtime plans' largest radix (FP32), one at a time, and
 * keeps the fastest choices for the context's later calls.  phi_short
 * holds the level's potential on return.  Synchronises `stream` and the
 * device several times: APM_E_STATE while `stream` is being captured. */
apm_status apm_autotune_level(apm_ctx* ctx, int32_t level, const int64_t* const* gmf,
                              void* const* phi_short, void* stream);

/* The shapes in use for `level`, and setting them (for instance from a cache
 * of earlier autotuner results).  apm_set_fft_shapes synchronises the device;
 * APM_E_INVALID for a budget < 1, a thread count, plan, packing or max_radix
 * outside the rules above (FP64: max_radix 8). */
apm_status apm_get_fft_shapes(const apm_ctx* ctx, int32_t level, apm_fft_shapes* out);
apm_status apm_set_fft_shapes(apm_ctx* ctx, int32_t level, const apm_fft_shapes* shapes);

/* The kernel that FFT pass `pass` (0 x forward, 1 y forward, 2 z with the
 * table, 3 y inverse, 4 x inverse) runs for each of the n grids of `level`
 * under its current shapes, in the level's grid order (that of
 * apm_solve_level's arrays): kinds[i] = 0 the runtime-planned kernel, 1 the
 * kernel with the compile-time plan of the grid's length, 2 the fused plane
 * kernel (this x pass and the y pass together), 3 nothing (the grid's y pass
 * is done by the fused kernel).  An extension without a counterpart in the
 * paper (its cost accounting names the passes, not their kernels).
 * APM_E_STATE without a hierarchy; APM_E_INVALID for a bad level or pass, or
 * n different from the level's grid count. */
apm_status apm_get_pass_kernels(const apm_ctx* ctx, int32_t level, int32_t pass, int32_t* kinds, int32_t n);

/* TSC interpolation of the cell accelerations to the particles (Sec. 2, the
 * same 27 weights as the deposit, at the same drifted position).  Only
 * particles owned by `level` are written: those inside the interior of a grid
 * of this level and not inside any grid of level+1 (the finest grid holding a
 * particle supplies its acceleration).  On an isolated root the cloud folds
 * into the edge cells as in the deposit.
 *  acc     : HOST array (grids of the level) of the apm_accel outputs
 *  acc_out : device array of 3 n floats/doubles (x, y, z components, n each);
 *            may be NULL when n == 0 */
apm_status apm_interp(apm_ctx* ctx, int32_t level, const void* const* acc,
                      const apm_particles* particles, double half_dt, void* acc_out,
                      void* stream);

/* apm_interp for every level at once: one pass over the particles that
 * converts each position once, finds its finest owning grid (searching from
 * the root down) and interpolates that grid's accelerations.  Every particle
 * owned by some grid is written, with the values apm_interp level by level
 * writes.  Not in the paper: a batching of its per-level interpolations.
 *  acc : HOST array of n_grids device pointers in hierarchy order (the
 *        apm_accel output of each grid) */
apm_status apm_interp_all(apm_ctx* ctx, const void* const* acc, const apm_particles* particles,
                          double half_dt, void* acc_out, void* stream);

/* One timestep of n particles (SoA, device arrays, updated in place) given
 * their accelerations `acc` (device, 3n values of the context precision, as
 * apm_interp writes them) evaluated at the half-step drifted positions
 * x + v dt/2, which is where apm_deposit and apm_interp place the particles
 * for half_dt = dt/2:
 *   v' = v + a dt,   x' = x + ((v + v')/2) dt
 * (drift-kick-drift leapfrog), every FP64 operation rounded in this order.
 * All levels advance with the same dt: the paper's evolutions without
 * subcycling (Sec. 3.1, 3.5).  The paper names no integrator; this one drives
 * those tests.  Positions are not wrapped (the deposit wraps periodic
 * coordinates itself). */
apm_status apm_kick_drift(apm_ctx* ctx, int64_t n, double* x, double* y, double* z, double* vx,
                          double* vy, double* vz, const void* acc, double dt, void* stream);

/* Kernel tracing.  While enabled, every kernel the context launches is
 * bracketed by CUDA events recorded on the stream it runs on (events come from
 * a pool of `capacity` pairs allocated here; launches beyond it are not
 * timed).  apm_profile_read synchronises the device, adds the elapsed times of
 * the recorded launches of kernel `kernel` (0 <= kernel < apm_kernel_count())
 * to its totals and returns the totals since the last enable:
 * launches and summed device milliseconds.  An FFT pass whose grids run
 * different kernels (segments) is one bracket that counts each segment's
 * launch; a y pass fused into its x pass launches and counts nothing.
 * Disabling frees the pool. */
apm_status apm_profile_enable(apm_ctx* ctx, int32_t on, int32_t capacity);
apm_status apm_profile_read(apm_ctx* ctx, int32_t kernel, int64_t* launches, double* total_ms);
int32_t apm_kernel_count(void);
const char* apm_kernel_name(int32_t kernel);

/* Potential of one periodic root grid without allocating anything.
 * The paper has no counterpart.  Some callers cannot call cudaMalloc:
 * applications that give the whole device to their own memory pool at
 * start-up (a library allocating behind their back would fail, or break the
 * pool's accounting), and loops that must not stall on the device-wide
 * synchronisation cudaFree implies.  This entry point needs no context and
 * allocates nothing; it computes what apm_solve_level computes for a periodic
 * root of n^3 cells (box side `box`, smoothing a = a_over_dx * box / n) with
 * the two-point-difference optimal Green's function (APM_GRAD_FD2) and the
 * FP32 path's default FFT stages (radices up to 16), in FP32, with every
 * intermediate (twiddles, the Green's table, the FFT spectra, a status word)
 * kept in one fixed 24 MiB device array that each GPU loading the library
 * holds until the process exits.
 *  gmf       : device, n^3 int64 cell masses * 2^mass_frac_bits (x fastest)
 *  phi_short : device, (n+4)^3 floats, cells [-2, n+2) (periodic wrap)
 * n must be {2,3,5,7}-smooth with 4 <= n <= 128; larger or non-smooth n return
 * APM_E_INVALID (the fixed array holds at most a 128^3 grid).
 * The first call on a device looks up the array's device address and sets the
 * FFT kernels' shared-memory limit (host-side set-up, once per device, with that
 * device current); make that first call before any stream capture.
 * All calls share the one array, which keeps the last call's contents: each
 * call rebuilds everything it reads and clears its status word first, but
 * calls whose work overlaps on the GPU (different streams, or different host
 * threads) race on it and must be serialised by the caller.
 * There is no status reader: if the x-forward pass's bounded wait for its row
 * copy runs out (about a second; not expected in normal operation), the whole
 * phi_short window is filled with NaN instead of a partial result. */
apm_status apm_solve_periodic_noalloc(int32_t n, double box, double a_over_dx,
                                      int32_t mass_frac_bits, const int64_t* gmf,
                                      float* phi_short, void* stream);

/* Synchronises `stream`, returns the first error the kernels latched since the
 * last call (APM_OK if none) and clears it. */
apm_status apm_sync_status(apm_ctx* ctx, void* stream);

/* Static description of a status code. */
const char* apm_status_string(apm_status s);

/* Frees everything the context owns (synchronises the device first). */
void apm_destroy(apm_ctx* ctx);

/* Library version string. */
const char* apm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* APM_H */
