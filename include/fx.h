/*
 * fx.h -- C ABI of libfx, the GB300 (sm_103a) block-AMR compressible Euler
 * hot path.
 *
 * The operations follow the problem statement of Flash-X (arXiv 2208.11630):
 * physics units update the mesh one block at a time and call Grid functions
 * between those updates to reconcile block boundaries across refinement
 * levels (Section 2); the mesh is a uniform grid or an octree AMR grid
 * (PARAMESH, Section 2); the compressible hydro solver is explicit, unsplit
 * and of predictor-corrector type, with a perfect-gas EOS (Section 2.2).  The concrete scheme (MC-limited MUSCL-Hancock, HLLC, Berger-
 * Colella flux correction, CFL max-reduction) is the textbook one; the paper
 * prints no equations.
 *
 * Conventions shared by every call:
 *   - Return value: FX_OK (0) or a negative FX_ERR_* code; nothing throws.
 *     The text of the last error of a context is in fx_last_error().
 *   - Null handles: a call given a null context, block set or batch (or a
 *     null required pointer) returns FX_ERR_ARG without touching the device;
 *     exceptions: fx_finalize(NULL) does nothing and returns FX_OK,
 *     fx_last_error(NULL) returns "null context", fx_block_fluxes(NULL, b)
 *     returns NULL.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *     default stream).  Every call is stream-ordered and asynchronous unless
 *     its comment says it synchronises.
 *   - Ownership: state buffers are owned by the caller and only borrowed; the
 *     library owns its mesh tables, flux registers and reduction scratch and
 *     frees them in fx_blocks_destroy / fx_finalize.
 *   - Threads: one context per host thread.
 *   - Layout of a state buffer: U[block][var][z][y][x], x fastest,
 *     var = (rho, m_x, m_y, m_z, E), P = nxb + 2*nguard cells per padded
 *     axis, one z-plane in 2D (m_z stays 0).  Element type: double for
 *     FX_F64, float for FX_F32BULK.  Interior cell (i, j, k) is at padded
 *     index (i + nguard, j + nguard, k + nguard) (k + 0 in 2D).
 *   - Device errors (a non-positive density or pressure after an update) are
 *     latched in a device status word and reported by fx_status().
 */
#ifndef FX_H
#define FX_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FX_API __attribute__((visibility("default")))
#else
#define FX_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fx_ctx fx_ctx;        /* opaque: options, last error          */
typedef struct fx_blocks fx_blocks;  /* opaque: one block set (mesh + state) */

enum {
  FX_OK = 0,
  FX_ERR_ARG = -1,         /* invalid argument                              */
  FX_ERR_CUDA = -2,        /* a CUDA runtime call failed                    */
  FX_ERR_OOM = -3,         /* device or host allocation failed              */
  FX_ERR_UNPHYSICAL = -4,  /* rho <= 0 or p <= 0 (or NaN) after an update   */
  FX_ERR_TIMEOUT = -5,     /* a bounded device wait gave up                 */
  FX_ERR_STATE = -6,       /* call out of order (e.g. no state attached)    */
  FX_ERR_MESH = -7         /* mesh not a valid 2:1-balanced octree          */
};

enum { FX_F64 = 0, FX_F32BULK = 1 };        /* state element type            */
enum { FX_BC_OUTFLOW = 0, FX_BC_PERIODIC = 1, FX_BC_REFLECT = 2 };

/* fx_init: create a context for a perfect gas with ratio of specific heats
 * `gamma` (> 1), default block size `nxb` interior cells per axis (a
 * multiple of 8 in 8..64) and `nguard` guard cells per side (2..nxb/2; the
 * scheme reads 2).
 * Paper: the perfect-gas EOS of Section 2.2; blocks with guard cells of the
 * Grid unit, Section 2.  *out receives the context.  Errors: FX_ERR_ARG,
 * FX_ERR_CUDA (no usable device), FX_ERR_OOM. */
FX_API int fx_init(double gamma, int nxb, int nguard, fx_ctx **out);

/* fx_finalize: destroy a context (block sets must be destroyed first). */
FX_API int fx_finalize(fx_ctx *ctx);

/* fx_set_option: set a numeric option of the context.
 *   "cfl_form"  0 = dt from the sum over directions of (|u_d|+c)/dx_d
 *               (default), 1 = from the maximum over directions;
 *   "reflux"    1 = apply fine-to-coarse flux correction (default), 0 = off;
 *   "integrator" 0 = MUSCL-Hancock (default); 1 = SSP-RK2 with plain
 *               MC-limited PLM face states and the same HLLC flux (the
 *               method-of-lines family of the Spark solver, Section 2.2):
 *               U1 = U + dt L(U), coarse-fine fill of U1,
 *               U <- (U + (U1 + dt L(U1))) / 2 in the current buffer, flux
 *               correction with the stage-averaged fluxes; 2 = SSP-RK3 of
 *               Shu and Osher with the same face states and flux:
 *               U2 = 3/4 U + 1/4 (U1 + dt L(U1)) in a third state buffer
 *               that the library allocates on first use (the size of one
 *               state buffer, freed with the block set), coarse-fine fill
 *               of U2, U <- 1/3 U + 2/3 (U2 + dt L(U2)), flux correction with
 *               the fluxes weighted 1/6, 1/6, 2/3.  Batches accept only
 *               integrator 0;
 *   "f64_arith" 0 = the update of FX_F64 block sets runs in
 *               FP64 arithmetic (default); 1 = in double-word arithmetic:
 *               each value an unevaluated sum of two FP32 numbers (48
 *               significant bits, relative precision near 2^-47, FP32
 *               exponent range), on the FP32 pipe.  The state stays FP64 and
 *               every other kernel (guard fill, prolongation, flux
 *               correction, dt) is unchanged; results differ from the FP64
 *               update by the double-word rounding (about 1e-14 relative per
 *               step).  Applies to the single-gas and multispecies
 *               MUSCL-Hancock updates and to the SSP-RK stages; ignored by
 *               FX_F32BULK; batches honour it per request (fx_batch_add).
 *               2 = in FP32 arithmetic (the other reading of an FP32 path,
 *               kept as an ablation of FX_F32BULK): the state stays FP64
 *               (80 bytes of HBM per zone update), primitives, slopes,
 *               predictor and HLLC run in FP32, the flux divergence is
 *               added to the FP64 state in FP64 and the next dt is reduced
 *               in FP64; errors of FP32 arithmetic (about 1e-7 relative per
 *               step).  Single-gas MUSCL-Hancock only: fx_hydro_advance
 *               refuses it with the SSP-RK integrators or species, and
 *               fx_batch_add refuses such block sets (FX_ERR_ARG).
 * Errors: FX_ERR_ARG for an unknown key or value. */
FX_API int fx_set_option(fx_ctx *ctx, const char *key, double value);

/* fx_set_species: make block sets created afterwards with this context a
 * multispecies perfect gas (Section 2.2: the perfect-gas EOS has a
 * multispecies variant) of `nspec` (0..4; 0 = the single gas of fx_init)
 * species with ratios of specific heats gamma_k[k] (> 1) and molar masses
 * A_k[k] (> 0).  Such block sets carry nvar = 5 + nspec variables per cell
 * (state buffers of nblocks * nvar * PZ * P * P elements; the last nspec
 * variables are rho X_k, the partial densities of mass fractions X_k, and
 * the primitive input of fx_prim_to_cons carries X_k there); a cell's gamma
 * follows the ideal-gas mixture rule
 *   gamma - 1 = (sum_k X_k / A_k) / (sum_k X_k / (A_k (gamma_k - 1))).
 * The mass fractions are reconstructed and predicted like a transverse
 * velocity and HLLC carries each side's fractions through the star region.
 * Multispecies block sets are stepped with integrator 0 and outside batches.
 * Errors: FX_ERR_ARG. */
FX_API int fx_set_species(fx_ctx *ctx, int nspec, const double *gamma_k, const double *A_k);

/* fx_last_error: NUL-terminated text of the last error of `ctx` (owned by
 * the context, valid until its next call). */
FX_API const char *fx_last_error(const fx_ctx *ctx);

/* fx_blocks_create: describe a block set and attach its two state buffers.
 * Paper: uniform grid or PARAMESH octree of blocks (Section 2).
 *   ndim        2 or 3;
 *   nblocks     number of blocks (leaves and non-leaf parents);
 *   nxb         interior cells per axis of every block (0 = context default);
 *   nroot[3]    level-0 blocks per axis (entries beyond ndim ignored);
 *   level[nb]   refinement level of each block, 0 = coarsest;
 *   origin[nb][3] lower-corner cell index of each block in the lattice of its
 *               own level (level l has nroot[d]*nxb*2^l cells along d);
 *   parent[nb]  index of the parent block, -1 for level-0 blocks.  A block
 *               is a leaf iff it is nobody's parent; non-leaf blocks hold the
 *               restriction of their children;
 *   lo[3], hi[3] physical domain; bc[6] = {x-, x+, y-, y+, z-, z+}
 *               boundary kinds (FX_BC_*; periodic must be set on both sides).
 *               Outflow guards copy the nearest interior cell, periodic ones
 *               wrap, reflecting ones take the mirror-image cell with the
 *               wall-normal momentum negated (a solid slip wall);
 *   precision   FX_F64 or FX_F32BULK (element type of the state buffers);
 *   U0, U1      caller-owned device buffers of nblocks*nvar*PZ*P*P elements
 *               (nvar = 5, or 5 + nspec after fx_set_species),
 *               16-byte aligned.  U0 holds the initial state; U1 receives the
 *               first update; they alternate afterwards (fx_blocks_current).
 * The mesh must be 2:1 balanced (every guard region is covered by a block of
 * the same level or by a leaf one level coarser).  Host arrays are copied;
 * the call synchronises.  Errors: FX_ERR_ARG, FX_ERR_MESH, FX_ERR_OOM,
 * FX_ERR_CUDA. */
FX_API int fx_blocks_create(fx_ctx *ctx, int ndim, int nblocks, int nxb, const int nroot[3],
                     const int *level, const int64_t *origin, const int *parent,
                     const double lo[3], const double hi[3], const int bc[6],
                     int precision, void *U0, void *U1, fx_blocks **out);

/* fx_blocks_destroy: free the library-owned tables of a block set (the
 * caller's buffers are untouched). */
FX_API int fx_blocks_destroy(fx_blocks *bs);

/* fx_blocks_mark_dirty: tell the library that the caller wrote the current
 * state buffer directly (not through an fx_* call), so that the next
 * fx_compute_dt reads the state instead of reusing the signal-speed maximum
 * of the last update, and the next guard fill restricts the parents again
 * instead of relying on the restriction that ended the last update. */
FX_API int fx_blocks_mark_dirty(fx_blocks *bs);

/* fx_blocks_current: index (0 or 1) of the buffer that holds the current
 * state; flips after every fx_hydro_advance.  Negative on error. */
FX_API int fx_blocks_current(const fx_blocks *bs);

/* fx_prim_to_cons: fill the current buffer from primitive variables
 * W[block][var][z][y][x] (device, double, var = rho, u, v, w, p; same
 * layout and size as a state buffer) using the perfect-gas EOS
 * E = p/(gamma-1) + rho |v|^2 / 2 (Section 2.2).  Every cell is converted. */
FX_API int fx_prim_to_cons(fx_ctx *ctx, fx_blocks *bs, const double *W_dev, void *stream);

/* fx_guardcell_fill: fill the guard cells of every leaf of the current
 * buffer -- the Grid's reconciliation of block boundaries across levels
 * (Section 2):
 *   1. restrict every non-leaf block from its children (pairwise mean),
 *      finest level first;
 *   2. same-level copy from neighbour blocks, with outflow (zero-gradient)
 *      or periodic physical boundaries;
 *   3. level by level, conservative MC-limited linear prolongation into the
 *      guards of leaves next to a coarser leaf.
 * All nguard layers are filled, corners and edges included. */
FX_API int fx_guardcell_fill(fx_ctx *ctx, fx_blocks *bs, void *stream);

/* fx_guardcell_fill_amr: the coarse-fine part of the guard fill -- what the
 * fused fx_hydro_advance does not read directly from same-level neighbours
 * (Section 2's reconciliation of block boundaries across levels):
 * restriction of every parent, the same-level guards of coarse leaves that
 * feed a prolongation, and the prolonged guards of leaves next to a coarser
 * leaf.  A no-op on a uniform grid.  Enough for fx_hydro_advance. */
FX_API int fx_guardcell_fill_amr(fx_ctx *ctx, fx_blocks *bs, void *stream);

/* fx_compute_dt: CFL time step from the current buffer's leaf interiors,
 * dt = cfl / max_cells sum_d (|u_d| + c) / dx_d, c = sqrt(gamma p / rho)
 * (the maximum over d with cfl_form = 1).  The maximum is an exact,
 * order-independent reduction.  `dt_dev` is a device double that receives
 * dt (kept on the device so that a captured graph needs no host trip).
 * When the current state was produced by fx_hydro_advance and nothing wrote
 * it since, the update already reduced its signal speeds and only the final
 * division runs; otherwise the state is read again.  A caller that writes
 * the state buffers itself must call fx_blocks_mark_dirty afterwards.  A
 * leaf cell with negative pressure (no sound speed) makes dt NaN in both
 * forms, wherever it sits. */
FX_API int fx_compute_dt(fx_ctx *ctx, fx_blocks *bs, double cfl, double *dt_dev, void *stream);

/* fx_hydro_advance: one unsplit second-order step of all leaves with the
 * time step read from the device double *dt_dev -- the per-block physics
 * update of Section 2 with the predictor-corrector hydro of Section 2.2:
 * primitive variables, MC-limited slopes, MUSCL-Hancock half step, HLLC
 * fluxes, conservative update into the other buffer; then the fine-to-coarse
 * flux correction at coarse-fine faces (if the "reflux" option is on) and
 * restriction into the parents.  Same-level neighbour data are read straight
 * from the neighbours' interiors (identical to the guard copy); guards covered
 * by a coarser leaf must have been filled (fx_guardcell_fill or fx_step).  The
 * new state's buffer becomes current. */
FX_API int fx_hydro_advance(fx_ctx *ctx, fx_blocks *bs, const double *dt_dev, void *stream);

/* fx_step: fx_compute_dt, fx_guardcell_fill_amr and fx_hydro_advance in
 * order.  Same-level guards are not written (the fused update reads the
 * neighbours); call fx_guardcell_fill to materialise every guard cell. */
FX_API int fx_step(fx_ctx *ctx, fx_blocks *bs, double cfl, double *dt_dev, void *stream);

/* fx_conserved_totals: out_host[v] = sum over leaf interior cells of U_v dV
 * for the current buffer (v < nvar: 5, or 5 + nspec for a multispecies
 * block set), summed per block in a fixed order on the device and over
 * blocks with compensated summation on the host.  Synchronises. */
FX_API int fx_conserved_totals(fx_ctx *ctx, fx_blocks *bs, double *out_host, void *stream);

/* fx_status: synchronise the device and report the latched device status of
 * the block set (FX_OK or FX_ERR_UNPHYSICAL); clears the latch. */
FX_API int fx_status(fx_ctx *ctx, fx_blocks *bs);

/* fx_run_host: end-to-end convenience for callers that hold the state in
 * host memory.  Copies U_host_in (page-locked host memory recommended) into
 * the current buffer, runs `nsteps` full steps with CFL number `cfl`, and
 * copies the current buffer to U_host_out.  *t_host (may be NULL) receives
 * the simulated time advanced.  Synchronises. */
FX_API int fx_run_host(fx_ctx *ctx, fx_blocks *bs, const void *U_host_in, void *U_host_out,
                int nsteps, double cfl, double *t_host, void *stream);

/* fx_run_host_interior: like fx_run_host, for callers that hold only the
 * interior cells: W_in and W_out are packed conserved states
 * [nblocks][nvar][nz][nxb][nxb] (nz = nxb in 3D, 1 in 2D; x fastest; element
 * type of the block set's precision), page-locked host memory recommended.
 * Guard cells never cross the host link (they are rebuilt by the guard fill),
 * so each direction moves (nxb/(nxb+2 nguard))^ndim of fx_run_host's bytes.
 * On a single-level block set the last step's update runs in chunks of
 * blocks whose interiors are downloaded while later chunks compute.  The
 * first call allocates a device staging buffer of the packed size and two
 * streams; they live as long as the block set.  Results equal fx_run_host's
 * bit for bit.  Synchronises.  Errors: FX_ERR_ARG, FX_ERR_STATE (block set
 * in a batch), FX_ERR_OOM, FX_ERR_CUDA. */
FX_API int fx_run_host_interior(fx_ctx *ctx, fx_blocks *bs, const void *W_in, void *W_out,
                                int nsteps, double cfl, double *t_host, void *stream);

/* ---- regridding (dynamic refinement) ----------------------------------
 * Paper: the Grid unit's octree adapts to the solution (PARAMESH, Section 2).
 * The criterion is Loehner's (1987) normalised second derivative, evaluated
 * per cell on density and pressure (the FLASH-family default refinement
 * variables), maximised over each leaf.  Two calls change the mesh, so that
 * the caller can allocate the new state buffers in between:
 *
 * fx_regrid_plan: restricts the parents and fills every guard layer of the
 *   current state (leaf interiors unchanged), computes the indicator with
 *   filter `filter` (0.01 typical), and plans the new mesh: leaves above
 *   `refine_cutoff` are split (up to level `max_level`), sibling leaves all
 *   below `derefine_cutoff` merge into their parent, then splits are added
 *   and merges cancelled until touching leaf regions (faces, edges, corners,
 *   periodic wrap) differ by at most one level.  *nblocks_new receives the
 *   new block count.  Synchronises `stream`.  Errors: FX_ERR_ARG,
 *   FX_ERR_STATE (in a batch), FX_ERR_OOM, FX_ERR_CUDA, FX_ERR_MESH.
 * fx_regrid_errors: the indicator per block of the current mesh from the
 *   last plan (-1 for parents); err_host holds nblocks doubles.
 * fx_regrid_mesh: the planned mesh (nblocks_new entries, sorted by level,
 *   then z, y, x of the origin): level, origin [n][3] in the block's level
 *   lattice, parent (-1 at level 0).
 * fx_regrid_apply: moves the state onto the planned mesh in the new
 *   caller-owned buffers U0_new, U1_new (nblocks_new * nvar * PZ * P * P
 *   elements, 16-byte aligned; U0_new becomes current): kept blocks copy
 *   their interior, new children take the conservative MC-limited linear
 *   prolongation of their parent, parents are restricted.  The handle then
 *   describes the new mesh (tables rebuilt, old buffers no longer used: the
 *   caller may free them after this call returns).  Totals are conserved to
 *   rounding.  Synchronises.  Errors: FX_ERR_STATE (no plan / in a batch),
 *   FX_ERR_ARG, FX_ERR_OOM, FX_ERR_CUDA, FX_ERR_MESH. */
FX_API int fx_regrid_plan(fx_ctx *ctx, fx_blocks *bs, double refine_cutoff,
                          double derefine_cutoff, double filter, int max_level, void *stream,
                          int *nblocks_new);
FX_API int fx_regrid_errors(const fx_blocks *bs, double *err_host);
FX_API int fx_regrid_mesh(const fx_blocks *bs, int *level, int64_t *origin, int *parent);
FX_API int fx_regrid_apply(fx_ctx *ctx, fx_blocks *bs, void *U0_new, void *U1_new,
                           void *stream);

/* fx_regrid_plan_host: the planning step of fx_regrid_plan alone -- marking
 * and 2:1 balance, the same rules and the same sorted result -- for a mesh
 * and per-block indicator values given in host arrays.  Host code only: it
 * needs no context and no GPU (plan on another host, or check the planner
 * against an independent implementation).  Paper: Section 2 (the Grid unit
 * refines and derefines the octree).
 *   ndim, nxb, nroot[3], bc[6] (x-, x+, y-, y+, z-, z+), nblocks, level,
 *   origin [nblocks][3] (cell index in the block's level lattice), parent:
 *   as for fx_blocks_create, and checked by the same rules.
 *   err [nblocks]: indicator of each leaf (ignored for parents).
 *   refine_cutoff, derefine_cutoff, max_level: as for fx_regrid_plan.
 *   cap: entries of the caller-owned output arrays level_new [cap],
 *   origin_new [cap][3], parent_new [cap] (as fx_regrid_mesh writes them)
 *   and map_new [cap][3] = (kind 0 kept / 1 new child, old block if kept
 *   else old parent, octant: bit d set for the upper half along axis d).
 *   *nblocks_new receives the planned block count, also when it exceeds
 *   cap (then FX_ERR_ARG and no output written; cap = 0 asks for the count).
 *   msg (may be null): receives a NUL-terminated reason on error, at most
 *   msg_len bytes.
 * Errors: FX_ERR_ARG (null or out-of-range argument, cap too small),
 *   FX_ERR_MESH (a mesh fx_blocks_create would refuse; not covering the
 *   domain, not 2:1 balanced, or a lattice too large for the planner). */
FX_API int fx_regrid_plan_host(int ndim, int nxb, const int nroot[3], const int bc[6],
                               int nblocks, const int *level, const int64_t *origin,
                               const int *parent, const double *err, double refine_cutoff,
                               double derefine_cutoff, int max_level, int cap, int *nblocks_new,
                               int *level_new, int64_t *origin_new, int *parent_new, int *map_new,
                               char *msg, int msg_len);

/* fx_block_fluxes: device pointer to the flux registers of block `b`
 * ([2*ndim faces x-,x+,y-,y+,z-,z+][nvar][nxb^(ndim-1)], lower transverse axis
 * fastest) written by the last fx_hydro_advance, or NULL if the block has no
 * coarse-fine face.  For diagnostics and tests. */
FX_API const double *fx_block_fluxes(const fx_blocks *bs, int b);

/* ---- batched stepping of many block sets ----------------------------------
 * A batch advances many independent block sets (requests) together: each
 * step is one CUDA graph replay in which every phase of the step -- dt,
 * coarse-fine guard fill, the fused update, flux correction, restriction --
 * is one kernel launch over a work list spanning all requests, the update
 * being a persistent kernel per (dimension, precision, tile) group.  A
 * request whose update alone fills the GPU (at least one wave of the
 * per-block-set update's CTAs: leaves x tiles per block >= CTAs per SM x SMs)
 * is stepped instead by the kernels of fx_step, on a branch of the same
 * graph; its result is bitwise that of stepping it alone.  Block sets of
 * different sizes, block counts, levels and precisions mix freely; each
 * keeps its own dt.  This is the paper's block-by-block update (Section 2)
 * organised for one GPU; the batching itself has no counterpart in the
 * paper.  A block set in a batch must not be stepped or destroyed directly
 * until fx_batch_remove returns it. */
typedef struct fx_batch fx_batch;

/* fx_batch_create: empty batch with room for `max_requests` block sets. */
FX_API int fx_batch_create(fx_ctx *ctx, int max_requests, fx_batch **out);
/* fx_batch_destroy: synchronise and free the batch (block sets are released). */
FX_API int fx_batch_destroy(fx_batch *b);
/* fx_batch_add: add block set `bs` to advance `nsteps` steps with CFL number
 * `cfl` from its current state; *slot_out receives its slot.  It joins at the
 * next fx_batch_run (the graph is re-captured); its parents are restricted
 * on `stream` first if the state has changed since they last were.
 * Synchronises `stream`.  The
 * update of an FX_F64 block set whose context has "f64_arith" = 1 runs in
 * double-word arithmetic inside the batch too (compute class 2 below). */
FX_API int fx_batch_add(fx_batch *b, fx_blocks *bs, double cfl, int nsteps, void *stream,
                        int *slot_out);
/* fx_batch_run: `nsteps` batched steps; every request with steps left
 * advances one step per batched step.  Asynchronous on `stream`. */
FX_API int fx_batch_run(fx_batch *b, int nsteps, void *stream);
/* fx_batch_poll: steps_left[slot] for every slot (-1 = empty).  Synchronises. */
FX_API int fx_batch_poll(fx_batch *b, int *steps_left, void *stream);
/* fx_batch_remove: release the block set in `slot` (cancelling it if steps
 * remain); its current buffer is whatever the batch produced.  Synchronises. */
FX_API int fx_batch_remove(fx_batch *b, int slot, void *stream);
/* fx_batch_tune: autotune the update launch of each (dimension, compute class)
 * group whose blocks allow 16x16 tiles: the tile edge (16 or 8) and the CTAs
 * per SM of the persistent kernel, by timing each candidate on a sample of
 * the batch's own work items with dt = 0 (after a coarse-fine guard fill;
 * neither changes any state) and scaling to the whole group.  Choices are
 * cached per (dimension, precision, SM count, set of block edges).  `report`
 * (may be NULL; room for 193 ints) receives (tile, ctas, estimated
 * microseconds per update of the group) triples, 0 terminated.  Requests
 * stepped by the per-block-set kernels do not use the choice.
 * Synchronises. */
FX_API int fx_batch_tune(fx_batch *b, void *stream, int *report);
/* fx_batch_choice: the launch choice in use for a (ndim, precision) group;
 * precision is the update's compute class: FX_F64 (0), FX_F32BULK (1), or 2
 * for FP64 block sets updated in double-word arithmetic. */
FX_API int fx_batch_choice(const fx_batch *b, int ndim, int precision, int *tile,
                           int *ctas_per_sm);
/* fx_batch_path: how the request in `slot` is stepped: *path = 0 by the
 * batched phases and the persistent update, 1 by the per-block-set kernels
 * of fx_step on a branch of the graph (its update alone fills the GPU).
 * Fixed by the request's mesh, precision and this GPU, not by the rest of
 * the batch.  Errors: FX_ERR_ARG for a null pointer or an empty slot. */
FX_API int fx_batch_path(const fx_batch *b, int slot, int *path);

/* Largest block count fx_compute_dt_noalloc accepts (size of its fixed
 * device scratch, one 8-byte partial per block plus a counter: 256 KB). */
#define FX_NOALLOC_MAX_BLOCKS 32768

/* fx_compute_dt_noalloc: the CFL time step of fx_compute_dt for callers that
 * cannot allocate device memory (a host callback, an allocator's own
 * bookkeeping, a process whose device memory belongs to another runtime, a
 * loop that forbids allocation after start-up).  The paper has no counterpart;
 * this entry point exists only so that such callers need no block set.
 *   U_dev      caller-owned device state, FP64, layout of a single-gas state
 *              buffer: nblocks blocks of 5 variables [block][5][PZ][P][P]
 *              (rho, mx, my, mz, E), one refinement level, every block
 *              counted.  A multispecies buffer (5 + nspec variables per cell,
 *              fx_set_species) is outside this call's contract: it would be
 *              read at the wrong block stride with the wrong EOS;
 *   dx[3]      cell widths (dx[2] ignored in 2D); gamma, cfl, cfl_form as in
 *              fx_init / fx_compute_dt / fx_set_option("cfl_form");
 *   dt_dev     caller-owned device double that receives dt;
 *   errbuf     optional caller buffer (errlen bytes) for an error message.
 * It allocates nothing: its scratch is a fixed array inside the library that
 * every GPU loading the library holds until exit.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) with the device
 * current; make that first call before any stream capture.  The call clears
 * the scratch counter on `stream` before the kernel.  All calls share the
 * scratch: calls that may overlap on the GPU race and must be ordered by the
 * caller.  A cell with negative pressure (no sound speed) makes dt NaN, in
 * both CFL forms and wherever the cell sits, as with fx_compute_dt; no status
 * word is latched, so a caller that cannot rule such states out checks dt.
 * Errors: FX_ERR_ARG (including nblocks > FX_NOALLOC_MAX_BLOCKS),
 * FX_ERR_CUDA. */
FX_API int fx_compute_dt_noalloc(const double *U_dev, int ndim, int nblocks, int nxb, int nguard,
                                 const double dx[3], double gamma, double cfl, int cfl_form,
                                 double *dt_dev, void *stream, char *errbuf, size_t errlen);

/* fx_kernel_launches: number of CUDA kernels this library has launched in
 * the process so far (all contexts).  Diagnostics for benchmarks. */
FX_API long long fx_kernel_launches(void);

/* fx_fma_probe: a measurement aid with no counterpart in the paper.  Runs
 * `ctas` CTAs of 256 threads, each thread 8 independent chains of `iters`
 * fused multiply-adds in FP64 (precision FX_F64) or FP32 (FX_F32BULK), and
 * writes one value per CTA to the caller-owned device array out_dev (ctas
 * elements of that type).  *flops (if not null) receives the flops the launch
 * performs, 2 * 8 * iters * ctas * 256.  Timed with events around it on
 * `stream`, it gives the FMA pipe's throughput under the clocks of the
 * moment, the peak that the FP64 update's arithmetic is set against.
 * Asynchronous.  Errors: FX_ERR_ARG (bad precision, ctas < 1, iters < 1,
 * null out_dev), FX_ERR_CUDA. */
FX_API int fx_fma_probe(int precision, int ctas, int iters, void *out_dev, void *stream,
                        double *flops);

/* fx_dword_selftest: apply one operation of the double-word arithmetic of
 * the "f64_arith" option element by element, for testing it against FP64:
 * out[i] = op(a[i], b[i]) with both inputs converted to double-words and the
 * result converted back.  op: 0 a + b, 1 a - b, 2 a * b, 3 a / b, 4 sqrt(a),
 * 5 1/sqrt(a), 6 a (the conversion round trip), 7 fma(a, b, a).  a_dev,
 * b_dev, out_dev: caller-owned device arrays of n doubles (b_dev unused by
 * ops 4-6).  Asynchronous on `stream`.
 * Errors: FX_ERR_ARG for a bad op, n < 0 or a null array; FX_ERR_CUDA. */
FX_API int fx_dword_selftest(int op, const double *a_dev, const double *b_dev, double *out_dev,
                             int n, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FX_H */
