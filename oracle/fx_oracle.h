/*
 * fx_oracle.h -- plain FP64 CPU oracle of the block-AMR unsplit Euler step.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the correctness reference for the
 * CUDA path.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load it; the product library never links or calls it, and the two
 * share no code.
 *
 * What it computes (Flash-X, arXiv 2208.11630, Section 2: physics advances
 * the mesh one block at a time, with Grid calls in between that reconcile
 * block boundaries across refinement levels, on a uniform or octree AMR grid;
 * Section 2.2: an unsplit predictor-corrector compressible hydro solver with
 * a perfect-gas EOS).  The paper names the method family only; the
 * concrete scheme is the textbook one:
 *   - perfect-gas EOS, p = (gamma-1)(E - |m|^2 / (2 rho)), c = sqrt(gamma p / rho);
 *   - MC-limited piecewise-linear slopes of the primitive variables
 *     (van Leer 1977);
 *   - MUSCL-Hancock half-step predictor in primitive form (Toro, "Riemann
 *     Solvers and Numerical Methods for Fluid Dynamics", ch. 14);
 *   - HLLC flux with Davis wave-speed estimates (Toro, Spruce & Speares 1994;
 *     Toro ch. 10);
 *   - conservative unsplit update, fine-to-coarse flux correction
 *     (Berger & Colella 1989), restriction into parents;
 *   - CFL time step from the maximum signal speed.
 * Guard cells: same-level copy, outflow (zero-gradient) or periodic physical
 * boundaries, restriction of finer data, conservative MC-limited linear
 * prolongation of coarser data.
 *
 * Layout: U[block][var][z][y][x], var = (rho, mx, my, mz, E), P = nxb + 2 ng
 * cells per padded axis, one z-plane in 2D.  Everything is FP64.
 *
 * Parity status of each function is recorded beside it:
 *   "pinned"   -- checked by the CPU tests against closed forms, invariants,
 *                 brute force or textbook values;
 *   "unpinned" -- no independent check exists (none in this file).
 */
#ifndef FX_ORACLE_H
#define FX_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_mesh or_mesh;

/* Build the oracle's own view of a block set (levels, origins in the block's
 * level lattice, parents).  bc[6] = {x-, x+, y-, y+, z-, z+}, 0 = outflow,
 * 1 = periodic (both sides of an axis), 2 = reflecting wall.  Returns NULL on invalid input (message via or_last_error). */
or_mesh *or_mesh_create(int ndim, int nxb, int ng, int nb, const int nroot[3],
                        const int *level, const int64_t *origin, const int *parent,
                        const double lo[3], const double hi[3], const int bc[6],
                        double gamma);
void or_mesh_destroy(or_mesh *m);
/* Multispecies perfect gas (Section 2.2 names a multispecies variant of the
 * perfect-gas EOS): nspec (<= 4) species with ratios of specific heats
 * gamma_k and molar masses A_k; the state then carries 5 + nspec variables
 * per cell, the last nspec being rho X_k (mass fractions X_k, advected with
 * the flow; HLLC keeps each side's X through the star region), and a cell's
 * gamma follows the ideal-gas mixture rule
 * gamma - 1 = (sum X_k / A_k) / (sum X_k / (A_k (gamma_k - 1))).
 * Call before any use of the mesh.  Pinned: one species equal to the single
 * gas, two identical species equal to one gas with exact species transport,
 * the scalar-advection special case for X, the EOS mixture closed form, and
 * L1 convergence to the exact two-gas Riemann solution. */
int or_mesh_set_species(or_mesh *m, int nspec, const double *gamma_k, const double *A_k);
const char *or_last_error(void);
void or_set_threads(int n);
int or_get_threads(void);

/* EOS conversions over every cell of every block (pinned: round trip). */
void or_prim_to_cons(const or_mesh *m, const double *W, double *U);
void or_cons_to_prim(const or_mesh *m, const double *U, double *W);

/* Guard-cell fill of all leaves (pinned: brute-force global indexing,
 * linear-field prolongation, restrict-of-prolong identity).  Returns 0 or -1. */
int or_guardcell_fill(const or_mesh *m, double *U);

/* CFL time step: dt = cfl / max over leaf interior cells of
 * sum_d (|u_d| + c) / dx_d (form 0) or max_d (|u_d| + c) / dx_d (form 1).
 * A cell with no sound speed (p / rho < 0 gives NaN) makes dt NaN in both
 * forms, wherever it sits; returns -4 when dt is not finite.
 * Pinned: uniform-state closed form, order independence, a planted
 * negative-pressure cell giving NaN. */
int or_compute_dt(const or_mesh *m, const double *U, double cfl, int form, double *dt);

/* One hydro step of the leaves: reads U (guards filled), writes interiors of
 * Unew, then applies flux correction (if reflux != 0) and restricts into
 * parents.  If bflux != NULL it receives every leaf's block-boundary fluxes,
 * [nb][2*ndim faces: x-, x+, y-, y+, z-, z+][5][nxb^(ndim-1)] (transverse
 * index order: the lower axis fastest).  If sel != NULL only the nsel listed
 * leaves are advanced and no correction or restriction is done.
 * Returns 0, or -4 if a new interior cell has rho <= 0 or p <= 0.
 * Pinned: Sod exact solution (L1 convergence), conservation, uniform state,
 * mirror symmetry, decomposition invariance, scalar-advection special case,
 * geometric reflux check. */
int or_hydro_advance(const or_mesh *m, const double *U, double *Unew, double dt,
                     int reflux, double *bflux, int nsel, const int *sel);

/* SSP-RK2 variant of the step (method-of-lines, the family of Flash-X's
 * Spark solver, Section 2.2): plain MC-limited PLM face states (no Hancock
 * predictor), HLLC, U1 = U + dt L(U), guard fill of U1, then
 * Unew = (U + (U1 + dt L(U1))) / 2; flux correction with the stage-averaged
 * fluxes; restriction into parents.  U must have filled guards.  bflux as in
 * or_hydro_advance (stage-averaged).  Pinned: scalar-advection special case
 * (textbook Heun + MC-PLM), Sod L1 convergence, linear waves at second order,
 * conservation (periodic, AMR with correction), uniform state. */
int or_hydro_advance_rk2(const or_mesh *m, const double *U, double *Unew, double dt, int reflux,
                         double *bflux);

/* SSP-RK3 variant (Shu-Osher three-stage form, the third-order member of the
 * same family): U1 = U + dt L(U); U2 = 3/4 U + 1/4 (U1 + dt L(U1));
 * Unew = 1/3 U + 2/3 (U2 + dt L(U2)), guard fills of U1 and U2, flux
 * correction with the fluxes weighted 1/6, 1/6, 2/3.  Pinned: scalar-advection
 * special case (textbook SSP-RK3 + MC-PLM), third-order temporal convergence
 * on smooth data, conservation (periodic, AMR with correction), uniform
 * state. */
int or_hydro_advance_rk3(const or_mesh *m, const double *U, double *Unew, double dt, int reflux,
                         double *bflux);

/* Restriction of every non-leaf block from its children, finest level first:
 * each parent cell is the pairwise mean (x pairs, then y, then z) of the
 * 2^d child cells it covers.  Pinned: uniform state, linear-field exactness
 * via prolongation, conservation with flux correction. */
void or_restrict_parents(const or_mesh *m, double *U);

/* Sum over leaf interior cells of U dV per variable (out: 5 + nspec values;
 * compensated sums, fixed order).  Pinned by conservation tests. */
void or_conserved_totals(const or_mesh *m, const double *U, double *out);

/* Regridding (dynamic refinement of the PARAMESH-style octree, Section 2).
 * or_regrid_errors: per block, the maximum over interior cells and over
 * density and pressure of Loehner's (1987) normalised second-derivative
 * indicator with filter eps (-1 for non-leaf blocks).  U must have filled
 * guards.  Pinned: zero on linear fields, closed forms on a quadratic and a
 * step.
 * or_regrid_plan: leaves with error > rc (and level < max_level) are
 * refined; a parent whose children are all leaves with error < dc (none
 * refined) is coarsened; then, until nothing changes, any leaf region two or
 * more levels coarser than a touching region (faces, edges, corners;
 * periodic wrap) is refined, or its coarsening cancelled.  Writes the new
 * mesh sorted by (level, z, y, x of the origin) with parents, and per new
 * block kind 0 = kept (src = old block) or 1 = new child (src = old parent,
 * oct = octant).  Returns the new block count, or -1 (capacity / error).
 * or_regrid_transfer: kept blocks copy their interior, new children take
 * the conservative MC-limited linear prolongation of the parent (the guard
 * prolongation's formula; Uold guards filled) -- per coarse cell, unless that
 * would leave a non-positive density or pressure in one of its children, in
 * which case all of them take the coarse value.  Parents of the new mesh are
 * left to or_restrict_parents.  Pinned: conservation, uniform state, linear
 * fields, 2:1 balance and requests honoured (brute force). */
int or_regrid_errors(const or_mesh *m, const double *U, double eps, double *err);
int or_regrid_plan(const or_mesh *m, const double *err, double rc, double dc, int max_level,
                   int cap, int *level_out, int64_t *origin_out, int *parent_out, int *kind_out,
                   int *src_out, int *oct_out);
int or_regrid_transfer(const or_mesh *om, const double *Uold, const or_mesh *nm, const int *kind,
                       const int *src, const int *oct, double *Unew);

/* Point functions for unit pins. */
double or_mc(double a, double b);
void or_hllc(const double WL[5], const double WR[5], int dir, double gamma, double F[5]);

/* Exact Riemann solver for the 1D Euler equations (test tool; Toro ch. 4).
 * star[4] = {p*, u*, rho*L, rho*R}; returns -1 on vacuum generation. */
int or_riemann_star(const double WL[3], const double WR[3], double gamma, double star[4]);
/* Sample the self-similar solution at xi = x / t: out = {rho, u, p}. */
int or_riemann_sample(const double WL[3], const double WR[3], double gamma, double xi,
                      double out[3]);
/* The same for two gases: gamma gL left of the contact, gR right of it. */
int or_riemann_star2(const double WL[3], const double WR[3], double gL, double gR,
                     double star[4]);
int or_riemann_sample2(const double WL[3], const double WR[3], double gL, double gR, double xi,
                       double out[3]);

#ifdef __cplusplus
}
#endif
#endif
