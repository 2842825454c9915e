/*
 * oracle.c -- plain FP64 CPU oracle of the block-AMR unsplit Euler step.
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).  It
 * shares no code with the CUDA path.  Every routine is a direct, unoptimised
 * restatement of the definition it cites; loops run over cells, the only
 * parallelism is OpenMP over independent blocks.
 *
 * Scheme (Flash-X, arXiv 2208.11630, Section 2 and Section 2.2; concrete
 * formulas from the textbook methods the hydro solver family uses):
 *   EOS        perfect gas, p = (gamma-1)(E - |m|^2/(2 rho))
 *   slopes     MC limiter on primitives (van Leer 1977)
 *   predictor  MUSCL-Hancock half step, primitive quasi-linear form (Toro ch. 14)
 *   flux       HLLC, Davis speeds (Toro, Spruce & Speares 1994; Toro ch. 10)
 *   update     unsplit conservative update, directions summed x, y, z
 *   walls      outflow (nearest interior cell), periodic (wrap), reflecting
 *              (mirror image with the wall-normal momentum negated)
 *   AMR        restriction (pairwise mean of children), MC-limited conservative
 *              linear prolongation, fine-to-coarse flux correction
 *              (Berger & Colella 1989)
 *   dt         CFL max-reduction of the signal speed
 *
 * Readings where the paper is silent (all listed in the design notes):
 *   primitive (not characteristic) reconstruction; primitive-form Hancock;
 *   Davis wave speeds; positivity fallback to first order for a cell whose
 *   face states are not positive; sum-form CFL by default; MC prolongation on
 *   conserved variables; pairwise summation in restriction and flux averaging.
 *
 * Build with -ffp-contract=off so that x86 and Arm hosts give identical bits.
 */
#include "fx_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Op-count instrumentation: OR_STEP(k) opens one unit of work of step k of
 * the scheme (one cell's primitives, one cell's slopes and predictor, one
 * face's flux, one cell's update, one cell's signal speed); the counting
 * build (opcount.cpp) attributes the arithmetic that follows to it.  It
 * compiles to nothing here and changes no arithmetic. */
#ifndef OR_STEP
#define OR_STEP(k) ((void)0)
#endif

#define OR_MAXLEV 16
#define OR_MAXSP 4                /* species of the multispecies perfect gas */
#define OR_MAXV (5 + OR_MAXSP)    /* conserved variables per cell, at most */

struct or_mesh {
  int ndim, nxb, ng, nb, P, PZ, lmax;
  int nroot[3];
  double lo[3], hi[3], gamma;
  int bc[3][2];
  int *level, *parent, *leaf, *child; /* child: [nb][8] */
  int64_t *origin;                    /* [nb][3] */
  int64_t ncell[OR_MAXLEV][3];        /* cells per axis at each level */
  int64_t nblk[OR_MAXLEV][3];         /* blocks per axis at each level */
  double dx[OR_MAXLEV][3];
  int *lut[OR_MAXLEV];                /* dense block lookup per level */
  int nspec, nv;                      /* species; variables per cell = 5 + nspec */
  double spa[OR_MAXSP], spb[OR_MAXSP]; /* 1 / A_k and 1 / (A_k (gamma_k - 1)) */
};

static char g_err[256];
static int g_threads = 0;

const char *or_last_error(void) { return g_err; }

void or_set_threads(int n) { g_threads = n; }

int or_get_threads(void) {
#ifdef _OPENMP
  return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
  return 1;
#endif
}

static void set_err(const char *s) { snprintf(g_err, sizeof g_err, "%s", s); }

/* ------------------------------------------------------------------------ */
/* indexing                                                                  */
/* ------------------------------------------------------------------------ */

static size_t cell_index(const or_mesh *m, int b, int v, int k, int j, int i) {
  return ((((size_t)b * m->nv + v) * m->PZ + k) * m->P + j) * m->P + i;
}

static int lookup(const or_mesh *m, int l, const int64_t bcoord[3]) {
  if (l < 0 || l > m->lmax) return -1;
  for (int d = 0; d < 3; d++)
    if (bcoord[d] < 0 || bcoord[d] >= m->nblk[l][d]) return -1;
  int64_t idx = (bcoord[2] * m->nblk[l][1] + bcoord[1]) * m->nblk[l][0] + bcoord[0];
  return m->lut[l][idx];
}

/* ------------------------------------------------------------------------ */
/* mesh                                                                      */
/* ------------------------------------------------------------------------ */

void or_mesh_destroy(or_mesh *m) {
  if (!m) return;
  for (int l = 0; l < OR_MAXLEV; l++) free(m->lut[l]);
  free(m->level); free(m->parent); free(m->leaf); free(m->child); free(m->origin);
  free(m);
}

or_mesh *or_mesh_create(int ndim, int nxb, int ng, int nb, const int nroot[3],
                        const int *level, const int64_t *origin, const int *parent,
                        const double lo[3], const double hi[3], const int bc[6],
                        double gamma) {
  if ((ndim != 2 && ndim != 3) || nxb < 2 || (nxb % 2) || ng < 2 || nb < 1) {
    set_err("bad ndim/nxb/ng/nb");
    return NULL;
  }
  or_mesh *m = (or_mesh *)calloc(1, sizeof *m);
  m->ndim = ndim; m->nxb = nxb; m->ng = ng; m->nb = nb;
  m->nspec = 0; m->nv = 5;
  m->P = nxb + 2 * ng; m->PZ = ndim == 3 ? m->P : 1;
  m->gamma = gamma;
  for (int d = 0; d < 3; d++) {
    m->nroot[d] = d < ndim ? nroot[d] : 1;
    m->lo[d] = lo[d]; m->hi[d] = hi[d];
    m->bc[d][0] = bc[2 * d]; m->bc[d][1] = bc[2 * d + 1];
  }
  m->level = (int *)malloc(sizeof(int) * nb);
  m->parent = (int *)malloc(sizeof(int) * nb);
  m->leaf = (int *)malloc(sizeof(int) * nb);
  m->child = (int *)malloc(sizeof(int) * nb * 8);
  m->origin = (int64_t *)malloc(sizeof(int64_t) * nb * 3);
  m->lmax = 0;
  for (int b = 0; b < nb; b++) {
    m->level[b] = level[b];
    m->parent[b] = parent[b];
    m->leaf[b] = 1;
    for (int c = 0; c < 8; c++) m->child[b * 8 + c] = -1;
    for (int d = 0; d < 3; d++) m->origin[b * 3 + d] = d < ndim ? origin[b * 3 + d] : 0;
    if (level[b] < 0 || level[b] >= OR_MAXLEV) { set_err("bad level"); or_mesh_destroy(m); return NULL; }
    if (level[b] > m->lmax) m->lmax = level[b];
  }
  for (int l = 0; l <= m->lmax; l++) {
    int64_t tot = 1;
    for (int d = 0; d < 3; d++) {
      if (d < ndim) {
        m->nblk[l][d] = (int64_t)m->nroot[d] << l;
        m->ncell[l][d] = m->nblk[l][d] * nxb;
        m->dx[l][d] = (hi[d] - lo[d]) / (double)m->ncell[l][d];
      } else {
        m->nblk[l][d] = 1; m->ncell[l][d] = 1; m->dx[l][d] = 1.0;
      }
      tot *= m->nblk[l][d];
    }
    m->lut[l] = (int *)malloc(sizeof(int) * tot);
    for (int64_t i = 0; i < tot; i++) m->lut[l][i] = -1;
  }
  for (int b = 0; b < nb; b++) {
    int64_t bcoord[3];
    for (int d = 0; d < 3; d++) {
      int64_t o = m->origin[b * 3 + d];
      if (o % nxb) { set_err("origin not a multiple of nxb"); or_mesh_destroy(m); return NULL; }
      bcoord[d] = o / nxb;
    }
    int l = m->level[b];
    for (int d = 0; d < 3; d++)
      if (bcoord[d] < 0 || bcoord[d] >= m->nblk[l][d]) { set_err("block outside domain"); or_mesh_destroy(m); return NULL; }
    int64_t idx = (bcoord[2] * m->nblk[l][1] + bcoord[1]) * m->nblk[l][0] + bcoord[0];
    if (m->lut[l][idx] >= 0) { set_err("duplicate block"); or_mesh_destroy(m); return NULL; }
    m->lut[l][idx] = b;
  }
  for (int b = 0; b < nb; b++) {
    int p = m->parent[b];
    if (p < 0) continue;
    if (p >= nb || m->level[p] != m->level[b] - 1) { set_err("bad parent"); or_mesh_destroy(m); return NULL; }
    int oct = 0;
    for (int d = 0; d < ndim; d++) {
      int64_t rel = m->origin[b * 3 + d] - 2 * m->origin[p * 3 + d];
      if (rel != 0 && rel != nxb) { set_err("child not inside parent"); or_mesh_destroy(m); return NULL; }
      if (rel) oct |= 1 << d;
    }
    m->child[p * 8 + oct] = b;
    m->leaf[p] = 0;
  }
  for (int b = 0; b < nb; b++) {
    if (m->leaf[b]) continue;
    for (int c = 0; c < (1 << ndim); c++)
      if (m->child[b * 8 + c] < 0) { set_err("parent with missing child"); or_mesh_destroy(m); return NULL; }
  }
  return m;
}

/* ------------------------------------------------------------------------ */
/* EOS                                                                       */
/* ------------------------------------------------------------------------ */

/* Ratio of specific heats of a cell from its primitive state W (mass
 * fractions in W[5..]): the mesh's gamma for a single gas; for the
 * multispecies perfect gas the mixture of ideal gases,
 * gamma - 1 = (sum_k X_k / A_k) / (sum_k X_k / (A_k (gamma_k - 1))),
 * i.e. the ratio of the mass-weighted heat capacities. */
static double cell_gamma(const or_mesh *m, const double *W) {
  if (m->nspec == 0) return m->gamma;
  double q1 = 0.0, q2 = 0.0;
  for (int k = 0; k < m->nspec; k++) {
    q1 = q1 + W[5 + k] * m->spa[k];
    q2 = q2 + W[5 + k] * m->spb[k];
  }
  return 1.0 + q1 / q2;
}

/* Conserved from primitive with a given gamma (species: rho X_k). */
static void cons_g(const double *W, int nv, double gamma, double *U) {
  double rho = W[0];
  U[0] = rho;
  U[1] = rho * W[1];
  U[2] = rho * W[2];
  U[3] = rho * W[3];
  U[4] = W[4] / (gamma - 1.0) + 0.5 * rho * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
  for (int v = 5; v < nv; v++) U[v] = rho * W[v];
}

static void prim_from_cons(const or_mesh *m, const double *U, double *W) {
  double rho = U[0];
  W[0] = rho;
  W[1] = U[1] / rho;
  W[2] = U[2] / rho;
  W[3] = U[3] / rho;
  for (int v = 5; v < m->nv; v++) W[v] = U[v] / rho;
  double gamma = cell_gamma(m, W);
  W[4] = (gamma - 1.0) * (U[4] - 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / rho);
}

static void cons_from_prim(const or_mesh *m, const double *W, double *U) {
  cons_g(W, m->nv, cell_gamma(m, W), U);
}

int or_mesh_set_species(or_mesh *m, int nspec, const double *gamma_k, const double *A_k) {
  if (nspec < 0 || nspec > OR_MAXSP) { set_err("nspec out of range"); return -1; }
  for (int k = 0; k < nspec; k++)
    if (!(gamma_k[k] > 1.0) || !(A_k[k] > 0.0)) { set_err("bad species constants"); return -1; }
  m->nspec = nspec;
  m->nv = 5 + nspec;
  for (int k = 0; k < nspec; k++) {
    m->spa[k] = 1.0 / A_k[k];
    m->spb[k] = 1.0 / (A_k[k] * (gamma_k[k] - 1.0));
  }
  return 0;
}

static size_t ncells_total(const or_mesh *m) {
  return (size_t)m->nb * m->PZ * m->P * m->P;
}

void or_prim_to_cons(const or_mesh *m, const double *W, double *U) {
  size_t per = (size_t)m->PZ * m->P * m->P;
  int nv = m->nv;
  for (int b = 0; b < m->nb; b++)
    for (size_t c = 0; c < per; c++) {
      double w[OR_MAXV], u[OR_MAXV];
      for (int v = 0; v < nv; v++) w[v] = W[((size_t)b * nv + v) * per + c];
      cons_from_prim(m, w, u);
      for (int v = 0; v < nv; v++) U[((size_t)b * nv + v) * per + c] = u[v];
    }
  (void)ncells_total;
}

void or_cons_to_prim(const or_mesh *m, const double *U, double *W) {
  size_t per = (size_t)m->PZ * m->P * m->P;
  int nv = m->nv;
  for (int b = 0; b < m->nb; b++)
    for (size_t c = 0; c < per; c++) {
      double w[OR_MAXV], u[OR_MAXV];
      for (int v = 0; v < nv; v++) u[v] = U[((size_t)b * nv + v) * per + c];
      prim_from_cons(m, u, w);
      for (int v = 0; v < nv; v++) W[((size_t)b * nv + v) * per + c] = w[v];
    }
}

/* ------------------------------------------------------------------------ */
/* MC limiter (van Leer 1977)                                                */
/* ------------------------------------------------------------------------ */

double or_mc(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  double s = fmin(fmin(2.0 * fabs(a), 2.0 * fabs(b)), 0.5 * fabs(a + b));
  return a > 0.0 ? s : -s;
}

/* ------------------------------------------------------------------------ */
/* guard cells                                                               */
/* ------------------------------------------------------------------------ */

/* Interior value of a cell of the level-l lattice that lies inside some block
 * of level l; a non-leaf block's value is the pairwise mean of its children
 * (restriction).  g must lie inside the domain. */
static double interior_value(const or_mesh *m, const double *U, int l, const int64_t g[3],
                             int v) {
  int64_t bcoord[3];
  for (int d = 0; d < 3; d++) bcoord[d] = g[d] / m->nxb;
  int b = lookup(m, l, bcoord);
  if (b < 0) return NAN;
  if (m->leaf[b]) {
    int loc[3];
    for (int d = 0; d < 3; d++) loc[d] = (int)(g[d] - m->origin[b * 3 + d]) + (d < m->ndim ? m->ng : 0);
    return U[cell_index(m, b, v, loc[2], loc[1], loc[0])];
  }
  /* restriction: pairwise sums x first, then y, then z */
  double f[8];
  for (int c = 0; c < (1 << m->ndim); c++) {
    int64_t gf[3];
    for (int d = 0; d < 3; d++) gf[d] = d < m->ndim ? 2 * g[d] + ((c >> d) & 1) : 0;
    f[c] = interior_value(m, U, l + 1, gf, v);
  }
  if (m->ndim == 2) return ((f[0] + f[1]) + (f[2] + f[3])) * 0.25;
  return (((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7]))) * 0.125;
}

/* Value of a guard cell at level-l lattice position g (may lie outside the
 * domain).  Returns 0 on success. */
static int guard_value(const or_mesh *m, const double *U, int l, const int64_t gin[3], int v,
                       double *out) {
  int64_t g[3];
  int flip = 0;                                 /* momentum components to negate */
  for (int d = 0; d < 3; d++) {
    g[d] = gin[d];
    if (d >= m->ndim) { g[d] = 0; continue; }
    int64_t N = m->ncell[l][d];
    if (g[d] < 0 || g[d] >= N) {
      int kind = m->bc[d][g[d] < 0 ? 0 : 1];
      if (kind == 1) {
        g[d] = ((g[d] % N) + N) % N;            /* periodic: wrap */
      } else if (kind == 2) {
        g[d] = g[d] < 0 ? -1 - g[d] : 2 * N - 1 - g[d];  /* reflecting: mirror */
        if (v == 1 + d) flip ^= 1;              /* ... with the normal momentum negated */
      } else {
        g[d] = g[d] < 0 ? 0 : N - 1;            /* outflow: nearest interior cell */
      }
    }
  }
  int64_t bcoord[3];
  for (int d = 0; d < 3; d++) bcoord[d] = g[d] / m->nxb;
  int b = lookup(m, l, bcoord);
  if (b >= 0) {
    *out = interior_value(m, U, l, g, v);
    if (flip) *out = -*out;
    return 0;
  }
  /* covered by a coarser leaf: conservative MC-limited linear prolongation */
  if (l == 0) return -1;
  int64_t gc[3], cb[3];
  for (int d = 0; d < 3; d++) { gc[d] = g[d] / 2; cb[d] = gc[d] / m->nxb; }
  if (m->ndim == 2) { gc[2] = 0; cb[2] = 0; }
  int c = lookup(m, l - 1, cb);
  if (c < 0 || !m->leaf[c]) return -1;
  int loc[3];
  for (int d = 0; d < 3; d++) loc[d] = (int)(gc[d] - m->origin[c * 3 + d]) + (d < m->ndim ? m->ng : 0);
  double uc = U[cell_index(m, c, v, loc[2], loc[1], loc[0])];
  double val = uc;
  for (int d = 0; d < m->ndim; d++) {
    int lm[3] = {loc[0], loc[1], loc[2]}, lp[3] = {loc[0], loc[1], loc[2]};
    lm[d] -= 1; lp[d] += 1;
    double um = U[cell_index(m, c, v, lm[2], lm[1], lm[0])];
    double up = U[cell_index(m, c, v, lp[2], lp[1], lp[0])];
    double sigma = or_mc(uc - um, up - uc);
    double s = (g[d] % 2 == 0) ? -0.25 : 0.25;
    val = val + s * sigma;
  }
  *out = flip ? -val : val;
  return 0;
}

int or_guardcell_fill(const or_mesh *m, double *U) {
  int fail = 0;
  int P = m->P, PZ = m->PZ, ng = m->ng, n = m->nxb;
  for (int l = 0; l <= m->lmax; l++) {
#pragma omp parallel for schedule(dynamic) num_threads(or_get_threads()) reduction(| : fail)
    for (int b = 0; b < m->nb; b++) {
      if (m->level[b] != l || !m->leaf[b]) continue;
      for (int k = 0; k < PZ; k++)
        for (int j = 0; j < P; j++)
          for (int i = 0; i < P; i++) {
            int inside = (i >= ng && i < ng + n) && (j >= ng && j < ng + n) &&
                         (m->ndim == 2 || (k >= ng && k < ng + n));
            if (inside) continue;
            int64_t g[3];
            g[0] = m->origin[b * 3 + 0] + (i - ng);
            g[1] = m->origin[b * 3 + 1] + (j - ng);
            g[2] = m->ndim == 3 ? m->origin[b * 3 + 2] + (k - ng) : 0;
            for (int v = 0; v < m->nv; v++) {
              double val;
              if (guard_value(m, U, l, g, v, &val)) { fail |= 1; val = NAN; }
              U[cell_index(m, b, v, k, j, i)] = val;
            }
          }
    }
  }
  if (fail) { set_err("guard cell without a source block (mesh not 2:1 balanced?)"); return -1; }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* time step                                                                 */
/* ------------------------------------------------------------------------ */

/* Larger of two signal speeds, where a NaN wins and stays: a cell with
 * non-positive density or pressure has no sound speed, and the time step of a
 * state holding one is NaN rather than a finite value that hides the cell. */
static double sig_max(double a, double b) {
  if (isnan(a)) return a;
  if (isnan(b)) return b;
  return b > a ? b : a;
}

int or_compute_dt(const or_mesh *m, const double *U, double cfl, int form, double *dt) {
  int n = m->nxb, ng = m->ng;
  int nz = m->ndim == 3 ? n : 1, kz = m->ndim == 3 ? ng : 0;
  double *bmax = (double *)calloc((size_t)m->nb, sizeof(double));  /* per-block maxima */
#pragma omp parallel for schedule(static) num_threads(or_get_threads())
  for (int b = 0; b < m->nb; b++) {
    if (!m->leaf[b]) continue;
    const double *dx = m->dx[m->level[b]];
    double smax = 0.0;
    for (int k = 0; k < nz; k++)
      for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) {
          OR_STEP(5);   /* CFL signal speed of one cell */
          double u[OR_MAXV], w[OR_MAXV];
          for (int v = 0; v < m->nv; v++) u[v] = U[cell_index(m, b, v, k + kz, j + ng, i + ng)];
          prim_from_cons(m, u, w);
          double c = sqrt(cell_gamma(m, w) * w[4] / w[0]);
          double s = 0.0;
          for (int d = 0; d < m->ndim; d++) {
            double sd = (fabs(w[1 + d]) + c) / dx[d];
            if (form == 0) s = s + sd;
            else s = sig_max(s, sd);
          }
          smax = sig_max(smax, s);
        }
    bmax[b] = smax;
  }
  double smax = 0.0;
  for (int b = 0; b < m->nb; b++) smax = sig_max(smax, bmax[b]);
  free(bmax);
  *dt = cfl / smax;
  return isfinite(*dt) ? 0 : -4;
}

/* ------------------------------------------------------------------------ */
/* HLLC flux (Toro, Spruce & Speares 1994)                                   */
/* ------------------------------------------------------------------------ */

static void phys_flux(const double *W, const double *Uc, int nv, int d, double *F) {
  int nrm = 1 + d;
  double un = W[nrm];
  F[0] = W[0] * un;
  for (int k = 0; k < 3; k++) F[1 + k] = W[0] * un * W[1 + k];
  F[nrm] += W[4];
  F[4] = un * (Uc[4] + W[4]);
  for (int v = 5; v < nv; v++) F[v] = W[0] * un * W[v];
}

/* HLLC with the ratio of specific heats of each side (gL, gR); passive
 * species keep their side's mass fraction through the star region. */
static void hllc_core(const double *WL, const double *WR, int nv, int d, double gL, double gR,
                      double *F) {
  int nrm = 1 + d;
  double rL = WL[0], pL = WL[4], uL = WL[nrm];
  double rR = WR[0], pR = WR[4], uR = WR[nrm];
  double cL = sqrt(gL * pL / rL), cR = sqrt(gR * pR / rR);
  double SL = fmin(uL - cL, uR - cR);
  double SR = fmax(uL + cL, uR + cR);
  double UL[OR_MAXV], UR[OR_MAXV], FL[OR_MAXV], FR[OR_MAXV];
  cons_g(WL, nv, gL, UL);
  cons_g(WR, nv, gR, UR);
  phys_flux(WL, UL, nv, d, FL);
  phys_flux(WR, UR, nv, d, FR);
  double Sst = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) /
               (rL * (SL - uL) - rR * (SR - uR));
  const double *WK, *UK, *FK;
  double SK;
  if (SL >= 0.0) { for (int q = 0; q < nv; q++) F[q] = FL[q]; return; }
  if (Sst >= 0.0) { WK = WL; UK = UL; FK = FL; SK = SL; }
  else if (SR > 0.0) { WK = WR; UK = UR; FK = FR; SK = SR; }
  else { for (int q = 0; q < nv; q++) F[q] = FR[q]; return; }
  double rK = WK[0], uK = WK[nrm], pK = WK[4];
  double fac = rK * (SK - uK) / (SK - Sst);
  double Us[OR_MAXV];
  Us[0] = fac;
  for (int k = 0; k < 3; k++) Us[1 + k] = fac * WK[1 + k];
  Us[nrm] = fac * Sst;
  Us[4] = fac * (UK[4] / rK + (Sst - uK) * (Sst + pK / (rK * (SK - uK))));
  for (int q = 5; q < nv; q++) Us[q] = fac * WK[q];
  for (int q = 0; q < nv; q++) F[q] = FK[q] + SK * (Us[q] - UK[q]);
}

void or_hllc(const double WL[5], const double WR[5], int d, double gamma, double F[5]) {
  hllc_core(WL, WR, 5, d, gamma, gamma, F);
}

/* ------------------------------------------------------------------------ */
/* hydro step of one leaf block                                              */
/* ------------------------------------------------------------------------ */

typedef struct {
  double *W;    /* [nv][PZ][P][P] primitives */
  double *FSm;  /* [3][nv][PZ][P][P] face state at the lower face of a cell, per direction */
  double *FSp;  /* [3][nv][PZ][P][P] face state at the upper face */
  double *F;    /* [3][nv][PZ][P][P] flux through the lower face of a cell */
} or_work;

static size_t wi(const or_mesh *m, int v, int k, int j, int i) {
  return (((size_t)v * m->PZ + k) * m->P + j) * m->P + i;
}

/* One leaf: Unew = U + dt L(U), or with Uavg != NULL an SSP-RK stage
 * Unew = wa Uavg + wb (U + dt L(U)).  predictor = 1: MUSCL-Hancock face
 * states; 0: plain MC-limited PLM face states (method-of-lines). */
static int advance_block(const or_mesh *m, const double *U, double *Unew, double dt, int b,
                         or_work *w, double *bflux, int predictor, const double *Uavg,
                         double wa, double wb) {
  int P = m->P, PZ = m->PZ, ng = m->ng, n = m->nxb, nd = m->ndim;
  int nv = m->nv;
  size_t per = (size_t)nv * PZ * P * P;
  const double *dx = m->dx[m->level[b]];
  int lo[3], hi[3];  /* padded index range of the interior, per axis */
  for (int d = 0; d < 3; d++) {
    lo[d] = d < nd ? ng : 0;
    hi[d] = d < nd ? ng + n : 1;
  }
  /* 1. primitives on every padded cell */
  for (int k = 0; k < PZ; k++)
    for (int j = 0; j < P; j++)
      for (int i = 0; i < P; i++) {
        OR_STEP(0);   /* primitives of one cell */
        double u[OR_MAXV], q[OR_MAXV];
        for (int v = 0; v < nv; v++) u[v] = U[cell_index(m, b, v, k, j, i)];
        prim_from_cons(m, u, q);
        for (int v = 0; v < nv; v++) w->W[wi(m, v, k, j, i)] = q[v];
      }
  /* 2. slopes, Hancock predictor and face states on the interior grown by one */
  for (int k = lo[2] - (nd == 3); k < hi[2] + (nd == 3); k++)
    for (int j = lo[1] - 1; j < hi[1] + 1; j++)
      for (int i = lo[0] - 1; i < hi[0] + 1; i++) {
        OR_STEP(1);   /* slopes, predictor and face states of one cell */
        double W0[OR_MAXV], dW[3][OR_MAXV] = {{0}}, Wh[OR_MAXV], fm[3][OR_MAXV], fp[3][OR_MAXV];
        for (int v = 0; v < nv; v++) W0[v] = w->W[wi(m, v, k, j, i)];
        for (int d = 0; d < nd; d++) {
          int om[3] = {i, j, k}, op[3] = {i, j, k};
          om[d] -= 1; op[d] += 1;
          for (int v = 0; v < nv; v++) {
            double wm = w->W[wi(m, v, om[2], om[1], om[0])];
            double wp = w->W[wi(m, v, op[2], op[1], op[0])];
            dW[d][v] = or_mc(W0[v] - wm, wp - W0[v]);
          }
        }
        /* primitive quasi-linear form: A_d(W) dW_d for each direction */
        double acc[OR_MAXV] = {0};
        double gamma = cell_gamma(m, W0);
        for (int d = 0; d < nd; d++) {
          int nrm = 1 + d;
          double un = W0[nrm], r = W0[0], p = W0[4];
          double a[OR_MAXV];
          a[0] = un * dW[d][0] + r * dW[d][nrm];
          for (int t = 0; t < 3; t++) a[1 + t] = un * dW[d][1 + t];
          a[nrm] = a[nrm] + dW[d][4] / r;
          a[4] = gamma * p * dW[d][nrm] + un * dW[d][4];
          for (int v = 5; v < nv; v++) a[v] = un * dW[d][v];   /* advected mass fractions */
          for (int v = 0; v < nv; v++) acc[v] = acc[v] + a[v] / dx[d];
        }
        for (int v = 0; v < nv; v++) Wh[v] = predictor ? W0[v] - 0.5 * dt * acc[v] : W0[v];
        int bad = 0;
        for (int d = 0; d < nd; d++)
          for (int v = 0; v < nv; v++) {
            fm[d][v] = Wh[v] - 0.5 * dW[d][v];
            fp[d][v] = Wh[v] + 0.5 * dW[d][v];
          }
        for (int d = 0; d < nd; d++)
          if (!(fm[d][0] > 0.0) || !(fm[d][4] > 0.0) || !(fp[d][0] > 0.0) || !(fp[d][4] > 0.0))
            bad = 1;
        if (bad) /* positivity fallback: first order for this cell */
          for (int d = 0; d < nd; d++)
            for (int v = 0; v < nv; v++) { fm[d][v] = W0[v]; fp[d][v] = W0[v]; }
        for (int d = 0; d < nd; d++)
          for (int v = 0; v < nv; v++) {
            w->FSm[d * per + wi(m, v, k, j, i)] = fm[d][v];
            w->FSp[d * per + wi(m, v, k, j, i)] = fp[d][v];
          }
      }
  /* 3. HLLC flux through the lower face of every cell that owns a face of the
   *    interior: along d the cell index runs lo..hi (hi = upper block face). */
  for (int d = 0; d < nd; d++) {
    int hk = hi[2] + (d == 2), hj = hi[1] + (d == 1), hii = hi[0] + (d == 0);
    for (int k = lo[2]; k < hk; k++)
      for (int j = lo[1]; j < hj; j++)
        for (int i = lo[0]; i < hii; i++) {
          OR_STEP(2);   /* flux through one face */
          int o[3] = {i, j, k};
          o[d] -= 1;
          double WL[OR_MAXV], WR[OR_MAXV], F[OR_MAXV];
          for (int v = 0; v < nv; v++) {
            WL[v] = w->FSp[d * per + wi(m, v, o[2], o[1], o[0])];
            WR[v] = w->FSm[d * per + wi(m, v, k, j, i)];
          }
          hllc_core(WL, WR, nv, d, cell_gamma(m, WL), cell_gamma(m, WR), F);
          for (int v = 0; v < nv; v++) w->F[d * per + wi(m, v, k, j, i)] = F[v];
        }
  }
  /* 4. conservative update of the interior, directions summed x, y, z */
  int bad = 0;
  for (int k = lo[2]; k < hi[2]; k++)
    for (int j = lo[1]; j < hi[1]; j++)
      for (int i = lo[0]; i < hi[0]; i++) {
        OR_STEP(3);   /* conservative update of one cell */
        double un[OR_MAXV];
        for (int v = 0; v < nv; v++) {
          double div = 0.0;
          for (int d = 0; d < nd; d++) {
            int o[3] = {i, j, k};
            o[d] += 1;
            double fl = w->F[d * per + wi(m, v, k, j, i)];
            double fr = w->F[d * per + wi(m, v, o[2], o[1], o[0])];
            div = div + (fl - fr) / dx[d];
          }
          un[v] = U[cell_index(m, b, v, k, j, i)] + dt * div;
          if (Uavg) un[v] = wa * Uavg[cell_index(m, b, v, k, j, i)] + wb * un[v];
          Unew[cell_index(m, b, v, k, j, i)] = un[v];
        }
        OR_STEP(4);   /* positivity check of the new cell (a diagnostic) */
        double q[OR_MAXV];
        prim_from_cons(m, un, q);
        if (!(q[0] > 0.0) || !(q[4] > 0.0)) bad = 1;
      }
  /* 5. block-boundary fluxes for flux correction */
  if (bflux) {
    int nf = nd == 3 ? n * n : n;
    for (int d = 0; d < nd; d++)
      for (int s = 0; s < 2; s++) {
        double *dst = bflux + (((size_t)b * 2 * nd + 2 * d + s) * nv) * nf;
        int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2; /* transverse axes, lower first */
        for (int v = 0; v < m->nv; v++)
          for (int t2 = 0; t2 < (nd == 3 ? n : 1); t2++)
            for (int t1 = 0; t1 < n; t1++) {
              int c[3];
              c[d] = s == 0 ? lo[d] : hi[d];
              c[a1] = lo[a1] + t1;
              if (nd == 3) c[a2] = lo[a2] + t2; else c[2] = 0;
              dst[(size_t)v * nf + (size_t)t2 * n + t1] = w->F[d * per + wi(m, v, c[2], c[1], c[0])];
            }
      }
  }
  return bad;
}

static void reflux_block(const or_mesh *m, double *Unew, double dt, int c, const double *bflux) {
  int nd = m->ndim, n = m->nxb, ng = m->ng, l = m->level[c];
  int nf = nd == 3 ? n * n : n;
  if (l >= m->lmax) return;
  for (int d = 0; d < nd; d++)
    for (int s = 0; s < 2; s++) {
      /* same-level neighbour across this face */
      int64_t bc[3];
      for (int e = 0; e < 3; e++) bc[e] = m->origin[c * 3 + e] / n;
      bc[d] += s ? 1 : -1;
      int64_t NB = m->nblk[l][d];
      if (bc[d] < 0 || bc[d] >= NB) {
        if (m->bc[d][s] != 1) continue;
        bc[d] = (bc[d] + NB) % NB;
      }
      int nb = lookup(m, l, bc);
      if (nb < 0 || m->leaf[nb]) continue;
      int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;
      /* fine-lattice index of the fine cells on the far side of the face */
      int64_t NF = m->ncell[l + 1][d];
      int64_t gfd = s ? 2 * (m->origin[c * 3 + d] + n) : 2 * m->origin[c * 3 + d] - 1;
      gfd = ((gfd % NF) + NF) % NF;
      int fine_face = s ? 0 : 1; /* the fine block's lower (s=+) or upper face */
      const double *Fc = bflux + (((size_t)c * 2 * nd + 2 * d + s) * m->nv) * nf;
      for (int t2 = 0; t2 < (nd == 3 ? n : 1); t2++)
        for (int t1 = 0; t1 < n; t1++)
          for (int v = 0; v < m->nv; v++) {
            double f[4];
            int cnt = 0;
            for (int b2 = 0; b2 < (nd == 3 ? 2 : 1); b2++)
              for (int b1 = 0; b1 < 2; b1++) {
                int64_t gf[3] = {0, 0, 0};
                gf[d] = gfd;
                gf[a1] = 2 * (m->origin[c * 3 + a1] + t1) + b1;
                if (nd == 3) gf[a2] = 2 * (m->origin[c * 3 + a2] + t2) + b2;
                int64_t fb[3];
                for (int e = 0; e < 3; e++) fb[e] = gf[e] / n;
                int fblk = lookup(m, l + 1, fb);
                int u1 = (int)(gf[a1] - m->origin[fblk * 3 + a1]);
                int u2 = nd == 3 ? (int)(gf[a2] - m->origin[fblk * 3 + a2]) : 0;
                const double *Ff = bflux + (((size_t)fblk * 2 * nd + 2 * d + fine_face) * m->nv) * nf;
                f[cnt++] = Ff[(size_t)v * nf + (size_t)u2 * n + u1];
              }
            double fbar = nd == 3 ? ((f[0] + f[1]) + (f[2] + f[3])) * 0.25 : (f[0] + f[1]) * 0.5;
            double fc = Fc[(size_t)v * nf + (size_t)t2 * n + t1];
            int cc[3];
            cc[d] = s ? ng + n - 1 : ng;
            cc[a1] = ng + t1;
            if (nd == 3) cc[a2] = ng + t2; else cc[2] = 0;
            size_t idx = cell_index(m, c, v, cc[2], cc[1], cc[0]);
            double corr = dt * (fc - fbar) / m->dx[l][d];
            if (s) Unew[idx] = Unew[idx] + corr;
            else Unew[idx] = Unew[idx] - corr;
          }
    }
}

static void restrict_block(const or_mesh *m, double *U, int p) {
  int nd = m->ndim, n = m->nxb, ng = m->ng;
  int nz = nd == 3 ? n : 1, kz = nd == 3 ? ng : 0;
  for (int v = 0; v < m->nv; v++)
    for (int k = 0; k < nz; k++)
      for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) {
          int cx = 2 * i >= n, cy = 2 * j >= n, cz = nd == 3 && 2 * k >= n;
          int ch = m->child[p * 8 + cx + 2 * cy + 4 * cz];
          int fi = 2 * i - cx * n, fj = 2 * j - cy * n, fk = 2 * k - cz * n;
          double f[8];
          for (int c = 0; c < (1 << nd); c++) {
            int a = c & 1, bb = (c >> 1) & 1, cc = (c >> 2) & 1;
            f[c] = U[cell_index(m, ch, v, nd == 3 ? fk + cc + ng : 0, fj + bb + ng, fi + a + ng)];
          }
          double val = nd == 2 ? ((f[0] + f[1]) + (f[2] + f[3])) * 0.25
                               : (((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7]))) * 0.125;
          U[cell_index(m, p, v, k + kz, j + ng, i + ng)] = val;
        }
}

void or_restrict_parents(const or_mesh *m, double *U) {
  for (int l = m->lmax - 1; l >= 0; l--) {
#pragma omp parallel for schedule(dynamic) num_threads(or_get_threads())
    for (int b = 0; b < m->nb; b++)
      if (!m->leaf[b] && m->level[b] == l) restrict_block(m, U, b);
  }
}

int or_hydro_advance(const or_mesh *m, const double *U, double *Unew, double dt, int reflux,
                     double *bflux, int nsel, const int *sel) {
  size_t per = (size_t)m->nv * m->PZ * m->P * m->P;
  int nd = m->ndim, n = m->nxb;
  int nf = nd == 3 ? n * n : n;
  double *flux = bflux;
  int own = 0;
  if (!flux && !sel && m->lmax > 0) {
    flux = (double *)calloc((size_t)m->nb * 2 * nd * m->nv * nf, sizeof(double));
    own = 1;
  }
  int count = sel ? nsel : m->nb;
  int bad = 0;
#pragma omp parallel num_threads(or_get_threads()) reduction(| : bad)
  {
    or_work w;
    w.W = (double *)malloc(sizeof(double) * per);
    w.FSm = (double *)malloc(sizeof(double) * per * 3);
    w.FSp = (double *)malloc(sizeof(double) * per * 3);
    w.F = (double *)malloc(sizeof(double) * per * 3);
#pragma omp for schedule(dynamic)
    for (int t = 0; t < count; t++) {
      int b = sel ? sel[t] : t;
      if (!m->leaf[b]) continue;
      bad |= advance_block(m, U, Unew, dt, b, &w, flux, 1, NULL, 0.0, 1.0);
    }
    free(w.W); free(w.FSm); free(w.FSp); free(w.F);
  }
  if (!sel && m->lmax > 0) {
    if (reflux) {
#pragma omp parallel for schedule(dynamic) num_threads(or_get_threads())
      for (int b = 0; b < m->nb; b++)
        if (m->leaf[b]) reflux_block(m, Unew, dt, b, flux);
    }
    for (int l = m->lmax - 1; l >= 0; l--) {
#pragma omp parallel for schedule(dynamic) num_threads(or_get_threads())
      for (int b = 0; b < m->nb; b++)
        if (!m->leaf[b] && m->level[b] == l) restrict_block(m, Unew, b);
    }
    /* positivity after correction */
    int nz = nd == 3 ? n : 1, kz = nd == 3 ? m->ng : 0;
    for (int b = 0; b < m->nb && !bad; b++) {
      if (!m->leaf[b]) continue;
      for (int k = 0; k < nz; k++)
        for (int j = 0; j < n; j++)
          for (int i = 0; i < n; i++) {
            double u[OR_MAXV], q[OR_MAXV];
            for (int v = 0; v < m->nv; v++) u[v] = Unew[cell_index(m, b, v, k + kz, j + m->ng, i + m->ng)];
            prim_from_cons(m, u, q);
            if (!(q[0] > 0.0) || !(q[4] > 0.0)) bad = 1;
          }
    }
  }
  if (own) free(flux);
  return bad ? -4 : 0;
}

/* SSP-RK2 (Shu-Osher / Heun) with MC-limited PLM and HLLC, the second-order
 * method-of-lines family of Flash-X's Spark solver (Section 2.2):
 *   U1 = U + dt L(U);  guard fill of U1;  U2 = (U + (U1 + dt L(U1))) / 2.
 * The coarse-fine correction uses the stage-averaged fluxes (F1 + F2) / 2 on
 * both sides, which is what the two-stage update of a coarse cell used. */
int or_hydro_advance_rk2(const or_mesh *m, const double *U, double *Unew, double dt, int reflux,
                         double *bflux) {
  size_t per = (size_t)m->nv * m->PZ * m->P * m->P;
  size_t tot = per * (size_t)m->nb;
  int nd = m->ndim, n = m->nxb;
  int nf = nd == 3 ? n * n : n;
  size_t nfl = (size_t)m->nb * 2 * nd * m->nv * nf;
  double *U1 = (double *)malloc(sizeof(double) * tot);
  double *f1 = (double *)calloc(nfl, sizeof(double));
  double *f2 = (double *)calloc(nfl, sizeof(double));
  memcpy(U1, U, sizeof(double) * tot);
  int bad = 0;
  for (int stage = 0; stage < 2; stage++) {
#pragma omp parallel num_threads(or_get_threads()) reduction(| : bad)
    {
      or_work w;
      w.W = (double *)malloc(sizeof(double) * per);
      w.FSm = (double *)malloc(sizeof(double) * per * 3);
      w.FSp = (double *)malloc(sizeof(double) * per * 3);
      w.F = (double *)malloc(sizeof(double) * per * 3);
#pragma omp for schedule(dynamic)
      for (int b = 0; b < m->nb; b++) {
        if (!m->leaf[b]) continue;
        if (stage == 0) bad |= advance_block(m, U, U1, dt, b, &w, f1, 0, NULL, 0.0, 1.0);
        else bad |= advance_block(m, U1, Unew, dt, b, &w, f2, 0, U, 0.5, 0.5);
      }
      free(w.W); free(w.FSm); free(w.FSp); free(w.F);
    }
    if (stage == 0) {
      or_restrict_parents(m, U1);
      if (or_guardcell_fill(m, U1)) bad = 1;
    }
  }
  for (size_t q = 0; q < nfl; q++) f1[q] = (f1[q] + f2[q]) * 0.5;
  if (m->lmax > 0) {
    if (reflux) {
#pragma omp parallel for schedule(dynamic) num_threads(or_get_threads())
      for (int b = 0; b < m->nb; b++)
        if (m->leaf[b]) reflux_block(m, Unew, dt, b, f1);
    }
    or_restrict_parents(m, Unew);
  }
  int nz = nd == 3 ? n : 1, kz = nd == 3 ? m->ng : 0;
  for (int b = 0; b < m->nb && !bad; b++) {
    if (!m->leaf[b]) continue;
    for (int k = 0; k < nz; k++)
      for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) {
          double u[OR_MAXV], q[OR_MAXV];
          for (int v = 0; v < m->nv; v++) u[v] = Unew[cell_index(m, b, v, k + kz, j + m->ng, i + m->ng)];
          prim_from_cons(m, u, q);
          if (!(q[0] > 0.0) || !(q[4] > 0.0)) bad = 1;
        }
  }
  if (bflux) memcpy(bflux, f1, sizeof(double) * nfl);
  free(U1); free(f1); free(f2);
  return bad ? -4 : 0;
}

/* Positivity of the leaf interiors of U (0 if every cell has rho > 0, p > 0). */
static int leaves_positive(const or_mesh *m, const double *U) {
  int nd = m->ndim, n = m->nxb;
  int nz = nd == 3 ? n : 1, kz = nd == 3 ? m->ng : 0;
  for (int b = 0; b < m->nb; b++) {
    if (!m->leaf[b]) continue;
    for (int k = 0; k < nz; k++)
      for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) {
          double u[OR_MAXV], q[OR_MAXV];
          for (int v = 0; v < m->nv; v++) u[v] = U[cell_index(m, b, v, k + kz, j + m->ng, i + m->ng)];
          prim_from_cons(m, u, q);
          if (!(q[0] > 0.0) || !(q[4] > 0.0)) return 1;
        }
  }
  return 0;
}

/* SSP-RK3 of Shu and Osher (1988) with MC-limited PLM and HLLC, the
 * third-order member of the Spark family (Section 2.2):
 *   U1 = U + dt L(U)
 *   U2 = 3/4 U + 1/4 (U1 + dt L(U1))
 *   Unew = 1/3 U + 2/3 (U2 + dt L(U2)),
 * with a guard fill of U1 and of U2.  Unrolled, Unew = U + dt (L(U)/6 +
 * L(U1)/6 + 2 L(U2)/3), so the coarse-fine correction uses the fluxes
 * weighted 1/6, 1/6, 2/3 on both sides. */
int or_hydro_advance_rk3(const or_mesh *m, const double *U, double *Unew, double dt, int reflux,
                         double *bflux) {
  size_t per = (size_t)m->nv * m->PZ * m->P * m->P;
  size_t tot = per * (size_t)m->nb;
  int nd = m->ndim, n = m->nxb;
  int nf = nd == 3 ? n * n : n;
  size_t nfl = (size_t)m->nb * 2 * nd * m->nv * nf;
  double *U1 = (double *)malloc(sizeof(double) * tot);
  double *U2 = (double *)malloc(sizeof(double) * tot);
  double *f[3];
  for (int q = 0; q < 3; q++) f[q] = (double *)calloc(nfl, sizeof(double));
  memcpy(U1, U, sizeof(double) * tot);
  memcpy(U2, U, sizeof(double) * tot);
  const double wa[3] = {0.0, 0.75, 1.0 / 3.0}, wb[3] = {1.0, 0.25, 2.0 / 3.0};
  const double *src[3] = {U, U1, U2};
  double *dst[3] = {U1, U2, Unew};
  int bad = 0;
  for (int stage = 0; stage < 3; stage++) {
#pragma omp parallel num_threads(or_get_threads()) reduction(| : bad)
    {
      or_work w;
      w.W = (double *)malloc(sizeof(double) * per);
      w.FSm = (double *)malloc(sizeof(double) * per * 3);
      w.FSp = (double *)malloc(sizeof(double) * per * 3);
      w.F = (double *)malloc(sizeof(double) * per * 3);
#pragma omp for schedule(dynamic)
      for (int b = 0; b < m->nb; b++) {
        if (!m->leaf[b]) continue;
        bad |= advance_block(m, src[stage], dst[stage], dt, b, &w, f[stage], 0,
                             stage ? U : NULL, wa[stage], wb[stage]);
      }
      free(w.W); free(w.FSm); free(w.FSp); free(w.F);
    }
    if (stage < 2) {
      or_restrict_parents(m, dst[stage]);
      if (or_guardcell_fill(m, dst[stage])) bad = 1;
    }
  }
  for (size_t q = 0; q < nfl; q++)
    f[0][q] = (f[0][q] + f[1][q]) * (1.0 / 6.0) + f[2][q] * (2.0 / 3.0);
  if (m->lmax > 0) {
    if (reflux) {
#pragma omp parallel for schedule(dynamic) num_threads(or_get_threads())
      for (int b = 0; b < m->nb; b++)
        if (m->leaf[b]) reflux_block(m, Unew, dt, b, f[0]);
    }
    or_restrict_parents(m, Unew);
  }
  if (!bad) bad = leaves_positive(m, Unew);
  if (bflux) memcpy(bflux, f[0], sizeof(double) * nfl);
  free(U1); free(U2);
  for (int q = 0; q < 3; q++) free(f[q]);
  return bad ? -4 : 0;
}

/* ------------------------------------------------------------------------ */
/* regridding                                                                */
/* ------------------------------------------------------------------------ */

/* Loehner's (1987) normalised second-derivative indicator of one interior
 * cell (i, j, k) of a scalar field q given on a block's padded array
 * [PZ][P][P] (guards filled at depth 1, edges and corners included):
 *   E = sqrt( sum_{a,b} (N_ab / (dx_a dx_b))^2 / sum_{a,b} (D_ab / (dx_a dx_b))^2 )
 * over ordered direction pairs, with
 *   a = b:  N = (q+ - q0) - (q0 - q-),
 *           D = |q+ - q0| + |q0 - q-| + eps (|q+| + 2|q0| + |q-|)
 *   a != b: N = ((q++ - q-+) - (q+- - q--)) / 4,
 *           D = (|q++ - q-+| + |q+- - q--|) / 4 + eps (|q++| + |q-+| + |q+-| + |q--|) / 4
 * (first sign: direction a, second: direction b); E = 0 where the
 * denominator vanishes. */
static double loehner_cell(const or_mesh *m, const double *q, int lev, int k, int j, int i,
                           double eps) {
  int P = m->P, nd = m->ndim;
  double num = 0.0, den = 0.0;
  for (int a = 0; a < nd; a++)
    for (int b = 0; b < nd; b++) {
      double nu, de;
      if (a == b) {
        int p[3] = {i, j, k}, q_[3] = {i, j, k};
        p[a] += 1;
        q_[a] -= 1;
        double up = q[((size_t)p[2] * P + p[1]) * P + p[0]];
        double u0 = q[((size_t)k * P + j) * P + i];
        double um = q[((size_t)q_[2] * P + q_[1]) * P + q_[0]];
        nu = (up - u0) - (u0 - um);
        de = fabs(up - u0) + fabs(u0 - um) + eps * (fabs(up) + 2.0 * fabs(u0) + fabs(um));
      } else {
        double u[2][2];
        for (int sa = 0; sa < 2; sa++)
          for (int sb = 0; sb < 2; sb++) {
            int c[3] = {i, j, k};
            c[a] += sa ? 1 : -1;
            c[b] += sb ? 1 : -1;
            u[sa][sb] = q[((size_t)c[2] * P + c[1]) * P + c[0]];
          }
        nu = ((u[1][1] - u[0][1]) - (u[1][0] - u[0][0])) * 0.25;
        de = (fabs(u[1][1] - u[0][1]) + fabs(u[1][0] - u[0][0])) * 0.25 +
             eps * (fabs(u[1][1]) + fabs(u[0][1]) + fabs(u[1][0]) + fabs(u[0][0])) * 0.25;
      }
      double sc = 1.0 / (m->dx[lev][a] * m->dx[lev][b]);
      nu = nu * sc;
      de = de * sc;
      num = num + nu * nu;
      den = den + de * de;
    }
  return den > 0.0 ? sqrt(num / den) : 0.0;
}

int or_regrid_errors(const or_mesh *m, const double *U, double eps, double *err) {
  int P = m->P, PZ = m->PZ, ng = m->ng, n = m->nxb, nd = m->ndim;
  size_t plane = (size_t)PZ * P * P;
#pragma omp parallel num_threads(or_get_threads())
  {
    double *rho = (double *)malloc(sizeof(double) * plane);
    double *pre = (double *)malloc(sizeof(double) * plane);
#pragma omp for schedule(dynamic)
    for (int b = 0; b < m->nb; b++) {
      if (!m->leaf[b]) { err[b] = -1.0; continue; }
      for (size_t c = 0; c < plane; c++) {
        double u[OR_MAXV], w[OR_MAXV];
        for (int v = 0; v < m->nv; v++) u[v] = U[((size_t)b * m->nv + v) * plane + c];
        prim_from_cons(m, u, w);
        rho[c] = w[0];
        pre[c] = w[4];
      }
      double e = 0.0;
      int k0 = nd == 3 ? ng : 0, k1 = nd == 3 ? ng + n : 1;
      for (int k = k0; k < k1; k++)
        for (int j = ng; j < ng + n; j++)
          for (int i = ng; i < ng + n; i++) {
            double a = loehner_cell(m, rho, m->level[b], k, j, i, eps);
            double c2 = loehner_cell(m, pre, m->level[b], k, j, i, eps);
            if (a > e) e = a;
            if (c2 > e) e = c2;
          }
      err[b] = e;
    }
    free(rho);
    free(pre);
  }
  return 0;
}

typedef struct {
  int level;
  int64_t o[3];
  int kind, src, oct;
} rg_entry;

static int rg_cmp(const void *x, const void *y) {
  const rg_entry *a = (const rg_entry *)x, *b = (const rg_entry *)y;
  if (a->level != b->level) return a->level < b->level ? -1 : 1;
  for (int d = 2; d >= 0; d--)
    if (a->o[d] != b->o[d]) return a->o[d] < b->o[d] ? -1 : 1;
  return 0;
}

int or_regrid_plan(const or_mesh *m, const double *err, double rc, double dc, int max_level,
                   int cap, int *level_out, int64_t *origin_out, int *parent_out, int *kind_out,
                   int *src_out, int *oct_out) {
  int nb = m->nb, nd = m->ndim, n = m->nxb;
  int *ref = (int *)calloc(nb, sizeof(int));
  int *der = (int *)calloc(nb, sizeof(int));
  /* requests */
  for (int b = 0; b < nb; b++)
    if (m->leaf[b] && err[b] > rc && m->level[b] < max_level) ref[b] = 1;
  for (int p = 0; p < nb; p++) {
    if (m->leaf[p]) continue;
    int ok = 1;
    for (int c = 0; c < (1 << nd); c++) {
      int ch = m->child[p * 8 + c];
      if (!m->leaf[ch] || !(err[ch] < dc) || ref[ch]) ok = 0;
    }
    der[p] = ok;
  }
  /* 2:1 balance on a lattice of blocks one level finer than the finest */
  int Lf = m->lmax + 1;
  int64_t gn[3];
  size_t tot = 1;
  for (int d = 0; d < 3; d++) {
    gn[d] = d < nd ? ((int64_t)m->nroot[d] << Lf) : 1;
    tot *= (size_t)gn[d];
  }
  int *LV = (int *)malloc(sizeof(int) * tot);
  int *OW = (int *)malloc(sizeof(int) * tot);
  int stuck = 0;
  for (int changed = 1; changed;) {
    changed = 0;
    for (int b = 0; b < nb; b++) {
      if (!m->leaf[b]) continue;
      int X = b, lvl = m->level[b] + ref[b];
      if (m->parent[b] >= 0 && der[m->parent[b]]) { X = m->parent[b]; lvl = m->level[X]; }
      int sh = Lf - m->level[X];
      int64_t lo[3], hi[3];
      for (int d = 0; d < 3; d++) {
        if (d < nd) { lo[d] = (m->origin[X * 3 + d] / n) << sh; hi[d] = lo[d] + ((int64_t)1 << sh); }
        else { lo[d] = 0; hi[d] = 1; }
      }
      for (int64_t z = lo[2]; z < hi[2]; z++)
        for (int64_t y = lo[1]; y < hi[1]; y++)
          for (int64_t x = lo[0]; x < hi[0]; x++) {
            size_t g = ((size_t)z * gn[1] + y) * gn[0] + x;
            LV[g] = lvl;
            OW[g] = X;
          }
    }
    for (int64_t z = 0; z < gn[2]; z++)
      for (int64_t y = 0; y < gn[1]; y++)
        for (int64_t x = 0; x < gn[0]; x++) {
          size_t g = ((size_t)z * gn[1] + y) * gn[0] + x;
          int X = OW[g];
          int need = 0;
          for (int dz = (nd == 3 ? -1 : 0); dz <= (nd == 3 ? 1 : 0) && !need; dz++)
            for (int dy = -1; dy <= 1 && !need; dy++)
              for (int dx = -1; dx <= 1 && !need; dx++) {
                int64_t h[3] = {x + dx, y + dy, z + dz};
                int skip = 0;
                for (int d = 0; d < nd; d++) {
                  if (h[d] < 0 || h[d] >= gn[d]) {
                    if (m->bc[d][h[d] < 0 ? 0 : 1] == 1) h[d] = (h[d] + gn[d]) % gn[d];
                    else skip = 1;
                  }
                }
                if (skip) continue;
                size_t gh = ((size_t)h[2] * gn[1] + h[1]) * gn[0] + h[0];
                if (LV[gh] > LV[g] + 1) need = 1;
              }
          if (!need) continue;
          if (!m->leaf[X]) {                  /* a coarsening that would unbalance */
            if (der[X]) { der[X] = 0; changed = 1; }
          } else if (!ref[X]) {               /* a leaf too coarse next to finer ones */
            ref[X] = 1;
            changed = 1;
          } else if (LV[g] == m->level[X] + 1) {
            stuck = 1;                        /* refined already: not reachable from a
                                                 balanced mesh */
          }
        }
    if (stuck) break;
  }
  free(LV);
  free(OW);
  if (stuck) { free(ref); free(der); set_err("regrid: mesh not 2:1 balanced"); return -1; }
  /* the new block list */
  rg_entry *e = (rg_entry *)malloc(sizeof(rg_entry) * ((size_t)nb * (1 + (1 << nd))));
  int ne = 0;
  for (int b = 0; b < nb; b++) {
    if (m->parent[b] >= 0 && der[m->parent[b]]) continue;
    e[ne].level = m->level[b];
    for (int d = 0; d < 3; d++) e[ne].o[d] = m->origin[b * 3 + d];
    e[ne].kind = 0; e[ne].src = b; e[ne].oct = 0;
    ne++;
    if (m->leaf[b] && ref[b])
      for (int c = 0; c < (1 << nd); c++) {
        e[ne].level = m->level[b] + 1;
        for (int d = 0; d < 3; d++)
          e[ne].o[d] = d < nd ? 2 * m->origin[b * 3 + d] + (((c >> d) & 1) ? n : 0) : 0;
        e[ne].kind = 1; e[ne].src = b; e[ne].oct = c;
        ne++;
      }
  }
  free(ref);
  free(der);
  if (ne > cap) { free(e); set_err("regrid: output capacity too small"); return -1; }
  qsort(e, ne, sizeof(rg_entry), rg_cmp);
  for (int i = 0; i < ne; i++) {
    level_out[i] = e[i].level;
    for (int d = 0; d < 3; d++) origin_out[i * 3 + d] = e[i].o[d];
    kind_out[i] = e[i].kind; src_out[i] = e[i].src; oct_out[i] = e[i].oct;
    parent_out[i] = -1;
    if (e[i].level == 0) continue;
    rg_entry key;
    key.level = e[i].level - 1;
    for (int d = 0; d < 3; d++) key.o[d] = d < nd ? ((e[i].o[d] / n) / 2) * n : 0;
    rg_entry *f = (rg_entry *)bsearch(&key, e, ne, sizeof(rg_entry), rg_cmp);
    if (!f) { free(e); set_err("regrid: block without parent"); return -1; }
    parent_out[i] = (int)(f - e);
  }
  free(e);
  return ne;
}

/* Conservative MC-limited linear prolongation of variable v of parent
 * block s, coarse cell pc (padded indices), to the fine cell whose fine
 * parities along x, y, z are par[] (0 lower half, 1 upper half). */
static double prolong_value(const or_mesh *om, const double *Uold, int s, int v, const int pc[3],
                            const int par[3]) {
  int nd = om->ndim;
  double uc = Uold[cell_index(om, s, v, pc[2], pc[1], pc[0])];
  double val = uc;
  for (int d = 0; d < nd; d++) {
    int lm[3] = {pc[0], pc[1], pc[2]}, lp[3] = {pc[0], pc[1], pc[2]};
    lm[d] -= 1;
    lp[d] += 1;
    double um = Uold[cell_index(om, s, v, lm[2], lm[1], lm[0])];
    double up = Uold[cell_index(om, s, v, lp[2], lp[1], lp[0])];
    double sigma = or_mc(uc - um, up - uc);
    double sg = par[d] ? 0.25 : -0.25;
    val = val + sg * sigma;
  }
  return val;
}

int or_regrid_transfer(const or_mesh *om, const double *Uold, const or_mesh *nm, const int *kind,
                       const int *src, const int *oct, double *Unew) {
  int n = nm->nxb, ng = nm->ng, nd = nm->ndim;
  int nz = nd == 3 ? n : 1, kz = nd == 3 ? ng : 0;
#pragma omp parallel for schedule(dynamic) num_threads(or_get_threads())
  for (int b = 0; b < nm->nb; b++) {
    int s = src[b];
    for (int k = 0; k < nz; k++)
      for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) {
          double out[OR_MAXV];
          if (kind[b] == 0) {
            for (int v = 0; v < nm->nv; v++) out[v] = Uold[cell_index(om, s, v, k + kz, j + ng, i + ng)];
          } else {
            /* new child: the parent's coarse cell and this cell's parities */
            int f[3] = {i, j, k}, pc[3], par[3];
            for (int d = 0; d < 3; d++) {
              int fine = d < nd ? ((oct[b] >> d) & 1) * n + f[d] : 0;
              pc[d] = d < nd ? fine / 2 + ng : 0;
              par[d] = fine % 2;
            }
            /* linear prolongation, unless it leaves a non-positive density
             * or pressure in any of the coarse cell's 2^d children: then
             * all of them take the coarse value (still conservative) */
            int ok = 1;
            for (int c = 0; c < (1 << nd) && ok; c++) {
              int pq[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
              double u[OR_MAXV], w[OR_MAXV];
              for (int v = 0; v < om->nv; v++) u[v] = prolong_value(om, Uold, s, v, pc, pq);
              prim_from_cons(om, u, w);
              if (!(w[0] > 0.0) || !(w[4] > 0.0)) ok = 0;
            }
            for (int v = 0; v < nm->nv; v++)
              out[v] = ok ? prolong_value(om, Uold, s, v, pc, par)
                          : Uold[cell_index(om, s, v, pc[2], pc[1], pc[0])];
          }
          for (int v = 0; v < nm->nv; v++) Unew[cell_index(nm, b, v, k + kz, j + ng, i + ng)] = out[v];
        }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* conserved totals                                                          */
/* ------------------------------------------------------------------------ */

void or_conserved_totals(const or_mesh *m, const double *U, double *out) {
  int n = m->nxb, ng = m->ng, nd = m->ndim;
  int nz = nd == 3 ? n : 1, kz = nd == 3 ? ng : 0;
  for (int v = 0; v < m->nv; v++) {
    double sum = 0.0, comp = 0.0;
    for (int b = 0; b < m->nb; b++) {
      if (!m->leaf[b]) continue;
      const double *dx = m->dx[m->level[b]];
      double dV = dx[0] * dx[1] * (nd == 3 ? dx[2] : 1.0);
      double bs = 0.0, bcmp = 0.0;
      for (int k = 0; k < nz; k++)
        for (int j = 0; j < n; j++)
          for (int i = 0; i < n; i++) {
            double y = U[cell_index(m, b, v, k + kz, j + ng, i + ng)] - bcmp;
            double t = bs + y;
            bcmp = (t - bs) - y;
            bs = t;
          }
      double y = bs * dV - comp;
      double t = sum + y;
      comp = (t - sum) - y;
      sum = t;
    }
    out[v] = sum;
  }
}
