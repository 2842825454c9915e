// grid_ops.cuh -- device bodies of the Grid-side operations, shared by the
// per-block-set kernels (k_grid.cu, k_amr.cu) and the batched step
// (k_batch.cu).  Each body handles one unit of work (a parent chunk, a padded
// z-plane of a leaf, a chunk of a coarse block's cells) for one block set
// described by a DevMesh.
//
// Paper: Flash-X (arXiv 2208.11630), Section 2 -- the Grid reconciles block
// boundaries across refinement levels between the per-block physics updates.
// Operators (textbook block-AMR): pairwise-mean restriction, same-level copy
// with outflow/periodic/reflecting boundaries, MC-limited conservative linear
// prolongation, Berger & Colella (1989) flux correction.
#pragma once

#include "eos.cuh"
#include "slot_map.cuh"

namespace fx {
namespace ops {

// Pressure from conserved variables u[0..nvar) (FP64).
__device__ __forceinline__ double cons_pressure(const DevMesh &m, const double *u) {
  double X[FX_MAXSPEC];
  for (int k = 0; k < m.nspec; ++k) X[k] = u[5 + k] / u[0];
  double g, gm1;
  mix_gamma<double>(m, X, m.nspec, g, gm1);
  return gm1 * (u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0]);
}

template <typename S>
__device__ __forceinline__ double ld(const S *p) { return static_cast<double>(*p); }

template <typename S>
__device__ __forceinline__ void st(S *p, double v) { *p = static_cast<S>(v); }

// Level-lattice index g mapped into [0, N) by the boundary kind of the side
// it lies beyond: periodic wraps, reflecting mirrors about the wall (sets
// `mirror`, the caller negates the wall-normal momentum), outflow clamps.
__device__ __forceinline__ int apply_bc(int g, int N, int kind_lo, int kind_hi, bool &mirror) {
  if (g < 0) {
    if (kind_lo == FX_BC_PERIODIC) return ((g % N) + N) % N;
    if (kind_lo == FX_BC_REFLECT) { mirror = true; return -1 - g; }
    return 0;
  }
  if (g >= N) {
    if (kind_hi == FX_BC_PERIODIC) return g % N;
    if (kind_hi == FX_BC_REFLECT) { mirror = true; return 2 * N - 1 - g; }
    return N - 1;
  }
  return g;
}

// van Leer's MC limiter.
__device__ __forceinline__ double mc_lim(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  double s = fmin(fmin(2.0 * fabs(a), 2.0 * fabs(b)), 0.5 * fabs(a + b));
  return a > 0.0 ? s : -s;
}

__device__ __forceinline__ int slot_of(int i, int lo, int hi) {
  return i < lo ? 0 : (i >= hi ? 2 : 1);
}

// Parent p, interior cells [chunk*blockDim, (chunk+1)*blockDim): the pairwise
// mean of the 2^d child cells (x pairs first, then y, then z), which restricts
// a uniform field to itself exactly.  Computed in the state's precision: an
// FP32 state converted to FP64 would put eight conversions and eight
// operations per value on the FP64 pipe, which this GPU runs at 1/64 of the
// FP32 rate (parents are guard sources only, never updated leaves).
template <typename S>
__device__ __forceinline__ void restrict_cells(const DevMesh &m, S *__restrict__ U, int p,
                                               int chunk) {
  const int n = m.nxb, ng = m.ng, P = m.P;
  const int nz = m.ndim == 3 ? n : 1;
  const int ncell = n * n * nz;
  const int c = chunk * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int i = c % n, j = (c / n) % n, k = c / (n * n);
  const int cx = 2 * i >= n, cy = 2 * j >= n, cz = (m.ndim == 3) && (2 * k >= n);
  const int ch = m.child[p * 8 + cx + 2 * cy + 4 * cz];
  const int fi = 2 * i - cx * n + ng, fj = 2 * j - cy * n + ng;
  const int fk = m.ndim == 3 ? 2 * k - cz * n + ng : 0;
  const S *F = U + (long long)ch * m.bstride;
  S *D = U + (long long)p * m.bstride;
  const int dk = m.ndim == 3 ? k + ng : 0;
  for (int v = 0; v < m.nvar; ++v) {
    const S *f = F + v * m.vstride + ((long long)fk * P + fj) * P + fi;
    S r;
    if (m.ndim == 2) {
      r = ((f[0] + f[1]) + (f[P] + f[P + 1])) * S(0.25);
    } else {
      const S *g = f + (long long)P * P;
      r = (((f[0] + f[1]) + (f[P] + f[P + 1])) + ((g[0] + g[1]) + (g[P] + g[P + 1]))) * S(0.125);
    }
    D[v * m.vstride + ((long long)dk * P + (j + ng)) * P + (i + ng)] = r;
  }
}

// Chebyshev distance of padded index i outside [lo, hi) (0 inside).
__device__ __forceinline__ int outside(int i, int lo, int hi) {
  return i < lo ? lo - i : (i >= hi ? i - hi + 1 : 0);
}

// Leaf b, padded z-plane k, whole CTA: every guard cell within `depth` of
// the interior (Chebyshev distance) whose slot is a same-level copy reads the
// source block's interior at the boundary-mapped global position.
template <typename S>
__device__ __forceinline__ void guard_copy_plane(const DevMesh &m, S *__restrict__ U, int b,
                                                 int k, int depth) {
  // per slot: its kind and its source as a linear map (slot_map.cuh)
  __shared__ int2 sl[27];
  __shared__ long long soff[27];
  __shared__ int4 smap[27];
  __syncthreads();
  if (threadIdx.x < 27) {
    sl[threadIdx.x] = m.slots[b * 27 + threadIdx.x];
    guard_source(m, b, threadIdx.x, soff[threadIdx.x], smap[threadIdx.x]);
  }
  __syncthreads();
  const int P = m.P, ng = m.ng, n = m.nxb;
  const int dz = m.ndim == 3 ? outside(k, ng, ng + n) : 0;
  if (dz > depth) return;
  const int sz = m.ndim == 3 ? slot_of(k, ng, ng + n) : 1;
  const long long vs = m.vstride;
  S *Ub = U + (long long)b * m.bstride;
  // the plane's cells within `depth` of the interior: a window of W x W
  const int W = n + 2 * depth, i0 = ng - depth;
  for (int c = threadIdx.x; c < W * W; c += blockDim.x) {
    const int i = i0 + c % W, j = i0 + c / W;
    const int q = slot_of(i, ng, ng + n) + 3 * slot_of(j, ng, ng + n) + 9 * sz;
    if (q == 13 || sl[q].x != SLOT_COPY) continue;
    const int4 mq = smap[q];
    const S *Us = U + (soff[q] + (i * mq.x + j * mq.y + k * mq.z));
    S *Ud = Ub + ((long long)k * P + j) * P + i;
    for (int v = 0; v < m.nvar; ++v) {
      const S x = Us[v * vs];
      Ud[v * vs] = (v >= 1 && v <= 3 && ((mq.w >> (v - 1)) & 1)) ? -x : x;
    }
  }
}

// MC limiter in the compute precision C (same definition as mc_lim).
template <typename C>
__device__ __forceinline__ C mc_lim_c(C a, C b) {
  if (a * b <= C(0)) return C(0);
  C s = fmin(fmin(C(2) * fabs(a), C(2) * fabs(b)), C(0.5) * fabs(a + b));
  return a > C(0) ? s : -s;
}

// Guard cell (i, j, k) (padded indices) of leaf b covered by coarse leaf cb:
// U_c + sum_d s_d MC(U_c - U_{c-e_d}, U_{c+e_d} - U_c) per variable, s_d =
// -1/4 for the lower fine half of the coarse cell along d and +1/4 for the
// upper half, summed x, y, z, in precision C; mirrored (and the wall-normal
// momentum negated) beyond a reflecting wall.
template <typename S, typename C>
__device__ __forceinline__ void prolong_guard_cell(const DevMesh &m, S *__restrict__ U, int b,
                                                   int cb, int i, int j, int k) {
  const int P = m.P, ng = m.ng, lev = m.level[b];
  const long long sP = P, sPP = (long long)P * P;
  int g[3];
  bool mir[3] = {false, false, false};
  g[0] = apply_bc(m.origin[3 * b] + i - ng, m.ncell[lev][0], m.bc[0][0], m.bc[0][1], mir[0]);
  g[1] = apply_bc(m.origin[3 * b + 1] + j - ng, m.ncell[lev][1], m.bc[1][0], m.bc[1][1], mir[1]);
  g[2] = m.ndim == 3 ? apply_bc(m.origin[3 * b + 2] + k - ng, m.ncell[lev][2], m.bc[2][0],
                                m.bc[2][1], mir[2])
                     : 0;
  const int cx = (g[0] >> 1) - m.origin[3 * cb] + ng;
  const int cy = (g[1] >> 1) - m.origin[3 * cb + 1] + ng;
  const int cz = m.ndim == 3 ? (g[2] >> 1) - m.origin[3 * cb + 2] + ng : 0;
  const S *Cc = U + (long long)cb * m.bstride + (cz * sPP + cy * sP + cx);
  S *Ud = U + (long long)b * m.bstride + ((long long)k * P + j) * P + i;
  const long long step[3] = {1, sP, sPP};
  for (int v = 0; v < m.nvar; ++v) {
    const S *cv = Cc + v * m.vstride;
    const C uc = C(*cv);
    C val = uc;
    for (int d = 0; d < m.ndim; ++d) {
      const C um = C(cv[-step[d]]), up = C(cv[step[d]]);
      const C sig = mc_lim_c<C>(uc - um, up - uc);
      const C off = (g[d] & 1) ? C(0.25) : C(-0.25);
      val = val + off * sig;
    }
    if (v >= 1 && v <= 3 && mir[v - 1]) val = -val;
    Ud[v * m.vstride] = S(val);
  }
}

// Leaf b, neighbour slot `slot` ((sx+1) + 3 (sy+1) + 9 (sz+1)) covered by a
// coarser leaf: every guard cell of that slot within `depth` of the
// interior, work items [first, ...) strided by `stride`.  The work is the
// slot's own cells (depth x n x n for a face slot, depth^2 x n for an edge,
// depth^3 for a corner), not the whole padded block.
//
// With an even depth and nxb (block origins are multiples of nxb), the two
// fine cells of every aligned pair along an axis map to one coarse cell under
// each boundary mapping (interior, periodic shift, reflecting mirror, outflow
// clamp), so a work item is one coarse cell: its MC slopes are formed once
// and its 2^d fine children written with the per-cell formula of
// prolong_guard_cell (same operations, same order, same values).  Otherwise
// a work item is one fine cell.
template <typename S, typename C = double>
__device__ __forceinline__ void guard_prolong_slot(const DevMesh &m, S *__restrict__ U, int b,
                                                   int slot, int depth, int first, int stride) {
  const int n = m.nxb, ng = m.ng, nd = m.ndim;
  const int2 sl = m.slots[b * 27 + slot];
  const int s3[3] = {slot % 3, (slot / 3) % 3, slot / 9};
  int lo[3], w[3];
  for (int d = 0; d < 3; ++d) {
    if (d >= nd) { lo[d] = 0; w[d] = 1; continue; }
    lo[d] = s3[d] == 0 ? ng - depth : (s3[d] == 1 ? ng : ng + n);
    w[d] = s3[d] == 1 ? n : depth;
  }
  if ((depth & 1) || (n & 1)) {
    const int ncell = w[0] * w[1] * w[2];
    for (int c = first; c < ncell; c += stride) {
      const int i = lo[0] + c % w[0], j = lo[1] + (c / w[0]) % w[1], k = lo[2] + c / (w[0] * w[1]);
      prolong_guard_cell<S, C>(m, U, b, sl.y, i, j, k);
    }
    return;
  }
  const int P = m.P, lev = m.level[b], cb = sl.y;
  const long long sP = P, sPP = (long long)P * P;
  const long long step[3] = {1, sP, sPP};
  const int h[3] = {w[0] / 2, w[1] / 2, nd == 3 ? w[2] / 2 : 1};
  const int nco = h[0] * h[1] * h[2];
  const int nch = nd == 3 ? 8 : 4;
  for (int c = first; c < nco; c += stride) {
    const int q[3] = {c % h[0], (c / h[0]) % h[1], c / (h[0] * h[1])};
    // the children's padded indices and, per axis, their lattice indices and
    // mirror flags after the boundary mapping (the pair shares its coarse cell)
    int fi[3][2], gi[3][2];
    bool mir[3] = {false, false, false};
    for (int d = 0; d < 3; ++d) {
      for (int e = 0; e < 2; ++e) {
        fi[d][e] = lo[d] + (d < nd ? 2 * q[d] + e : 0);
        gi[d][e] = d < nd ? apply_bc(m.origin[3 * b + d] + fi[d][e] - ng, m.ncell[lev][d],
                                     m.bc[d][0], m.bc[d][1], mir[d])
                          : 0;
      }
    }
    const int cx = (gi[0][0] >> 1) - m.origin[3 * cb] + ng;
    const int cy = (gi[1][0] >> 1) - m.origin[3 * cb + 1] + ng;
    const int cz = nd == 3 ? (gi[2][0] >> 1) - m.origin[3 * cb + 2] + ng : 0;
    const S *Cc = U + (long long)cb * m.bstride + (cz * sPP + cy * sP + cx);
    S *Ub = U + (long long)b * m.bstride;
    for (int v = 0; v < m.nvar; ++v) {
      const S *cv = Cc + v * m.vstride;
      const C uc = C(*cv);
      C sig[3];
      for (int d = 0; d < nd; ++d) {
        const C um = C(cv[-step[d]]), up = C(cv[step[d]]);
        sig[d] = mc_lim_c<C>(uc - um, up - uc);
      }
      const bool neg = v >= 1 && v <= 3 && mir[v - 1];
      for (int ch = 0; ch < nch; ++ch) {
        const int e[3] = {ch & 1, (ch >> 1) & 1, (ch >> 2) & 1};
        C val = uc;
        for (int d = 0; d < nd; ++d) {
          const C off = (gi[d][e[d]] & 1) ? C(0.25) : C(-0.25);
          val = val + off * sig[d];
        }
        if (neg) val = -val;
        const int k = nd == 3 ? fi[2][e[2]] : 0;
        Ub[((long long)k * P + fi[1][e[1]]) * P + fi[0][e[0]] + v * m.vstride] = S(val);
      }
    }
  }
}

// Coarse leaf it.block, cells [first, ncell) strided by `stride`: replace the
// coarse face flux F_c by the pairwise mean F_bar of the fine face fluxes,
//   upper face: U_c += dt/dx (F_c - F_bar); lower face: U_c -= dt/dx (F_c - F_bar),
// in the order x-, x+, y-, y+, z-, z+.  If smax is given, the corrected cell's
// CFL signal speed (state precision) joins the maximum.
template <typename S>
__device__ __forceinline__ void reflux_cells(const DevMesh &m, S *__restrict__ Unew,
                                             const RefluxItem &it, double dt,
                                             const double *__restrict__ regs,
                                             int *__restrict__ status,
                                             unsigned long long *__restrict__ smax, int form,
                                             int first, int stride) {
  const int c = it.block;
  const int n = m.nxb, ng = m.ng, P = m.P, nd = m.ndim;
  const int nz = nd == 3 ? n : 1;
  const int lev = m.level[c];
  const int nfc = m.nface_cells;
  const int nv = m.nvar;
  const long long rstride = (long long)m.nfaces * nv * nfc;
  const double *Fc = regs + (long long)m.regidx[c] * rstride;
  S *Uc = Unew + (long long)c * m.bstride;
  const int ncell = n * n * nz;
  for (int cell = first; cell < ncell; cell += stride) {
    const int ci[3] = {cell % n, (cell / n) % n, cell / (n * n)};
    bool surf = false;   // only cells on the block surface can be corrected
    for (int d = 0; d < nd; ++d) surf |= (ci[d] == 0 || ci[d] == n - 1);
    if (!surf) continue;
    const long long o = ((long long)(nd == 3 ? ci[2] + ng : 0) * P + (ci[1] + ng)) * P + (ci[0] + ng);
    double u[FX_MAXVAR];
    bool touched = false;
    for (int d = 0; d < nd; ++d) {
      const int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;
      for (int s = 0; s < 2; ++s) {
        const int f = 2 * d + s;
        if (it.fine[f][0] < 0) continue;
        if (ci[d] != (s ? n - 1 : 0)) continue;
        if (!touched) {
          for (int v = 0; v < nv; ++v) u[v] = double(Uc[o + v * m.vstride]);
          touched = true;
        }
        const int t1 = ci[a1], t2 = nd == 3 ? ci[a2] : 0;
        const int h1 = 2 * t1 >= n, h2 = nd == 3 && 2 * t2 >= n;
        const double *Ff = regs + (long long)it.fine[f][h1 + 2 * h2] * rstride;
        const int ff = 2 * d + (s ? 0 : 1);
        const int u1 = 2 * t1 - h1 * n, u2 = nd == 3 ? 2 * t2 - h2 * n : 0;
        for (int v = 0; v < nv; ++v) {
          const double *fv = Ff + (long long)(ff * nv + v) * nfc;
          double fbar;
          if (nd == 3) {
            fbar = ((fv[u2 * n + u1] + fv[u2 * n + u1 + 1]) +
                    (fv[(u2 + 1) * n + u1] + fv[(u2 + 1) * n + u1 + 1])) * 0.25;
          } else {
            fbar = (fv[u1] + fv[u1 + 1]) * 0.5;
          }
          const double fc = Fc[(long long)(f * nv + v) * nfc + t2 * n + t1];
          const double corr = dt * (fc - fbar) * m.idx[lev][d];
          u[v] = s ? u[v] + corr : u[v] - corr;
        }
      }
    }
    if (touched) {
      S us[FX_MAXVAR];
      for (int v = 0; v < nv; ++v) { us[v] = S(u[v]); Uc[o + v * m.vstride] = us[v]; }
      if (!(u[0] > 0.0) || !(2.0 * u[4] * u[0] > u[1] * u[1] + u[2] * u[2] + u[3] * u[3]))
        atomicOr(status, 1);
      if (smax) {
        // CFL signal speed of the corrected cell, in the state's precision
        const SignalConsts<S> k0(m, lev);
        const S sg = cell_signal<S>(m, us, m.nspec, k0, form);
        atomicMax(smax, (unsigned long long)__double_as_longlong(double(sg)));
      }
    }
  }
}

}  // namespace ops
}  // namespace fx
