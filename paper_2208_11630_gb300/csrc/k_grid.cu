// k_grid.cu -- Grid-side kernels of the block-AMR hot path: primitive to
// conserved conversion, restriction into parents, same-level guard copy with
// physical boundaries, and conservative MC-limited linear prolongation.
//
// Paper: Flash-X (arXiv 2208.11630), Section 2 -- physics updates blocks one by
// one and calls the Grid to reconcile block boundaries across refinement
// levels; the grid is a uniform grid or a PARAMESH octree.  The concrete operators (pairwise-mean
// restriction, MC-limited conservative prolongation, zero-gradient outflow)
// are the textbook block-AMR ones.
//
// All kernels are HBM-bound copies/stencils; x is the fastest axis and each
// CTA walks one padded z-plane so that warps read and write contiguous rows.
#include "fx_internal.h"

namespace fx {
namespace {

template <typename S>
__device__ __forceinline__ double ld(const S *p) { return static_cast<double>(*p); }

template <typename S>
__device__ __forceinline__ void st(S *p, double v) { *p = static_cast<S>(v); }

__device__ __forceinline__ int apply_bc(int g, int N, int kind_lo, int kind_hi) {
  if (g < 0) return kind_lo == 1 ? ((g % N) + N) % N : 0;
  if (g >= N) return kind_hi == 1 ? g % N : N - 1;
  return g;
}

// van Leer's MC limiter.
__device__ __forceinline__ double mc_lim(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  double s = fmin(fmin(2.0 * fabs(a), 2.0 * fabs(b)), 0.5 * fabs(a + b));
  return a > 0.0 ? s : -s;
}

template <typename S>
__global__ void k_prim_to_cons(DevMesh m, const double *__restrict__ W, S *__restrict__ U) {
  const long long per = m.vstride;
  const long long total = (long long)m.nb * per;
  const double igm1 = 1.0 / (m.gamma - 1.0);
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total;
       c += (long long)gridDim.x * blockDim.x) {
    const long long b = c / per, o = c % per;
    const double *w = W + b * m.bstride + o;
    S *u = U + b * m.bstride + o;
    double r = w[0], vx = w[per], vy = w[2 * per], vz = w[3 * per], p = w[4 * per];
    st(u, r);
    st(u + per, r * vx);
    st(u + 2 * per, r * vy);
    st(u + 3 * per, r * vz);
    st(u + 4 * per, p * igm1 + 0.5 * r * (vx * vx + vy * vy + vz * vz));
  }
}

// One CTA per (parent, chunk of interior cells): the parent's interior cell
// is the pairwise mean of the 2^d child cells it covers (x pairs first, then
// y, then z), which restricts a uniform field to itself exactly.
template <typename S>
__global__ void k_restrict(DevMesh m, S *__restrict__ U, const int *__restrict__ parents) {
  const int p = parents[blockIdx.x];
  const int n = m.nxb, ng = m.ng, P = m.P;
  const int nz = m.ndim == 3 ? n : 1;
  const int ncell = n * n * nz;
  const int c = blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int i = c % n, j = (c / n) % n, k = c / (n * n);
  const int cx = 2 * i >= n, cy = 2 * j >= n, cz = (m.ndim == 3) && (2 * k >= n);
  const int ch = m.child[p * 8 + cx + 2 * cy + 4 * cz];
  const int fi = 2 * i - cx * n + ng, fj = 2 * j - cy * n + ng;
  const int fk = m.ndim == 3 ? 2 * k - cz * n + ng : 0;
  const S *F = U + (long long)ch * m.bstride;
  S *D = U + (long long)p * m.bstride;
  const int dk = m.ndim == 3 ? k + ng : 0;
  for (int v = 0; v < 5; ++v) {
    const S *f = F + v * m.vstride + ((long long)fk * P + fj) * P + fi;
    double r;
    if (m.ndim == 2) {
      r = ((ld(f) + ld(f + 1)) + (ld(f + P) + ld(f + P + 1))) * 0.25;
    } else {
      const S *g = f + (long long)P * P;
      r = (((ld(f) + ld(f + 1)) + (ld(f + P) + ld(f + P + 1))) +
           ((ld(g) + ld(g + 1)) + (ld(g + P) + ld(g + P + 1)))) * 0.125;
    }
    st(D + v * m.vstride + ((long long)dk * P + (j + ng)) * P + (i + ng), r);
  }
}

__device__ __forceinline__ int slot_of(int i, int lo, int hi) {
  return i < lo ? 0 : (i >= hi ? 2 : 1);
}

// One CTA per (leaf, padded z-plane): every guard cell whose slot is a
// same-level copy reads the source block's interior at the boundary-mapped
// global position.
template <typename S>
__global__ void k_guard_copy(DevMesh m, S *__restrict__ U, const int *__restrict__ leaves) {
  const int b = leaves[blockIdx.x];
  const int k = blockIdx.y;
  __shared__ int2 sl[27];
  if (threadIdx.x < 27) sl[threadIdx.x] = m.slots[b * 27 + threadIdx.x];
  __syncthreads();
  const int P = m.P, ng = m.ng, n = m.nxb, lev = m.level[b];
  const int sz = m.ndim == 3 ? slot_of(k, ng, ng + n) : 1;
  const int ox = m.origin[3 * b], oy = m.origin[3 * b + 1], oz = m.origin[3 * b + 2];
  S *Ub = U + (long long)b * m.bstride;
  for (int c = threadIdx.x; c < P * P; c += blockDim.x) {
    const int i = c % P, j = c / P;
    const int sx = slot_of(i, ng, ng + n), sy = slot_of(j, ng, ng + n);
    if (sx == 1 && sy == 1 && sz == 1) continue;
    const int2 s = sl[sx + 3 * sy + 9 * sz];
    if (s.x != SLOT_COPY) continue;
    const int gx = apply_bc(ox + i - ng, m.ncell[lev][0], m.bc[0][0], m.bc[0][1]);
    const int gy = apply_bc(oy + j - ng, m.ncell[lev][1], m.bc[1][0], m.bc[1][1]);
    const int src = s.y;
    const int lx = gx - m.origin[3 * src] + ng, ly = gy - m.origin[3 * src + 1] + ng;
    int lz = 0;
    if (m.ndim == 3) {
      const int gz = apply_bc(oz + k - ng, m.ncell[lev][2], m.bc[2][0], m.bc[2][1]);
      lz = gz - m.origin[3 * src + 2] + ng;
    }
    const S *Us = U + (long long)src * m.bstride + ((long long)lz * P + ly) * P + lx;
    S *Ud = Ub + ((long long)k * P + j) * P + i;
#pragma unroll
    for (int v = 0; v < 5; ++v) Ud[v * m.vstride] = Us[v * m.vstride];
  }
}

// One CTA per (leaf, padded z-plane): guard cells covered by a coarser leaf
// get U_c + sum_d s_d MC(U_c - U_{c-e_d}, U_{c+e_d} - U_c), s_d = -1/4 for the
// lower fine half of the coarse cell along d and +1/4 for the upper half,
// summed x, y, z.  The coarse leaf's own guards (depth 1) must be filled.
template <typename S>
__global__ void k_guard_prolong(DevMesh m, S *__restrict__ U, const int *__restrict__ leaves) {
  const int b = leaves[blockIdx.x];
  const int k = blockIdx.y;
  __shared__ int2 sl[27];
  if (threadIdx.x < 27) sl[threadIdx.x] = m.slots[b * 27 + threadIdx.x];
  __syncthreads();
  const int P = m.P, ng = m.ng, n = m.nxb, lev = m.level[b];
  const int sz = m.ndim == 3 ? slot_of(k, ng, ng + n) : 1;
  const int ox = m.origin[3 * b], oy = m.origin[3 * b + 1], oz = m.origin[3 * b + 2];
  S *Ub = U + (long long)b * m.bstride;
  const long long sP = P, sPP = (long long)P * P;
  for (int c = threadIdx.x; c < P * P; c += blockDim.x) {
    const int i = c % P, j = c / P;
    const int sx = slot_of(i, ng, ng + n), sy = slot_of(j, ng, ng + n);
    if (sx == 1 && sy == 1 && sz == 1) continue;
    const int2 s = sl[sx + 3 * sy + 9 * sz];
    if (s.x != SLOT_PROLONG) continue;
    int g[3];
    g[0] = apply_bc(ox + i - ng, m.ncell[lev][0], m.bc[0][0], m.bc[0][1]);
    g[1] = apply_bc(oy + j - ng, m.ncell[lev][1], m.bc[1][0], m.bc[1][1]);
    g[2] = m.ndim == 3 ? apply_bc(oz + k - ng, m.ncell[lev][2], m.bc[2][0], m.bc[2][1]) : 0;
    const int cb = s.y;
    const int cx = (g[0] >> 1) - m.origin[3 * cb] + ng;
    const int cy = (g[1] >> 1) - m.origin[3 * cb + 1] + ng;
    const int cz = m.ndim == 3 ? (g[2] >> 1) - m.origin[3 * cb + 2] + ng : 0;
    const S *C = U + (long long)cb * m.bstride + (cz * sPP + cy * sP + cx);
    S *Ud = Ub + ((long long)k * P + j) * P + i;
    const long long step[3] = {1, sP, sPP};
    for (int v = 0; v < 5; ++v) {
      const S *cv = C + v * m.vstride;
      const double uc = ld(cv);
      double val = uc;
      for (int d = 0; d < m.ndim; ++d) {
        const double um = ld(cv - step[d]), up = ld(cv + step[d]);
        const double sig = mc_lim(uc - um, up - uc);
        const double off = (g[d] & 1) ? 0.25 : -0.25;
        val = val + off * sig;
      }
      st(Ud + v * m.vstride, val);
    }
  }
}

template <typename S>
cudaError_t prim_to_cons_t(const DevMesh &m, const double *W, void *U, cudaStream_t s) {
  long long total = (long long)m.nb * m.vstride;
  int grid = (int)((total + 255) / 256);
  if (grid > 152 * 32) grid = 152 * 32;
  k_prim_to_cons<S><<<grid, 256, 0, s>>>(m, W, static_cast<S *>(U));
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_prim_to_cons(const DevMesh &m, const double *W, void *U, int prec,
                                cudaStream_t s) {
  return prec == 0 ? prim_to_cons_t<double>(m, W, U, s) : prim_to_cons_t<float>(m, W, U, s);
}

cudaError_t launch_restrict(const DevMesh &m, void *U, int prec, const int *parents, int n,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int ncell = m.nxb * m.nxb * (m.ndim == 3 ? m.nxb : 1);
  dim3 grid(n, (ncell + 255) / 256);
  if (prec == 0) k_restrict<double><<<grid, 256, 0, s>>>(m, static_cast<double *>(U), parents);
  else k_restrict<float><<<grid, 256, 0, s>>>(m, static_cast<float *>(U), parents);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_guard_copy(const DevMesh &m, void *U, int prec, const int *leaves, int n,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  dim3 grid(n, m.PZ);
  if (prec == 0) k_guard_copy<double><<<grid, 256, 0, s>>>(m, static_cast<double *>(U), leaves);
  else k_guard_copy<float><<<grid, 256, 0, s>>>(m, static_cast<float *>(U), leaves);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_guard_prolong(const DevMesh &m, void *U, int prec, const int *leaves, int n,
                                 cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  dim3 grid(n, m.PZ);
  if (prec == 0) k_guard_prolong<double><<<grid, 256, 0, s>>>(m, static_cast<double *>(U), leaves);
  else k_guard_prolong<float><<<grid, 256, 0, s>>>(m, static_cast<float *>(U), leaves);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fx
