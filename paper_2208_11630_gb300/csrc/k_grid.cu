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
#include "grid_ops.cuh"

namespace fx {
namespace {

template <typename S>
__device__ __forceinline__ void st(S *p, double v) { *p = static_cast<S>(v); }

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
    double ig = igm1;
    if (m.nspec) {          // mass fractions follow; the cell's mixture gamma
      double X[FX_MAXSPEC], g, gm1;
      for (int k = 0; k < m.nspec; ++k) {
        X[k] = w[(5 + k) * per];
        st(u + (5 + k) * per, r * X[k]);
      }
      mix_gamma<double>(m, X, m.nspec, g, gm1);
      ig = 1.0 / gm1;
    }
    st(u, r);
    st(u + per, r * vx);
    st(u + 2 * per, r * vy);
    st(u + 3 * per, r * vz);
    st(u + 4 * per, p * ig + 0.5 * r * (vx * vx + vy * vy + vz * vz));
  }
}

// One CTA per (parent, chunk of interior cells).
template <typename S>
__global__ void k_restrict(DevMesh m, S *__restrict__ U, const int *__restrict__ parents,
                           const int *__restrict__ live) {
  if (live != nullptr && *live <= 0) return;
  ops::restrict_cells<S>(m, U, parents[blockIdx.x], blockIdx.y);
}

// One CTA per (leaf, padded z-plane): same-level guard copies up to `depth`.
template <typename S>
__global__ void k_guard_copy(DevMesh m, S *__restrict__ U, const int *__restrict__ leaves,
                             int depth, const int *__restrict__ live) {
  if (live != nullptr && *live <= 0) return;
  ops::guard_copy_plane<S>(m, U, leaves[blockIdx.x], blockIdx.y, depth);
}

// Interior cells of blocks [b0, b0 + nblk) between the padded block layout
// and a packed array [block][var][z][y][x] of interior cells (nvar variables) (packed index
// relative to block b0).  dir 0: packed -> padded; 1: padded -> packed.
template <typename S>
__global__ void k_pack(DevMesh m, S *__restrict__ U, S *__restrict__ Pk, int b0, int nblk,
                       int dir) {
  const int n = m.nxb, ng = m.ng, P = m.P;
  const int nz = m.ndim == 3 ? n : 1, gz = m.ndim == 3 ? ng : 0;
  const long long per_var = (long long)nz * n * n;
  const int nv = m.nvar;
  const long long total = (long long)nblk * nv * per_var;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total;
       c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % n), j = (int)((c / n) % n);
    const long long r = c / ((long long)n * n);
    const int k = (int)(r % nz);
    const long long bv = r / nz;
    const int v = (int)(bv % nv);
    const long long b = b0 + bv / nv;
    S *u = U + b * m.bstride + v * m.vstride + ((long long)(k + gz) * P + (j + ng)) * P + (i + ng);
    if (dir == 0) *u = Pk[c];
    else Pk[c] = *u;
  }
}

// One CTA per (leaf, slot covered by a coarser leaf): the prolonged guards
// of that slot within `depth`, in precision C.
template <typename S, typename C>
__global__ void k_guard_prolong_slots(DevMesh m, S *__restrict__ U, const int2 *__restrict__ items,
                                      int depth, const int *__restrict__ live) {
  if (live != nullptr && *live <= 0) return;
  const int2 it = items[blockIdx.x];
  ops::guard_prolong_slot<S, C>(m, U, it.x, it.y, depth, threadIdx.x, blockDim.x);
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

cudaError_t launch_pack(const DevMesh &m, void *U, int prec, void *packed, int b0, int nblk,
                        int dir, cudaStream_t s) {
  if (nblk <= 0) return cudaSuccess;
  const long long total =
      (long long)nblk * m.nvar * m.nxb * m.nxb * (m.ndim == 3 ? m.nxb : 1);
  long long grid = (total + 255) / 256;
  if (grid > 152 * 16) grid = 152 * 16;
  if (prec == 0)
    k_pack<double><<<(int)grid, 256, 0, s>>>(m, static_cast<double *>(U),
                                             static_cast<double *>(packed), b0, nblk, dir);
  else
    k_pack<float><<<(int)grid, 256, 0, s>>>(m, static_cast<float *>(U),
                                            static_cast<float *>(packed), b0, nblk, dir);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_restrict(const DevMesh &m, void *U, int prec, const int *parents, int n,
                            cudaStream_t s, const int *live) {
  if (n <= 0) return cudaSuccess;
  const int ncell = m.nxb * m.nxb * (m.ndim == 3 ? m.nxb : 1);
  dim3 grid(n, (ncell + 255) / 256);
  if (prec == 0) k_restrict<double><<<grid, 256, 0, s>>>(m, static_cast<double *>(U), parents, live);
  else k_restrict<float><<<grid, 256, 0, s>>>(m, static_cast<float *>(U), parents, live);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_guard_copy(const DevMesh &m, void *U, int prec, const int *leaves, int n,
                              int depth, cudaStream_t s, const int *live) {
  if (n <= 0) return cudaSuccess;
  dim3 grid(n, m.PZ);
  if (prec == 0) k_guard_copy<double><<<grid, 256, 0, s>>>(m, static_cast<double *>(U), leaves, depth, live);
  else k_guard_copy<float><<<grid, 256, 0, s>>>(m, static_cast<float *>(U), leaves, depth, live);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_guard_prolong_slots(const DevMesh &m, void *U, int prec, const int2 *items,
                                       int n, int depth, int state_precision_math,
                                       cudaStream_t s, const int *live) {
  if (n <= 0) return cudaSuccess;
  if (prec == 0)
    k_guard_prolong_slots<double, double><<<n, 128, 0, s>>>(m, static_cast<double *>(U), items, depth, live);
  else if (state_precision_math)
    k_guard_prolong_slots<float, float><<<n, 128, 0, s>>>(m, static_cast<float *>(U), items, depth, live);
  else
    k_guard_prolong_slots<float, double><<<n, 128, 0, s>>>(m, static_cast<float *>(U), items, depth, live);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fx
