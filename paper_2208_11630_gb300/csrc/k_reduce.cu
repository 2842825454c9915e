// k_reduce.cu -- CFL time step (max-reduction) and conserved totals.
//
// Paper: Flash-X (arXiv 2208.11630), Section 2 -- hyperbolic equations are
// advanced with explicit methods, whose stable step is set by the largest
// signal speed on the mesh.  dt = cfl / max_cells sum_d (|u_d| + c) / dx_d
// (or the maximum over d), c = sqrt(gamma p / rho) of the perfect gas
// (Section 2.2).  The maximum of non-negative doubles is taken on their bit
// patterns with atomicMax, which is exact and independent of order; the last
// CTA to finish writes dt and re-arms the two scratch words.
#include "eos.cuh"

namespace fx {
namespace {

template <typename S>
__global__ void k_dt(DevMesh m, const S *__restrict__ U, const int *__restrict__ leaves, int nleaves,
                     double cfl, int form, double *__restrict__ dt_out,
                     unsigned long long *__restrict__ scratch,
                     unsigned long long *__restrict__ max_out, int accumulate) {
  const int n = m.nxb, ng = m.ng, P = m.P, nd = m.ndim;
  const int nz = nd == 3 ? n : 1;
  const long long ncell = (long long)n * n * nz;
  const long long total = ncell * nleaves;
  // the signal speed is computed in the state's precision
  using C = S;
  C smax = C(0);
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < total;
       w += (long long)gridDim.x * blockDim.x) {
    const int b = leaves[w / ncell];
    const int c = (int)(w % ncell);
    const int i = c % n, j = (c / n) % n, k = c / (n * n);
    const S *u = U + (long long)b * m.bstride +
                 ((long long)(nd == 3 ? k + ng : 0) * P + (j + ng)) * P + (i + ng);
    const long long vs = m.vstride;
    C uc[FX_MAXVAR];
    for (int v = 0; v < m.nvar; ++v) uc[v] = u[v * vs];
    const SignalConsts<C> k0(m, m.level[b]);
    const C s = cell_signal<C>(m, uc, m.nspec, k0, form);
    smax = sig_max(smax, s);   // a NaN stays
  }
  // warp and CTA maximum on the bit patterns (non-negative doubles and NaN
  // order like their bits)
  unsigned long long bits = __double_as_longlong(double(smax));
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long other = __shfl_down_sync(0xffffffffu, bits, o);
    bits = other > bits ? other : bits;
  }
  __shared__ unsigned long long wmax[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) wmax[warp] = bits;
  __syncthreads();
  if (warp == 0) {
    bits = lane < (blockDim.x >> 5) ? wmax[lane] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long other = __shfl_down_sync(0xffffffffu, bits, o);
      bits = other > bits ? other : bits;
    }
    if (lane == 0) {
      atomicMax(&scratch[0], bits);
      __threadfence();
      const unsigned long long done = atomicAdd(&scratch[1], 1ull);
      if (done == gridDim.x - 1) {
        __threadfence();
        const unsigned long long mb = atomicAdd(&scratch[0], 0ull);
        if (max_out) {
          if (accumulate) atomicMax(max_out, mb);
          else *max_out = mb;
        } else {
          *dt_out = cfl / __longlong_as_double(mb);
        }
        scratch[0] = 0ull;
        scratch[1] = 0ull;
      }
    }
  }
}

// One CTA per leaf: per-variable sums over the interior in a fixed order
// (strided per thread, then a shared-memory tree), times the cell volume.
template <typename S>
__global__ void k_totals(DevMesh m, const S *__restrict__ U, const int *__restrict__ leaves,
                         double *__restrict__ out) {
  const int b = leaves[blockIdx.x];
  const int n = m.nxb, ng = m.ng, P = m.P, nd = m.ndim;
  const int nz = nd == 3 ? n : 1;
  const int ncell = n * n * nz;
  __shared__ double red[FX_MAXVAR][256];
  double acc[FX_MAXVAR] = {0};
  const int nv = m.nvar;
  const S *Ub = U + (long long)b * m.bstride;
  for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
    const int i = c % n, j = (c / n) % n, k = c / (n * n);
    const long long o = ((long long)(nd == 3 ? k + ng : 0) * P + (j + ng)) * P + (i + ng);
    for (int v = 0; v < nv; ++v) acc[v] += double(Ub[o + v * m.vstride]);
  }
  for (int v = 0; v < nv; ++v) red[v][threadIdx.x] = acc[v];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int v = 0; v < nv; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < nv) {
    const int lev = m.level[b];
    const double dV = m.dx[lev][0] * m.dx[lev][1] * (nd == 3 ? m.dx[lev][2] : 1.0);
    out[blockIdx.x * nv + threadIdx.x] = red[threadIdx.x][0] * dV;
  }
}

__global__ void k_dt_finalize(unsigned long long *__restrict__ smax, double cfl,
                              double *__restrict__ dt_out) {
  *dt_out = cfl / __longlong_as_double(*smax);
  *smax = 0ull;
}

}  // namespace

cudaError_t launch_dt_finalize(unsigned long long *smax, double cfl, double *dt_out,
                               cudaStream_t s) {
  k_dt_finalize<<<1, 1, 0, s>>>(smax, cfl, dt_out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_dt(const DevMesh &m, const void *U, int prec, const int *leaves, int n,
                      double cfl, int form, double *dt_out, unsigned long long *scratch,
                      cudaStream_t s) {
  if (n <= 0) return cudaErrorInvalidValue;
  const long long total = (long long)n * m.nxb * m.nxb * (m.ndim == 3 ? m.nxb : 1);
  long long grid = (total + 255) / 256;
  if (grid > 152 * 8) grid = 152 * 8;
  if (prec == 0)
    k_dt<double><<<(int)grid, 256, 0, s>>>(m, static_cast<const double *>(U), leaves, n, cfl, form,
                                           dt_out, scratch, nullptr, 0);
  else
    k_dt<float><<<(int)grid, 256, 0, s>>>(m, static_cast<const float *>(U), leaves, n, cfl, form,
                                          dt_out, scratch, nullptr, 0);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_signal_max(const DevMesh &m, const void *U, int prec, const int *leaves, int n,
                              int form, unsigned long long *max_out, unsigned long long *scratch,
                              cudaStream_t s, int accumulate) {
  if (n <= 0) return cudaErrorInvalidValue;
  const long long total = (long long)n * m.nxb * m.nxb * (m.ndim == 3 ? m.nxb : 1);
  long long grid = (total + 255) / 256;
  if (grid > 152 * 8) grid = 152 * 8;
  if (prec == 0)
    k_dt<double><<<(int)grid, 256, 0, s>>>(m, static_cast<const double *>(U), leaves, n, 1.0, form,
                                           nullptr, scratch, max_out, accumulate);
  else
    k_dt<float><<<(int)grid, 256, 0, s>>>(m, static_cast<const float *>(U), leaves, n, 1.0, form,
                                          nullptr, scratch, max_out, accumulate);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_totals(const DevMesh &m, const void *U, int prec, const int *leaves, int n,
                          double *out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (prec == 0) k_totals<double><<<n, 256, 0, s>>>(m, static_cast<const double *>(U), leaves, out);
  else k_totals<float><<<n, 256, 0, s>>>(m, static_cast<const float *>(U), leaves, out);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fx
