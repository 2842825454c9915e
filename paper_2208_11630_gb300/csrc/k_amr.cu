// k_amr.cu -- fine-to-coarse flux correction at coarse-fine faces.
//
// Paper: Flash-X (arXiv 2208.11630), Section 2 -- after the block-by-block
// update the Grid resolves fine-coarse boundaries.  Concrete operator:
// Berger & Colella (1989) refluxing.  A coarse leaf cell next to a finer
// neighbour replaces its own face flux F_c by the pairwise mean F_bar of the
// 2^(d-1) fine face fluxes that cover the face:
//   upper face: U_c += dt/dx (F_c - F_bar);  lower face: U_c -= dt/dx (F_c - F_bar),
// applied per cell in the order x-, x+, y-, y+, z-, z+.
#include "grid_ops.cuh"

namespace fx {
namespace {

template <typename S>
__global__ void k_reflux(DevMesh m, S *__restrict__ Unew, const RefluxItem *__restrict__ items,
                         const double *__restrict__ dtp, const double *__restrict__ regs,
                         int *__restrict__ status, unsigned long long *__restrict__ smax,
                         int form, const int *__restrict__ live) {
  if (live != nullptr && *live <= 0) return;
  __shared__ RefluxItem it;
  if (threadIdx.x == 0) it = items[blockIdx.x];
  __syncthreads();
  ops::reflux_cells<S>(m, Unew, it, *dtp, regs, status, smax, form,
                       blockIdx.y * blockDim.x + threadIdx.x, gridDim.y * blockDim.x);
}

}  // namespace

cudaError_t launch_reflux(const DevMesh &m, void *Unew, int prec, const RefluxItem *items, int n,
                          const double *dt, const double *regs, int *status,
                          unsigned long long *smax, int form, cudaStream_t s, const int *live) {
  if (n <= 0) return cudaSuccess;
  const int ncell = m.nxb * m.nxb * (m.ndim == 3 ? m.nxb : 1);
  dim3 grid(n, (ncell + 255) / 256);
  if (prec == 0) k_reflux<double><<<grid, 256, 0, s>>>(m, static_cast<double *>(Unew), items, dt, regs, status, smax, form, live);
  else k_reflux<float><<<grid, 256, 0, s>>>(m, static_cast<float *>(Unew), items, dt, regs, status, smax, form, live);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fx
