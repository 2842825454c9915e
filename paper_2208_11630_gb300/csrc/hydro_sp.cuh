// hydro_sp.cuh -- the multispecies tile kernel and its launch helper,
// shared by the FP64/FP32 instantiations (k_hydro_sp.cu) and the
// double-word ones (k_hydro_sp_dw.cu).
//
// Paper: Flash-X (arXiv 2208.11630), Section 2.2 -- the perfect-gas EOS has a
// multispecies variant.
#pragma once

#include "hydro_tile.cuh"

namespace fx {
namespace {

// More registers and shared memory per thread than the single-gas kernel:
// half the resident CTAs.
template <int NDIM, int T, typename S, typename R, int NS>
__global__ void __launch_bounds__(T *T, (T == 16 ? (sizeof(R) == 4 ? 2 : 1) : 4))
k_hydro_sp(DevMesh m, const S *__restrict__ U, S *Unew, const int *__restrict__ leaves,
           int tiles, const double *__restrict__ dtp, double *__restrict__ regs,
           int *__restrict__ status, unsigned long long *__restrict__ smax_out,
           const unsigned char *__restrict__ rmask, int cfl_form) {
  const int tpb = tiles * tiles;
  hydro_tile<NDIM, T, S, R, false, NS>(m, U, Unew, leaves[blockIdx.x / tpb], blockIdx.x % tpb,
                                       tiles, *dtp, regs, status, smax_out, rmask, cfl_form);
}

template <int NDIM, int T, typename S, typename R, int NS>
cudaError_t launch_sp_t(const DevMesh &m, const void *U, void *Unew, const int *leaves, int n,
                        const double *dt, double *regs, int *status, unsigned long long *smax,
                        const unsigned char *rmask, int form, cudaStream_t s) {
  const int tiles = m.nxb / T;
  const size_t smem = (size_t)Smem<T, NS>::total(NDIM == 3 ? 3 : 1) * sizeof(R);
  auto kern = k_hydro_sp<NDIM, T, S, R, NS>;
  static std::atomic<unsigned long long> attr_devs{0};
  if (cudaError_t e = set_smem_once((const void *)kern, smem, attr_devs); e != cudaSuccess)
    return e;
  kern<<<n * tiles * tiles, T * T, smem, s>>>(m, static_cast<const S *>(U), static_cast<S *>(Unew),
                                              leaves, tiles, dt, regs, status, smax, rmask, form);
  count_launch();
  return cudaGetLastError();
}

}  // namespace
}  // namespace fx
