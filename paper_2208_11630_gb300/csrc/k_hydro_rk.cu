// k_hydro_rk.cu -- stage kernels of the SSP Runge-Kutta variants (SSP-RK2,
// SSP-RK3): the fused tile update of hydro_tile.cuh with plain MC-limited
// PLM face states (no Hancock half step), the stage blend
// Unew = wa Uavg + wb (U + dt L(U)) and stage-weighted flux registers.
//
// Paper: Flash-X (arXiv 2208.11630), Section 2.2 -- the Spark solver family
// integrates in time with second- or third-order strong-stability-preserving
// Runge-Kutta methods.
#include "hydro_tile.cuh"

namespace fx {
namespace {

template <int NDIM, int T, typename S, typename R>
__global__ void __launch_bounds__(T *T, (T == 16 ? (sizeof(R) == 4 ? 4 : 2) : 6))
k_hydro_rk(DevMesh m, const S *__restrict__ U, S *Unew, const int *__restrict__ leaves,
           int tiles, const double *__restrict__ dtp, double *__restrict__ regs,
           int *__restrict__ status, unsigned long long *__restrict__ smax_out,
           const unsigned char *__restrict__ rmask, int cfl_form, HydroStage st) {
  const int tpb = tiles * tiles;
  hydro_tile<NDIM, T, S, R, true>(m, U, Unew, leaves[blockIdx.x / tpb], blockIdx.x % tpb, tiles,
                                  *dtp, regs, status, smax_out, rmask, cfl_form, st);
}

template <int NDIM, int T, typename S, typename R>
cudaError_t launch_rk_t(const DevMesh &m, const void *U, void *Unew, const int *leaves, int n,
                        const double *dt, double *regs, int *status, unsigned long long *smax,
                        const unsigned char *rmask, int form, const HydroStage &st,
                        cudaStream_t s) {
  const int tiles = m.nxb / T;
  const size_t smem = (size_t)Smem<T>::total(NDIM == 3 ? 3 : 1) * sizeof(R);
  auto kern = k_hydro_rk<NDIM, T, S, R>;
  static std::atomic<unsigned long long> attr_devs{0};
  if (cudaError_t e = set_smem_once((const void *)kern, smem, attr_devs); e != cudaSuccess)
    return e;
  kern<<<n * tiles * tiles, T * T, smem, s>>>(m, static_cast<const S *>(U), static_cast<S *>(Unew),
                                              leaves, tiles, dt, regs, status, smax, rmask, form,
                                              st);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_hydro_rk(const DevMesh &m, const void *U, void *Unew, int prec,
                            const int *leaves, int n, const double *dt, double *regs, int *status,
                            unsigned long long *smax, const unsigned char *rmask, int form,
                            cudaStream_t s, const HydroStage &st) {
  if (n <= 0) return cudaSuccess;
  const int T = (m.nxb % 16 == 0) ? 16 : 8;
  if (prec == 0) {
    if (m.ndim == 3)
      return T == 16 ? launch_rk_t<3, 16, double, double>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, st, s)
                     : launch_rk_t<3, 8, double, double>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, st, s);
    return T == 16 ? launch_rk_t<2, 16, double, double>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, st, s)
                   : launch_rk_t<2, 8, double, double>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, st, s);
  }
  if (m.ndim == 3)
    return T == 16 ? launch_rk_t<3, 16, float, float>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, st, s)
                   : launch_rk_t<3, 8, float, float>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, st, s);
  return T == 16 ? launch_rk_t<2, 16, float, float>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, st, s)
                 : launch_rk_t<2, 8, float, float>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, st, s);
}

}  // namespace fx
