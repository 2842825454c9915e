// k_hydro_dw.cu -- the fused MUSCL-Hancock / HLLC update of FP64 block sets
// computed in double-word arithmetic (dword.cuh): the state is read and
// written in FP64, every operation of the tile body runs on pairs of FP32
// numbers (about 2^-47 relative precision) on the FP32 pipe instead of the
// FP64 one.  Selected per context with the option "f64_arith" = 1; the
// per-block-set kernel and the batched persistent one (compute class 2).
//
// Paper: Flash-X (arXiv 2208.11630), Section 2.2 (unsplit predictor-corrector
// hydro) applied block by block (Section 2); the arithmetic is this GPU's
// choice, not the paper's.
#include "hydro_batch.cuh"

namespace fx {
namespace {

template <int NDIM, int T>
__global__ void __launch_bounds__(T *T, (T == 16 ? 2 : 6))
k_hydro_dw(DevMesh m, const double *__restrict__ U, double *Unew, const int *__restrict__ leaves,
           int tiles, const double *__restrict__ dtp, double *__restrict__ regs,
           int *__restrict__ status, unsigned long long *__restrict__ smax_out,
           const unsigned char *__restrict__ rmask, int cfl_form, const int *__restrict__ live) {
  if (live != nullptr && *live <= 0) return;   // a batched request with no steps left
  const int tpb = tiles * tiles;
  hydro_tile<NDIM, T, double, dw>(m, U, Unew, leaves[blockIdx.x / tpb], blockIdx.x % tpb, tiles,
                                  *dtp, regs, status, smax_out, rmask, cfl_form);
}

template <int NDIM, int T>
cudaError_t launch_dw_t(const DevMesh &m, const void *U, void *Unew, const int *leaves, int n,
                        const double *dt, double *regs, int *status, unsigned long long *smax,
                        const unsigned char *rmask, int form, cudaStream_t s, const int *live) {
  const int tiles = m.nxb / T;
  const size_t smem = (size_t)Smem<T>::total(NDIM == 3 ? 3 : 1) * sizeof(dw);
  auto kern = k_hydro_dw<NDIM, T>;
  static std::atomic<unsigned long long> attr_devs{0};
  if (cudaError_t e = set_smem_once((const void *)kern, smem, attr_devs); e != cudaSuccess)
    return e;
  kern<<<n * tiles * tiles, T * T, smem, s>>>(m, static_cast<const double *>(U),
                                              static_cast<double *>(Unew), leaves, tiles, dt, regs,
                                              status, smax, rmask, form, live);
  count_launch();
  return cudaGetLastError();
}

template <int NDIM, int T>
cudaError_t set_fit_dw_t(int *fit) {
  const size_t smem = (size_t)Smem<T>::total(NDIM == 3 ? 3 : 1) * sizeof(dw);
  auto kern = k_hydro_dw<NDIM, T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(fit, kern, T * T, smem);
}

// SSP Runge-Kutta stage in double-word arithmetic (plain PLM face states,
// stage blend and weighted registers as in k_hydro_rk.cu).
template <int NDIM, int T>
__global__ void __launch_bounds__(T *T, (T == 16 ? 2 : 6))
k_hydro_rk_dw(DevMesh m, const double *__restrict__ U, double *Unew,
              const int *__restrict__ leaves, int tiles, const double *__restrict__ dtp,
              double *__restrict__ regs, int *__restrict__ status,
              unsigned long long *__restrict__ smax_out, const unsigned char *__restrict__ rmask,
              int cfl_form, HydroStage st) {
  const int tpb = tiles * tiles;
  hydro_tile<NDIM, T, double, dw, true>(m, U, Unew, leaves[blockIdx.x / tpb], blockIdx.x % tpb,
                                        tiles, *dtp, regs, status, smax_out, rmask, cfl_form, st);
}

template <int NDIM, int T>
cudaError_t launch_rk_dw_t(const DevMesh &m, const void *U, void *Unew, const int *leaves, int n,
                           const double *dt, double *regs, int *status, unsigned long long *smax,
                           const unsigned char *rmask, int form, const HydroStage &st,
                           cudaStream_t s) {
  const int tiles = m.nxb / T;
  const size_t smem = (size_t)Smem<T>::total(NDIM == 3 ? 3 : 1) * sizeof(dw);
  auto kern = k_hydro_rk_dw<NDIM, T>;
  static std::atomic<unsigned long long> attr_devs{0};
  if (cudaError_t e = set_smem_once((const void *)kern, smem, attr_devs); e != cudaSuccess)
    return e;
  kern<<<n * tiles * tiles, T * T, smem, s>>>(m, static_cast<const double *>(U),
                                              static_cast<double *>(Unew), leaves, tiles, dt, regs,
                                              status, smax, rmask, form, st);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_hydro_rk_dw(const DevMesh &m, const void *U, void *Unew, const int *leaves,
                               int n, const double *dt, double *regs, int *status,
                               unsigned long long *smax, const unsigned char *rmask, int form,
                               cudaStream_t s, const HydroStage &st) {
  if (n <= 0) return cudaSuccess;
  const int T = (m.nxb % 16 == 0) ? 16 : 8;
  if (m.ndim == 3)
    return T == 16 ? launch_rk_dw_t<3, 16>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, st, s)
                   : launch_rk_dw_t<3, 8>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, st, s);
  return T == 16 ? launch_rk_dw_t<2, 16>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, st, s)
                 : launch_rk_dw_t<2, 8>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, st, s);
}

cudaError_t launch_hydro_dw(const DevMesh &m, const void *U, void *Unew, const int *leaves, int n,
                            const double *dt, double *regs, int *status,
                            unsigned long long *smax, const unsigned char *rmask, int form,
                            cudaStream_t s, const int *live) {
  if (n <= 0) return cudaSuccess;
  const int T = (m.nxb % 16 == 0) ? 16 : 8;
  if (m.ndim == 3)
    return T == 16 ? launch_dw_t<3, 16>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s, live)
                   : launch_dw_t<3, 8>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s, live);
  return T == 16 ? launch_dw_t<2, 16>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s, live)
                 : launch_dw_t<2, 8>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s, live);
}

cudaError_t hydro_set_fit_dw(int ndim, int nxb, int *fit) {
  const bool t16 = nxb % 16 == 0;
  if (ndim == 3) return t16 ? set_fit_dw_t<3, 16>(fit) : set_fit_dw_t<3, 8>(fit);
  return t16 ? set_fit_dw_t<2, 16>(fit) : set_fit_dw_t<2, 8>(fit);
}

cudaError_t hydro_batch_fit_dw(int ndim, int tile, int *fit) {
  if (ndim == 3) return tile == 16 ? fit_t<3, 16, double, dw>(fit) : fit_t<3, 8, double, dw>(fit);
  return tile == 16 ? fit_t<2, 16, double, dw>(fit) : fit_t<2, 8, double, dw>(fit);
}

cudaError_t launch_hydro_batch_dw(int ndim, int tile, const BatchReq *reqs, const int4 *items,
                                  int nitems, unsigned int *counter, int ctas_per_sm, int nsm,
                                  cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  if (ndim == 3)
    return tile == 16 ? launch_batch_t<3, 16, double, dw>(reqs, items, nitems, counter, ctas_per_sm, nsm, s)
                      : launch_batch_t<3, 8, double, dw>(reqs, items, nitems, counter, ctas_per_sm, nsm, s);
  return tile == 16 ? launch_batch_t<2, 16, double, dw>(reqs, items, nitems, counter, ctas_per_sm, nsm, s)
                    : launch_batch_t<2, 8, double, dw>(reqs, items, nitems, counter, ctas_per_sm, nsm, s);
}

}  // namespace fx
