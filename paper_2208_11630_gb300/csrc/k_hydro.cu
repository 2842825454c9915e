// k_hydro.cu -- fused unsplit MUSCL-Hancock / HLLC update of leaf blocks:
// the per-block-set kernel, the batched persistent kernel and their
// launchers.  The device body (scheme, layout, precision variants) is in
// hydro_tile.cuh.
//
// Paper: Flash-X (arXiv 2208.11630), Section 2.2 (unsplit predictor-corrector
// hydro) applied block by block (Section 2).
#include "hydro_batch.cuh"

namespace fx {
namespace {

template <int NDIM, int T, typename S, typename R>
__global__ void __launch_bounds__(T *T, (T == 16 ? (sizeof(R) == 4 ? 4 : 2) : 6))
k_hydro(DevMesh m, const S *__restrict__ U, S *Unew, const int *__restrict__ leaves,
        int tiles, const double *__restrict__ dtp, double *__restrict__ regs,
        int *__restrict__ status, unsigned long long *__restrict__ smax_out,
        const unsigned char *__restrict__ rmask, int cfl_form, const int *__restrict__ live) {
  if (live != nullptr && *live <= 0) return;   // a batched request with no steps left
  const int tpb = tiles * tiles;
  hydro_tile<NDIM, T, S, R>(m, U, Unew, leaves[blockIdx.x / tpb], blockIdx.x % tpb, tiles, *dtp,
                            regs, status, smax_out, rmask, cfl_form);
}

template <int NDIM, int T, typename S, typename R>
cudaError_t launch_t(const DevMesh &m, const void *U, void *Unew, const int *leaves, int n,
                     const double *dt, double *regs, int *status, unsigned long long *smax,
                     const unsigned char *rmask, int form, cudaStream_t s, const int *live) {
  const int tiles = m.nxb / T;
  const size_t smem = tile_smem_bytes<NDIM, T, R>();
  auto kern = k_hydro<NDIM, T, S, R>;
  static std::atomic<unsigned long long> attr_devs{0};
  if (cudaError_t e = set_smem_once((const void *)kern, smem, attr_devs); e != cudaSuccess)
    return e;
  kern<<<n * tiles * tiles, T * T, smem, s>>>(m, static_cast<const S *>(U), static_cast<S *>(Unew),
                                              leaves, tiles, dt, regs, status, smax, rmask, form,
                                              live);
  count_launch();
  return cudaGetLastError();
}

template <int NDIM, int T, typename S, typename R>
cudaError_t set_fit_t(int *fit) {
  const size_t smem = tile_smem_bytes<NDIM, T, R>();
  auto kern = k_hydro<NDIM, T, S, R>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(fit, kern, T * T, smem);
}

}  // namespace

cudaError_t hydro_set_fit(int ndim, int nxb, int cls, int *fit) {
  if (cls == 2) return hydro_set_fit_dw(ndim, nxb, fit);
  const bool t16 = nxb % 16 == 0;
  if (cls == 0) {
    if (ndim == 3) return t16 ? set_fit_t<3, 16, double, double>(fit) : set_fit_t<3, 8, double, double>(fit);
    return t16 ? set_fit_t<2, 16, double, double>(fit) : set_fit_t<2, 8, double, double>(fit);
  }
  if (ndim == 3) return t16 ? set_fit_t<3, 16, float, float>(fit) : set_fit_t<3, 8, float, float>(fit);
  return t16 ? set_fit_t<2, 16, float, float>(fit) : set_fit_t<2, 8, float, float>(fit);
}

cudaError_t hydro_batch_fit(int ndim, int tile, int prec, int *fit) {
  if (prec == 2) return hydro_batch_fit_dw(ndim, tile, fit);
  if (prec == 0) {
    if (ndim == 3) return tile == 16 ? fit_t<3, 16, double, double>(fit) : fit_t<3, 8, double, double>(fit);
    return tile == 16 ? fit_t<2, 16, double, double>(fit) : fit_t<2, 8, double, double>(fit);
  }
  if (ndim == 3) return tile == 16 ? fit_t<3, 16, float, float>(fit) : fit_t<3, 8, float, float>(fit);
  return tile == 16 ? fit_t<2, 16, float, float>(fit) : fit_t<2, 8, float, float>(fit);
}

cudaError_t launch_hydro_batch(int ndim, int tile, int prec, const BatchReq *reqs,
                               const int4 *items, int nitems, unsigned int *counter,
                               int ctas_per_sm, int nsm, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  if (prec == 2)
    return launch_hydro_batch_dw(ndim, tile, reqs, items, nitems, counter, ctas_per_sm, nsm, s);
  if (prec == 0) {
    if (ndim == 3)
      return tile == 16 ? launch_batch_t<3, 16, double, double>(reqs, items, nitems, counter, ctas_per_sm, nsm, s)
                        : launch_batch_t<3, 8, double, double>(reqs, items, nitems, counter, ctas_per_sm, nsm, s);
    return tile == 16 ? launch_batch_t<2, 16, double, double>(reqs, items, nitems, counter, ctas_per_sm, nsm, s)
                      : launch_batch_t<2, 8, double, double>(reqs, items, nitems, counter, ctas_per_sm, nsm, s);
  }
  if (ndim == 3)
    return tile == 16 ? launch_batch_t<3, 16, float, float>(reqs, items, nitems, counter, ctas_per_sm, nsm, s)
                      : launch_batch_t<3, 8, float, float>(reqs, items, nitems, counter, ctas_per_sm, nsm, s);
  return tile == 16 ? launch_batch_t<2, 16, float, float>(reqs, items, nitems, counter, ctas_per_sm, nsm, s)
                    : launch_batch_t<2, 8, float, float>(reqs, items, nitems, counter, ctas_per_sm, nsm, s);
}

cudaError_t launch_hydro(const DevMesh &m, const void *U, void *Unew, int prec, const int *leaves,
                         int n, const double *dt, double *regs, int *status,
                         unsigned long long *smax, const unsigned char *rmask, int form,
                         cudaStream_t s, const HydroStage &st) {
  if (n <= 0) return cudaSuccess;
  if (st.live && (m.nspec > 0 || !st.pred)) return cudaErrorInvalidValue;   // not batched
  if (m.nspec > 0) {   // multispecies gas (k_hydro_sp.cu): MUSCL-Hancock only
    if (!st.pred || st.Uavg || st.reg_add || st.reg_w != 1.0) return cudaErrorInvalidValue;
    if (st.dword) {
      if (prec != 0 || st.dword != 1) return cudaErrorInvalidValue;
      return launch_hydro_species_dw(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s);
    }
    return launch_hydro_species(m, U, Unew, prec, leaves, n, dt, regs, status, smax, rmask, form,
                                s);
  }
  if (!st.pred) {   // an SSP Runge-Kutta stage (k_hydro_rk.cu; double-word: k_hydro_dw.cu)
    if (st.dword) {
      if (prec != 0 || st.dword != 1) return cudaErrorInvalidValue;
      return launch_hydro_rk_dw(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s, st);
    }
    return launch_hydro_rk(m, U, Unew, prec, leaves, n, dt, regs, status, smax, rmask, form, s, st);
  }
  if (st.Uavg || st.reg_add || st.reg_w != 1.0) return cudaErrorInvalidValue;
  const int T = (m.nxb % 16 == 0) ? 16 : 8;
  if (st.dword == 2) {   // FP64 state, FP32 arithmetic (option f64_arith = 2)
    if (prec != 0) return cudaErrorInvalidValue;
    if (m.ndim == 3)
      return T == 16 ? launch_t<3, 16, double, float>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s, st.live)
                     : launch_t<3, 8, double, float>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s, st.live);
    return T == 16 ? launch_t<2, 16, double, float>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s, st.live)
                   : launch_t<2, 8, double, float>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s, st.live);
  }
  if (st.dword) {
    if (prec != 0) return cudaErrorInvalidValue;
    return launch_hydro_dw(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s, st.live);
  }
  if (prec == 0) {
    if (m.ndim == 3)
      return T == 16 ? launch_t<3, 16, double, double>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s, st.live)
                     : launch_t<3, 8, double, double>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s, st.live);
    return T == 16 ? launch_t<2, 16, double, double>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s, st.live)
                   : launch_t<2, 8, double, double>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s, st.live);
  }
  if (m.ndim == 3)
    return T == 16 ? launch_t<3, 16, float, float>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s, st.live)
                   : launch_t<3, 8, float, float>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s, st.live);
  return T == 16 ? launch_t<2, 16, float, float>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s, st.live)
                 : launch_t<2, 8, float, float>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s, st.live);
}

}  // namespace fx
