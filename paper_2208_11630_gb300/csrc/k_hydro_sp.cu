// k_hydro_sp.cu -- the fused MUSCL-Hancock / HLLC update for the multispecies
// perfect gas: the tile body of hydro_tile.cuh instantiated for 1 to 4
// advected species (mass fractions reconstructed and predicted like a
// transverse velocity, per-cell mixture gamma, species fluxes upwinded by
// HLLC).  Separate from k_hydro.cu so that the single-gas kernels compile
// unchanged and in parallel.
//
// Paper: Flash-X (arXiv 2208.11630), Section 2.2 -- the perfect-gas EOS has a
// multispecies variant.
#include "hydro_sp.cuh"

namespace fx {
namespace {

template <int NS>
cudaError_t launch_ns(const DevMesh &m, const void *U, void *Unew, int prec, const int *leaves,
                      int n, const double *dt, double *regs, int *status,
                      unsigned long long *smax, const unsigned char *rmask, int form,
                      cudaStream_t s) {
  const int T = (m.nxb % 16 == 0) ? 16 : 8;
  if (prec == 0) {
    if (m.ndim == 3)
      return T == 16 ? launch_sp_t<3, 16, double, double, NS>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s)
                     : launch_sp_t<3, 8, double, double, NS>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s);
    return T == 16 ? launch_sp_t<2, 16, double, double, NS>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s)
                   : launch_sp_t<2, 8, double, double, NS>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s);
  }
  if (m.ndim == 3)
    return T == 16 ? launch_sp_t<3, 16, float, float, NS>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s)
                   : launch_sp_t<3, 8, float, float, NS>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s);
  return T == 16 ? launch_sp_t<2, 16, float, float, NS>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s)
                 : launch_sp_t<2, 8, float, float, NS>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s);
}

}  // namespace

cudaError_t launch_hydro_species(const DevMesh &m, const void *U, void *Unew, int prec,
                                 const int *leaves, int n, const double *dt, double *regs,
                                 int *status, unsigned long long *smax,
                                 const unsigned char *rmask, int form, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  switch (m.nspec) {
    case 1: return launch_ns<1>(m, U, Unew, prec, leaves, n, dt, regs, status, smax, rmask, form, s);
    case 2: return launch_ns<2>(m, U, Unew, prec, leaves, n, dt, regs, status, smax, rmask, form, s);
    case 3: return launch_ns<3>(m, U, Unew, prec, leaves, n, dt, regs, status, smax, rmask, form, s);
    case 4: return launch_ns<4>(m, U, Unew, prec, leaves, n, dt, regs, status, smax, rmask, form, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fx
