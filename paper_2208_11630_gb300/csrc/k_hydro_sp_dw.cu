// k_hydro_sp_dw.cu -- the multispecies update of FP64 block sets in
// double-word arithmetic (dword.cuh), for 1 to 4 species: the kernels of
// hydro_sp.cuh with compute type dw.  Selected per context with the option
// "f64_arith" = 1.
//
// Paper: Flash-X (arXiv 2208.11630), Section 2.2 -- the perfect-gas EOS has a
// multispecies variant; the arithmetic is this GPU's choice, not the paper's.
#include "hydro_sp.cuh"

namespace fx {
namespace {

template <int NS>
cudaError_t launch_ns_dw(const DevMesh &m, const void *U, void *Unew, const int *leaves, int n,
                         const double *dt, double *regs, int *status, unsigned long long *smax,
                         const unsigned char *rmask, int form, cudaStream_t s) {
  const int T = (m.nxb % 16 == 0) ? 16 : 8;
  if (m.ndim == 3)
    return T == 16 ? launch_sp_t<3, 16, double, dw, NS>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s)
                   : launch_sp_t<3, 8, double, dw, NS>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s);
  return T == 16 ? launch_sp_t<2, 16, double, dw, NS>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s)
                 : launch_sp_t<2, 8, double, dw, NS>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s);
}

}  // namespace

cudaError_t launch_hydro_species_dw(const DevMesh &m, const void *U, void *Unew,
                                    const int *leaves, int n, const double *dt, double *regs,
                                    int *status, unsigned long long *smax,
                                    const unsigned char *rmask, int form, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  switch (m.nspec) {
    case 1: return launch_ns_dw<1>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s);
    case 2: return launch_ns_dw<2>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s);
    case 3: return launch_ns_dw<3>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s);
    case 4: return launch_ns_dw<4>(m, U, Unew, leaves, n, dt, regs, status, smax, rmask, form, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fx
