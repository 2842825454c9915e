// k_amr.cu -- fine-to-coarse flux correction at coarse-fine faces.
//
// Paper: Flash-X (arXiv 2208.11630), Section 2 -- after the block-by-block
// update the Grid resolves fine-coarse boundaries.  Concrete operator:
// Berger & Colella (1989) refluxing.  A coarse leaf cell next to a finer
// neighbour replaces its own face flux F_c by the pairwise mean F_bar of the
// 2^(d-1) fine face fluxes that cover the face:
//   upper face: U_c += dt/dx (F_c - F_bar);  lower face: U_c -= dt/dx (F_c - F_bar),
// applied per cell in the order x-, x+, y-, y+, z-, z+.
#include "fx_internal.h"

namespace fx {
namespace {

template <typename S>
__global__ void k_reflux(DevMesh m, S *__restrict__ Unew, const RefluxItem *__restrict__ items,
                         const double *__restrict__ dtp, const double *__restrict__ regs,
                         int *__restrict__ status, unsigned long long *__restrict__ smax,
                         int form) {
  __shared__ RefluxItem it;
  if (threadIdx.x == 0) it = items[blockIdx.x];
  __syncthreads();
  const int c = it.block;
  const int n = m.nxb, ng = m.ng, P = m.P, nd = m.ndim;
  const int nz = nd == 3 ? n : 1;
  const int lev = m.level[c];
  const double dt = *dtp;
  const int nfc = m.nface_cells;
  const long long rstride = (long long)m.nfaces * 5 * nfc;
  const double *Fc = regs + (long long)m.regidx[c] * rstride;
  S *Uc = Unew + (long long)c * m.bstride;
  const int ncell = n * n * nz;
  for (int cell = blockIdx.y * blockDim.x + threadIdx.x; cell < ncell;
       cell += gridDim.y * blockDim.x) {
    const int ci[3] = {cell % n, (cell / n) % n, cell / (n * n)};
    // only cells on the block surface can be corrected
    bool surf = false;
    for (int d = 0; d < nd; ++d) surf |= (ci[d] == 0 || ci[d] == n - 1);
    if (!surf) continue;
    const long long o = ((long long)(nd == 3 ? ci[2] + ng : 0) * P + (ci[1] + ng)) * P + (ci[0] + ng);
    double u[5];
    bool touched = false;
    for (int d = 0; d < nd; ++d) {
      const int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;
      for (int s = 0; s < 2; ++s) {
        const int f = 2 * d + s;
        if (it.fine[f][0] < 0) continue;
        if (ci[d] != (s ? n - 1 : 0)) continue;
        if (!touched) {
          for (int v = 0; v < 5; ++v) u[v] = double(Uc[o + v * m.vstride]);
          touched = true;
        }
        const int t1 = ci[a1], t2 = nd == 3 ? ci[a2] : 0;
        const int h1 = 2 * t1 >= n, h2 = nd == 3 && 2 * t2 >= n;
        const double *Ff = regs + (long long)it.fine[f][h1 + 2 * h2] * rstride;
        const int ff = 2 * d + (s ? 0 : 1);
        const int u1 = 2 * t1 - h1 * n, u2 = nd == 3 ? 2 * t2 - h2 * n : 0;
        for (int v = 0; v < 5; ++v) {
          const double *fv = Ff + (long long)(ff * 5 + v) * nfc;
          double fbar;
          if (nd == 3) {
            fbar = ((fv[u2 * n + u1] + fv[u2 * n + u1 + 1]) +
                    (fv[(u2 + 1) * n + u1] + fv[(u2 + 1) * n + u1 + 1])) * 0.25;
          } else {
            fbar = (fv[u1] + fv[u1 + 1]) * 0.5;
          }
          const double fc = Fc[(long long)(f * 5 + v) * nfc + t2 * n + t1];
          const double corr = dt * (fc - fbar) * m.idx[lev][d];
          u[v] = s ? u[v] + corr : u[v] - corr;
        }
      }
    }
    if (touched) {
      S us[5];
      for (int v = 0; v < 5; ++v) { us[v] = S(u[v]); Uc[o + v * m.vstride] = us[v]; }
      if (!(u[0] > 0.0) || !(2.0 * u[4] * u[0] > u[1] * u[1] + u[2] * u[2] + u[3] * u[3]))
        atomicOr(status, 1);
      if (smax) {
        // CFL signal speed of the corrected cell, in the state's precision
        const S ir = S(1) / us[0];
        const S pr = S(m.gamma - 1.0) * (us[4] - S(0.5) * (us[1] * us[1] + us[2] * us[2] + us[3] * us[3]) * ir);
        const S cs = sqrt(S(m.gamma) * pr * ir);
        S sg = S(0);
        for (int d = 0; d < nd; ++d) {
          const S sd = (fabs(us[1 + d] * ir) + cs) * S(m.idx[lev][d]);
          sg = form == 0 ? sg + sd : fmax(sg, sd);
        }
        atomicMax(smax, (unsigned long long)__double_as_longlong(double(sg)));
      }
    }
  }
}

}  // namespace

cudaError_t launch_reflux(const DevMesh &m, void *Unew, int prec, const RefluxItem *items, int n,
                          const double *dt, const double *regs, int *status,
                          unsigned long long *smax, int form, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int ncell = m.nxb * m.nxb * (m.ndim == 3 ? m.nxb : 1);
  dim3 grid(n, (ncell + 255) / 256);
  if (prec == 0) k_reflux<double><<<grid, 256, 0, s>>>(m, static_cast<double *>(Unew), items, dt, regs, status, smax, form);
  else k_reflux<float><<<grid, 256, 0, s>>>(m, static_cast<float *>(Unew), items, dt, regs, status, smax, form);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fx
