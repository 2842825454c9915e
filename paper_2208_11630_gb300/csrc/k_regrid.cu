// k_regrid.cu -- device side of regridding (dynamic refinement of the
// octree): the per-leaf error indicator and the transfer of the state onto a
// new mesh.
//
// Paper: Flash-X (arXiv 2208.11630), Section 2 -- AMR with an octree of blocks
// (PARAMESH).  Indicator: Loehner's (1987) normalised second derivative,
// evaluated on density and pressure; transfer: kept blocks copy their
// interior, new children take the conservative MC-limited linear
// prolongation of their parent (the coarse-fine guard operator), with
// injection where that would not be positive.
#include "grid_ops.cuh"

namespace fx {
namespace {

// Indicator of one cell for one field, from a window q of that field around
// the cell at index c0, whose neighbours along axis d sit at offsets lo[d]
// (minus side) and hi[d] (plus side): sqrt(sum N^2 / sum D^2) over ordered
// direction pairs (a, b), each term scaled by 1/(dx_a dx_b); diagonal pairs
// use the second difference over its first-difference magnitudes plus the
// filter eps times |q+| + 2|q0| + |q-|; off-diagonal pairs the mixed
// difference / 4 over the two a-differences at b -+ 1 / 4 plus eps times the
// four corner magnitudes / 4.  Zero where the denominator vanishes.
// sc[a][b] = 1/(dx_a dx_b) at the block's level.
template <int NDIM>
__device__ __forceinline__ double loehner(const double *q, const int (&lo)[3], const int (&hi)[3],
                                          int c0, const double (*sc)[3], double eps) {
  double num = 0.0, den = 0.0;
#pragma unroll
  for (int a = 0; a < NDIM; ++a)
#pragma unroll
    for (int b = 0; b < NDIM; ++b) {
      double nu, de;
      if (a == b) {
        const double up = q[c0 + hi[a]];
        const double u0 = q[c0];
        const double um = q[c0 + lo[a]];
        nu = (up - u0) - (u0 - um);
        de = fabs(up - u0) + fabs(u0 - um) + eps * (fabs(up) + 2.0 * fabs(u0) + fabs(um));
      } else {
        const double upp = q[c0 + hi[a] + hi[b]];
        const double ump = q[c0 + lo[a] + hi[b]];
        const double upm = q[c0 + hi[a] + lo[b]];
        const double umm = q[c0 + lo[a] + lo[b]];
        nu = ((upp - ump) - (upm - umm)) * 0.25;
        de = (fabs(upp - ump) + fabs(upm - umm)) * 0.25 +
             eps * (fabs(upp) + fabs(ump) + fabs(upm) + fabs(umm)) * 0.25;
      }
      nu = nu * sc[a][b];
      de = de * sc[a][b];
      num = num + nu * nu;
      den = den + de * de;
    }
  return den > 0.0 ? sqrt(num / den) : 0.0;
}

// Shared memory of k_regrid_err: a ring of three (2D: one) window planes of
// density and pressure over the (n + 2)^2 radius-1 window of a plane.
__host__ __device__ inline int regrid_err_smem(int ndim, int n) {
  return (ndim == 3 ? 3 : 1) * 2 * (n + 2) * (n + 2) * (int)sizeof(double);
}

// One CTA per leaf, marching the interior along z with the ring above, so
// that each cell's pressure is formed once rather than at every stencil
// point.  Maximum over interior cells and over both fields, into
// err_bits[leaf index] (bit pattern of a non-negative double; zeroed by the
// caller).  Guards must be filled at depth 1.
template <int NDIM, typename S>
__global__ void k_regrid_err(DevMesh m, const S *__restrict__ U, const int *__restrict__ leaves,
                             double eps, unsigned long long *__restrict__ err_bits) {
  extern __shared__ double win[];
  const int b = leaves[blockIdx.x];
  const int n = m.nxb, ng = m.ng, P = m.P;
  constexpr int nd = NDIM;
  const int W = n + 2, WW = W * W;
  const int nz = nd == 3 ? n : 1;
  const long long vs = m.vstride;
  const S *Ub = U + (long long)b * m.bstride;
  __shared__ double sc[3][3];
  if (threadIdx.x < 9) {
    const int lev = m.level[b], a = threadIdx.x / 3, c = threadIdx.x % 3;
    sc[a][c] = 1.0 / (m.dx[lev][a] * m.dx[lev][c]);
  }
  // window plane kw: padded z = kw + ng - 1 in 3D (kw = 0 is the plane below
  // the interior), the only plane in 2D; ring slot kw % 3
  auto load = [&](int kw) {
    double *dst = win + (nd == 3 ? kw % 3 : 0) * 2 * WW;
    const int kp = nd == 3 ? kw + ng - 1 : 0;
    for (int c = threadIdx.x; c < WW; c += blockDim.x) {
      const int i = c % W, j = c / W;
      const long long o = ((long long)kp * P + (j + ng - 1)) * P + (i + ng - 1);
      double u[FX_MAXVAR];
      for (int v = 0; v < m.nvar; ++v) u[v] = double(Ub[o + v * vs]);
      dst[c] = u[0];
      dst[WW + c] = ops::cons_pressure(m, u);
    }
  };
  double e = 0.0;
  if (nd == 3) {
    load(0);
    load(1);
  }
  for (int k = 0; k < nz; ++k) {
    load(nd == 3 ? k + 2 : 0);
    __syncthreads();
    const int s0 = nd == 3 ? (k + 1) % 3 : 0;      // ring slot of the cells' plane
    const int lo[3] = {-1, -W, nd == 3 ? (k % 3 - s0) * 2 * WW : 0};
    const int hi[3] = {1, W, nd == 3 ? ((k + 2) % 3 - s0) * 2 * WW : 0};
    for (int c = threadIdx.x; c < n * n; c += blockDim.x) {
      const int c0 = s0 * 2 * WW + (c / n + 1) * W + (c % n + 1);
      const double er = loehner<NDIM>(win, lo, hi, c0, sc, eps);
      const double ep = loehner<NDIM>(win + WW, lo, hi, c0, sc, eps);
      e = fmax(e, fmax(er, ep));
    }
    __syncthreads();   // the next load overwrites the slot of plane k
  }
  unsigned long long bits = __double_as_longlong(e);
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_down_sync(0xffffffffu, bits, o);
    bits = other > bits ? other : bits;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(err_bits + blockIdx.x, bits);
}

// New block j, padded z-plane blockIdx.y of its interior: kind 0 copies the
// interior of old block src, kind 1 prolongs from old parent src (octant
// oct; its guards filled at depth 1), in FP64, rounding once to S -- per
// coarse cell, with the coarse value injected into all its children when
// the linear form would leave one of them non-positive in density or
// pressure.
template <typename S>
__global__ void k_regrid_transfer(DevMesh mo, const S *__restrict__ Uold, DevMesh mn,
                                  S *__restrict__ Unew, const int4 *__restrict__ map) {
  const int j = blockIdx.x;
  const int4 w = map[j];            // (kind, src, oct, -)
  const int n = mn.nxb, ng = mn.ng, P = mn.P;
  const int kz = mn.ndim == 3 ? ng : 0;
  const int k = blockIdx.y;         // interior plane
  const S *Us = Uold + (long long)w.y * mo.bstride;
  S *Ud = Unew + (long long)j * mn.bstride;
  const long long sP = P, sPP = (long long)P * P;
  const long long step[3] = {1, sP, sPP};
  for (int c = threadIdx.x; c < n * n; c += blockDim.x) {
    const int i = c % n, jj = c / n;
    const long long od = ((long long)(k + kz) * P + (jj + ng)) * P + (i + ng);
    if (w.x == 0) {
      for (int v = 0; v < mn.nvar; ++v) Ud[od + v * mn.vstride] = Us[od + v * mo.vstride];
      continue;
    }
    const int f[3] = {((w.z >> 0) & 1) * n + i, ((w.z >> 1) & 1) * n + jj,
                      mn.ndim == 3 ? ((w.z >> 2) & 1) * n + k : 0};
    const long long oc = ((long long)(mn.ndim == 3 ? f[2] / 2 + ng : 0) * P + (f[1] / 2 + ng)) * P +
                         (f[0] / 2 + ng);
    // conserved variables of the fine cell with parities q of coarse cell oc
    auto prolong = [&](const int (&q)[3], double (&u)[FX_MAXVAR]) {
      for (int v = 0; v < mn.nvar; ++v) {
        const S *cv = Us + v * mo.vstride + oc;
        const double uc = double(*cv);
        double val = uc;
        for (int d = 0; d < mn.ndim; ++d) {
          const double um = double(cv[-step[d]]), up = double(cv[step[d]]);
          const double sig = ops::mc_lim(uc - um, up - uc);
          val = val + (q[d] ? 0.25 : -0.25) * sig;
        }
        u[v] = val;
      }
    };
    // linear prolongation unless one of the coarse cell's 2^d children would
    // get a non-positive density or pressure: then all take the coarse value
    bool ok = true;
    for (int c = 0; c < (1 << mn.ndim) && ok; ++c) {
      const int q[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
      double u[FX_MAXVAR];
      prolong(q, u);
      if (!(u[0] > 0.0) || !(ops::cons_pressure(mn, u) > 0.0)) ok = false;
    }
    double u[FX_MAXVAR];
    if (ok) {
      const int q[3] = {f[0] & 1, f[1] & 1, f[2] & 1};
      prolong(q, u);
    } else {
      for (int v = 0; v < mn.nvar; ++v) u[v] = double(Us[v * mo.vstride + oc]);
    }
    for (int v = 0; v < mn.nvar; ++v) Ud[od + v * mn.vstride] = S(u[v]);
  }
}

}  // namespace

cudaError_t launch_regrid_err(const DevMesh &m, const void *U, int prec, const int *leaves, int n,
                              double eps, unsigned long long *err_bits, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int smem = regrid_err_smem(m.ndim, m.nxb);
  auto go = [&](auto kern, const auto *Ut) {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
    }
    kern<<<n, 256, smem, s>>>(m, Ut, leaves, eps, err_bits);
    return cudaSuccess;
  };
  const double *U64 = static_cast<const double *>(U);
  const float *U32 = static_cast<const float *>(U);
  cudaError_t e = m.ndim == 3 ? (prec == 0 ? go(k_regrid_err<3, double>, U64) : go(k_regrid_err<3, float>, U32))
                              : (prec == 0 ? go(k_regrid_err<2, double>, U64) : go(k_regrid_err<2, float>, U32));
  if (e != cudaSuccess) return e;
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_regrid_transfer(const DevMesh &mo, const void *Uold, const DevMesh &mn,
                                   void *Unew, int prec, const int4 *map, cudaStream_t s) {
  if (mn.nb <= 0) return cudaSuccess;
  dim3 grid(mn.nb, mn.ndim == 3 ? mn.nxb : 1);
  if (prec == 0)
    k_regrid_transfer<double><<<grid, 256, 0, s>>>(mo, static_cast<const double *>(Uold), mn,
                                                   static_cast<double *>(Unew), map);
  else
    k_regrid_transfer<float><<<grid, 256, 0, s>>>(mo, static_cast<const float *>(Uold), mn,
                                                  static_cast<float *>(Unew), map);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fx
