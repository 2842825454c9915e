// eos.cuh -- perfect-gas equation of state shared by the device code: one gas
// of ratio of specific heats gamma, or the multispecies perfect gas
// (Section 2.2 of Flash-X, arXiv 2208.11630, names a multispecies variant of
// the perfect-gas EOS) whose cell gamma follows the ideal-gas mixture rule
//   gamma - 1 = (sum_k X_k / A_k) / (sum_k X_k / (A_k (gamma_k - 1)))
// over the mass fractions X_k = (rho X_k) / rho.
#pragma once

#include "dword.cuh"
#include "fx_internal.h"

#include <type_traits>

namespace fx {

// gamma and gamma - 1 of a cell in precision R from its mass fractions
// X[0..ns) (ns = 0: the mesh's gamma).
template <typename R>
__device__ __forceinline__ void mix_gamma(const DevMesh &m, const R *X, int ns, R &g, R &gm1) {
  if (ns == 0) {
    g = R(m.gamma);
    gm1 = R(m.gamma - 1.0);
    return;
  }
  R q1 = R(0), q2 = R(0);
  for (int k = 0; k < ns; ++k) {
    q1 = q1 + X[k] * R(m.spa[k]);
    q2 = q2 + X[k] * R(m.spb[k]);
  }
  g = R(1) + q1 / q2;
  gm1 = g - R(1);
}

// Larger of two CFL signal speeds.  A signal speed is non-negative, or NaN
// for a cell with non-positive density or pressure; on the bit patterns the
// non-negative values order like the values and every NaN sorts above them,
// so a NaN wins and stays in a running maximum (the time step of such a state
// comes out NaN instead of a finite value that hides the bad cell).  An
// integer maximum, off the floating-point pipes.
__device__ __forceinline__ double sig_max(double a, double b) {
  const unsigned long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  return __longlong_as_double((long long)(ia > ib ? ia : ib));
}
__device__ __forceinline__ float sig_max(float a, float b) {
  const unsigned ia = __float_as_uint(a), ib = __float_as_uint(b);
  return __uint_as_float(ia > ib ? ia : ib);
}
__device__ __forceinline__ dword::dw sig_max(dword::dw a, dword::dw b) {
  if (a.hi != a.hi) return a;
  if (b.hi != b.hi) return b;
  return a < b ? b : a;
}

// Per-block constants of cell_signal in precision R, formed once outside
// the cell loops: the single gas's gamma and gamma - 1, and 1/dx per axis
// (FP32: converted once; FP64: see the specialisation below).
template <typename R>
struct SignalConsts {
  R g, gm1, idx[3];
  __device__ __forceinline__ SignalConsts(const DevMesh &m, int lev)
      : g(R(m.gamma)), gm1(R(m.gamma - 1.0)),
        idx{R(m.idx[lev][0]), R(m.idx[lev][1]), R(m.idx[lev][2])} {}
};

// FP64: the constants are read from the mesh where they are used (no
// conversion to make, no registers held across the cell loops).
template <>
struct SignalConsts<double> {
  int lev;
  __device__ __forceinline__ SignalConsts(const DevMesh &, int l) : lev(l) {}
};

// CFL signal speed of one cell from its conserved variables u[0..5+ns) in
// precision R: sum over directions (form 0) or maximum (form 1) of
// (|u_d| + c) / dx_d, c = sqrt(gamma p / rho).  The fused epilogue of the
// update, the flux correction and the standalone reduction all use it, so
// that they agree bit for bit.  FP32 takes 1/rho and the square root from
// the approximate hardware instructions (a few units in the last place; the
// FP32-bulk update's own rounding is larger), FP64 the correctly rounded ones.
//   NDIM > 0: the dimension is known at compile time (the direction loop unrolls).
template <typename R, int NDIM = 0>
__device__ __forceinline__ R cell_signal(const DevMesh &m, const R *u, int ns,
                                         const SignalConsts<R> &k0, int form) {
  R ir;
  if constexpr (std::is_same<R, float>::value) ir = __fdividef(1.0f, u[0]);
  else ir = R(1) / u[0];
  R g, gm1;
  if constexpr (std::is_same<R, double>::value) {
    g = m.gamma;
    gm1 = m.gamma - 1.0;
  } else {
    g = k0.g;
    gm1 = k0.gm1;
  }
  if (ns > 0) {
    R X[FX_MAXSPEC];
    for (int k = 0; k < ns; ++k) X[k] = u[5 + k] * ir;
    mix_gamma<R>(m, X, ns, g, gm1);
  }
  const R pr = gm1 * (u[4] - R(0.5) * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) * ir);
  R cs;
  if constexpr (std::is_same<R, float>::value) {
    asm("sqrt.approx.f32 %0, %1;" : "=f"(cs) : "f"(g * pr * ir));
  } else {
    cs = sqrt(g * pr * ir);
  }
  R sg = R(0);
  auto term = [&](int d) {
    R idx_d;
    if constexpr (std::is_same<R, double>::value) idx_d = m.idx[k0.lev][d];
    else idx_d = k0.idx[d];
    const R sd = (fabs(u[1 + d] * ir) + cs) * idx_d;
    sg = form == 0 ? sg + sd : sig_max(sg, sd);
  };
  if constexpr (NDIM > 0) {
#pragma unroll
    for (int d = 0; d < NDIM; ++d) term(d);
  } else {
    for (int d = 0; d < m.ndim; ++d) term(d);
  }
  return sg;
}

}  // namespace fx
