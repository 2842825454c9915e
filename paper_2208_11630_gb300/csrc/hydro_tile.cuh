// hydro_tile.cuh -- device body of the fused unsplit update of one T x T column
// tile of a leaf block, shared by the MUSCL-Hancock kernels (k_hydro.cu) and
// the SSP Runge-Kutta stage kernels (k_hydro_rk.cu).
//
// Paper: Flash-X (arXiv 2208.11630), Section 2.2 -- an unsplit compressible
// hydro solver of predictor-corrector type, applied one block at a time
// (Section 2).  Concrete scheme (textbook): primitive variables, MC-
// limited slopes (van Leer 1977), Hancock half-step predictor in primitive
// form (Toro ch. 14), HLLC flux with Davis speeds (Toro, Spruce & Speares
// 1994), conservative update summed over x, y, z.  A cell whose predicted face
// states are not all positive in density and pressure falls back to first
// order (zero slopes, no predictor).
//
// GB300 design.  One CTA owns a T x T column tile of one block and marches it
// along z.  Guard cells of same-level neighbours are read directly from the
// neighbour's interior while the tile is loaded (the guard copy is fused
// away); only guards covered by a coarser leaf come from the padded array.
// Shared memory holds a ring of primitive planes (radius-2 halo in x and y)
// and the x/y face states of the current plane; each face flux is computed
// once by one thread and written over the face state it consumed.  The thread
// owning column (i, j) keeps its z face states and z fluxes in registers.  Per
// plane, three barriers: load + primitives, predictor, fluxes, update -- or,
// with the four-plane ring of the FP32 3D single-gas instances, the next
// plane's load in the predictor phase.  The FP64 3D single-gas 16 x 16 tile
// balances the phases instead: the halo-predictor warps' z faces go through
// shared memory to warps with a face round fewer, the other threads solve
// their z face in the predictor phase, and the plane after next is loaded in
// the flux phase by the warps with two face rounds (ZDefer).
//
// Precision variants (state type S, compute type R): FP64 state and
// arithmetic; FP32-bulk -- FP32 state, FP32 reconstruction and Riemann
// solver, and an update that adds to U the exactly differenced fluxes
// (TwoSum) scaled by dt/dx with a single final rounding, which matches an
// FP64 accumulation up to a fraction of an FP32 ulp at a tiny fraction of the
// cost of FP64 arithmetic on this GPU; or FP64 state with double-word
// arithmetic (R = dw, dword.cuh), where one inlined Riemann solver serves all
// faces of a thread to keep the much larger code within instruction fetch.
#pragma once

#include "dword.cuh"
#include "eos.cuh"
#include "slot_map.cuh"

#include <type_traits>

namespace fx {
namespace {

// Half of van Leer's MC slope: 0 if a and b differ in sign or one is zero,
// else sign(a) min(|a|, |b|, |a+b|/4) -- exactly MC(a, b) / 2, since scaling by
// powers of two is exact.  The sign tests run on the integer pipe.
//
// FP64: the minimum of the three non-negative magnitudes is taken on their bit
// patterns (which order like the values), keeping it off the FP64 pipe.
__device__ __forceinline__ double mc_half(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  const bool same = ((ia ^ ib) >= 0) && (ia << 1) != 0 && (ib << 1) != 0;
  const long long ma = ia & 0x7fffffffffffffffll, mb = ib & 0x7fffffffffffffffll;
  const long long mq = __double_as_longlong(0.25 * fabs(a + b));
  long long m = ma < mb ? ma : mb;
  m = mq < m ? mq : m;
  // sign of a on the minimum magnitude
  const long long r = m | (ia & (long long)0x8000000000000000ull);
  return same ? __longlong_as_double(r) : 0.0;
}

// FP32: PTX min.xorsign.abs gives u = min(|a|, |b|) carrying the sign
// sign(a) xor sign(b) -- positive exactly when a and b agree in sign -- so
// clamping u to [0, |a+b|/4] and giving it the sign of a + b (the sign of a
// when they agree) is the same value as the FP64 form, in six instructions
// and without compares or selects (only the sign of a zero result can
// differ, which no later sum or product turns into a nonzero value).
__device__ __forceinline__ float mc_half(float a, float b) {
  float u;
  asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(u) : "f"(a), "f"(b));
  const float s = a + b;
  return copysignf(fmaxf(fminf(u, 0.25f * fabsf(s)), 0.0f), s);
}

// x > 0 (false for zero, negative and NaN; +inf counts as positive), tested on
// the bit pattern.
__device__ __forceinline__ bool positive(double x) {
  return (unsigned long long)__double_as_longlong(x) - 1ull < 0x7ff0000000000000ull;
}
// FP32: a plain compare is cheaper than the bit test; +inf is the only
// value where the two forms differ, and it counts as positive in both.
__device__ __forceinline__ bool positive(float x) { return x > 0.0f; }

// x >= 0 (true for -0; a NaN with a clear sign bit would count as >= 0, which
// only matters for states that are already invalid), on the bit pattern.
__device__ __forceinline__ bool ge0(double x) {
  const long long i = __double_as_longlong(x);
  return i >= 0 || (i << 1) == 0;
}
__device__ __forceinline__ bool ge0(float x) { return x >= 0.0f; }
__device__ __forceinline__ bool gt0(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool gt0(float x) { return x > 0.0f; }

__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }

// Double-word compute type (FP64 state): signs from the leading word, which
// carries the sign of every nonzero value.
__device__ __forceinline__ bool positive(dw x) { return x.hi > 0.0f; }
__device__ __forceinline__ bool ge0(dw x) { return x.hi >= 0.0f; }
__device__ __forceinline__ bool gt0(dw x) { return x.hi > 0.0f; }
__device__ __forceinline__ dw rsqrt_r(dw x) { return rsqrt(x); }
__device__ __forceinline__ dw mc_half(dw a, dw b) {
  const bool same = (a.hi > 0.0f && b.hi > 0.0f) || (a.hi < 0.0f && b.hi < 0.0f);
  const dw s = fabs(a + b);
  const dw q(0.25f * s.hi, 0.25f * s.lo);          // exact scaling
  const dw m = fmin(fmin(fabs(a), fabs(b)), q);
  return same ? (a.hi < 0.0f ? -m : m) : dw(0.0f, 0.0f);
}

// Flux-register write: MUSCL-Hancock stores F; an SSP-RK stage stores or
// adds st.reg_w F (stage-weighted sums).
template <bool RK, typename R>
__device__ __forceinline__ void put_reg(double &r, R f, const HydroStage &st) {
  const double v = double(f);
  if constexpr (RK) r = st.reg_add ? fma(st.reg_w, v, r) : st.reg_w * v;
  else r = v;
}

// Quotient and reciprocal: IEEE division in FP64; the fast (MUFU-based,
// ~2 ulp) forms in FP32, whose error is far below the FP32 storage rounding.
__device__ __forceinline__ double div_r(double a, double b) { return a / b; }
__device__ __forceinline__ dw div_r(dw a, dw b) { return a / b; }
__device__ __forceinline__ float div_r(float a, float b) { return __fdividef(a, b); }

// c * (a - b) with the difference a - b taken exactly (Knuth's TwoSum error
// term), so that nearly equal face fluxes lose no digits before scaling.
__device__ __forceinline__ float scaled_diff(float a, float b, float c) {
  const float nb = -b;
  const float s = a + nb;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (nb - bb);
  return fmaf(c, s, c * e);
}

// HLLC flux along direction D from primitive left/right states.  One
// reciprocal square root per side gives both the sound speed and 1/rho:
// r = (gamma p rho)^(-1/2), c = gamma p r, 1/rho = c r.  The star state of the
// upwind side K needs S* and 1/(S_K - S*): one FP64 reciprocal, or two FP32
// fast divisions.
//
// Multispecies (NS > 0): each side's gamma follows from its mass fractions
// WL[5..], WR[5..], and the species fluxes are the mass flux times the
// upwind side's mass fractions (they pass unchanged through the star region).
template <int D, typename R, int NS = 0>
__device__ __forceinline__ void hllc(const R (&WL)[5 + NS], const R (&WR)[5 + NS], R g, R igm1,
                                     const DevMesh &m, R (&F)[5 + NS]) {
  constexpr int N = 1 + D;
  const R rL = WL[0], uL = WL[N], pL = WL[4];
  const R rR = WR[0], uR = WR[N], pR = WR[4];
  R gL = g, gR = g, igL = igm1, igR = igm1;
  if constexpr (NS > 0) {
    R gm1L, gm1R;
    mix_gamma<R>(m, WL + 5, NS, gL, gm1L);
    mix_gamma<R>(m, WR + 5, NS, gR, gm1R);
    igL = div_r(R(1), gm1L);
    igR = div_r(R(1), gm1R);
  }
  (void)m;
  const R gpL = gL * pL, gpR = gR * pR;
  const R qL = rsqrt_r(gpL * rL), qR = rsqrt_r(gpR * rR);
  const R cL = gpL * qL, cR = gpR * qR;
  const R SL = fmin(uL - cL, uR - cR);
  const R SR = fmax(uL + cL, uR + cR);
  const R dL = SL - uL, dR = SR - uR;
  // S* = A / B.  FP64: its sign (A = 0 or A, B of equal sign <=> S* >= 0)
  // picks the side, and S* and 1/(S_K - S*) both come from one reciprocal
  // below; FP32: two fast divisions.
  const R A = pR - pL + rL * uL * dL - rR * uR * dR;
  const R B = rL * dL - rR * dR;
  constexpr bool kF64 = std::is_same<R, double>::value;
  constexpr bool kDW = std::is_same<R, dw>::value;
  R Sst = R(0);
  bool sst_ge0;
  if constexpr (kF64) {
    const long long ia = __double_as_longlong(A), ib = __double_as_longlong(B);
    sst_ge0 = (ia << 1) == 0 || (ia ^ ib) >= 0;
  } else if constexpr (kDW) {
    sst_ge0 = A.hi == 0.0f || ((A.hi < 0.0f) == (B.hi < 0.0f));
  } else {
    Sst = div_r(A, B);
    sst_ge0 = ge0(Sst);
  }
  // Branches: S_L >= 0 -> F_L; S* >= 0 -> F*_L; S_R > 0 -> F*_R; else F_R.
  const bool caseA = ge0(SL);
  const bool useL = caseA || sst_ge0;
  const bool star = !caseA && (useL || gt0(SR));
  R W[5 + NS];
#pragma unroll
  for (int q = 0; q < 5 + NS; ++q) W[q] = useL ? WL[q] : WR[q];
  const R SK = useL ? SL : SR;
  const R irK = useL ? cL * qL : cR * qR;
  const R igK = useL ? igL : igR;
  const R rK = W[0], uK = W[N], pK = W[4];
  const R ke = R(0.5) * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
  const R EK = pK * igK + rK * ke;           // total energy of side K
  const R eK = pK * igK * irK + ke;          // E_K / rho_K
  const R mK = rK * uK;
  F[0] = mK;
#pragma unroll
  for (int t = 0; t < 3; ++t) F[1 + t] = mK * W[1 + t];
  F[N] += pK;
  F[4] = uK * (EK + pK);
  if (star) {
    const R dK = SK - uK;
    R inv;
    if constexpr (kF64 || kDW) {
      // S_K - S* = Q / B with Q = S_K B - A:  r = 1/(B Q), S* = A Q r,
      // 1/(S_K - S*) = B B r
      const R Q = SK * B - A;
      const R r = R(1) / (B * Q);
      Sst = A * Q * r;
      inv = B * B * r;
    } else {
      inv = div_r(R(1), SK - Sst);
    }
    const R fac = rK * dK * inv;                       // rho*_K
    const R ds = Sst - uK;
    // F*_K = F_K + S_K (U*_K - U_K).  Mass and momenta: U*_K - U_K is
    // (rho*_K - rho_K)(1, u, v, w) plus rho*_K (S* - u_K) in the normal
    // momentum, since the star velocity keeps the tangential components and
    // takes S* as the normal one.
    const R fr = SK * (fac - rK);
    const R Ue = fac * (eK + ds * Sst) + ds * pK * inv;  // rho*_K e*_K
    F[0] = F[0] + fr;
#pragma unroll
    for (int t = 0; t < 3; ++t) F[1 + t] = F[1 + t] + fr * W[1 + t];
    F[N] = F[N] + (SK * fac) * ds;
    F[4] = F[4] + SK * (Ue - EK);
  }
#pragma unroll
  for (int k = 0; k < NS; ++k) F[5 + k] = F[0] * W[5 + k];
}

// Primitives (rho, u, v, w, p) and 1/rho of one cell; with NS species also
// the mass fractions (w[6..6+NS)) and the cell's gamma (w[6+NS]).
template <typename S, typename R, int NS = 0>
__device__ __forceinline__ void prim(const S *u, long long vs, R gm1, const DevMesh &m,
                                     R (&w)[6 + NS + (NS > 0)]) {
  const R r = R(u[0]), mx = R(u[vs]), my = R(u[2 * vs]), mz = R(u[3 * vs]), E = R(u[4 * vs]);
  const R ir = div_r(R(1), r);
  w[0] = r;
  w[1] = mx * ir;
  w[2] = my * ir;
  w[3] = mz * ir;
  R gmc = gm1;
  if constexpr (NS > 0) {
    R X[NS], gc;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      X[k] = R(u[(5 + k) * vs]) * ir;
      w[6 + k] = X[k];
    }
    mix_gamma<R>(m, X, NS, gc, gmc);
    w[6 + NS] = gc;
  }
  (void)m;
  // kinetic energy density from u.m (= |m|^2 / rho)
  w[4] = gmc * fma(R(-0.5), w[1] * mx + w[2] * my + w[3] * mz, E);
  w[5] = ir;
}

// Shared-memory map, in elements of R.
template <int T, int NS = 0>
struct Smem {
  static constexpr int W4 = T + 4;          // ring plane width (radius-2 halo)
  static constexpr int W2 = T + 2;          // face-state row width (radius-1)
  static constexpr int NV = 6 + NS + (NS > 0);  // rho, u, v, w, p, 1/rho (, X_k, gamma)
  static constexpr int NF = 5 + NS;         // face-state / flux components
  static constexpr int RING = NV * W4 * W4; // one primitive plane
  static constexpr int FX = NF * T * W2;    // x face states [v][j][i+1]
  static constexpr int FY = NF * W2 * T;    // y face states [v][j+1][i]
  static constexpr int total(int nplanes) { return nplanes * RING + 2 * FX + 2 * FY; }
};

// Ring component of primitive variable v (the ring stores 1/rho at 5).
__host__ __device__ constexpr int ring_comp(int v) { return v < 5 ? v : v + 1; }

// Primitive ring of an instance.  FP32 3D single-gas tiles keep four planes
// of five components (1/rho is recomputed where it is used, one fast
// reciprocal per predicted cell), so that the next plane's load shares the
// predictor phase instead of taking a phase of its own; the others keep three
// planes of six (FP64: the stored 1/rho saves a division per predicted cell).
template <int NDIM, typename R, bool RK, int NS>
struct RingCfg {
  static constexpr bool four = std::is_same<R, float>::value && NDIM == 3 && NS == 0 && !RK;
  static constexpr int planes = NDIM == 3 ? (four ? 4 : 3) : 1;
};
template <int NDIM, int T, typename R, bool RK, int NS>
__host__ __device__ constexpr int ring_plane_elems() {
  return (RingCfg<NDIM, R, RK, NS>::four ? 5 : Smem<T, NS>::NV) * Smem<T, NS>::W4 * Smem<T, NS>::W4;
}
// FP64 3D single-gas 16 x 16 tiles move the z faces of the halo-predictor
// threads out of the predictor phase: those threads leave their two z face
// states in shared memory, other threads solve these faces in the flux phase,
// and every other thread solves its own z face right after its predictor, so
// that neither phase waits at its barrier for warps with twice the work.
template <int NDIM, int T, typename R, bool RK, int NS>
struct ZDefer {
  static constexpr bool on = std::is_same<R, double>::value && NDIM == 3 && T == 16 && !RK &&
                             NS == 0;
  static constexpr int elems = on ? 2 * (5 + NS) * 4 * T : 0;   // left and right states
};
// Dynamic shared memory of one tile instance, in bytes.
template <int NDIM, int T, typename R, bool RK = false, int NS = 0>
__host__ __device__ constexpr size_t tile_smem_bytes() {
  return (size_t)(RingCfg<NDIM, R, RK, NS>::planes * ring_plane_elems<NDIM, T, R, RK, NS>() +
                  2 * Smem<T, NS>::FX + 2 * Smem<T, NS>::FY + ZDefer<NDIM, T, R, RK, NS>::elems) *
         sizeof(R);
}

// Slopes, Hancock predictor and face states of the cell at tile-local (i, j)
// of the plane in ring slot s0 (neighbour planes in sm, sp).  Works with half
// slopes h = dW/2 throughout: the predictor is linear in the slopes, so
// A(W) h (2/dx) is exactly A(W) dW / dx, and the face states are W* -+ h.
// predict_wh forms the cell's primitives W0, half slopes h and half-step
// state Wh; predict and predict_face form the face states from them.
template <int NDIM, int T, typename R, bool PRED, int NS, bool RING4>
__device__ __forceinline__ void predict_wh(const R *__restrict__ ring, int sm, int s0, int sp,
                                           int i, int j, R hdt, const R (&idx2)[3], R g,
                                           R (&W0)[5 + NS], R (&h)[3][5 + NS], R (&Wh)[5 + NS]) {
  using SM = Smem<T, NS>;
  constexpr int NF = 5 + NS;
  constexpr int PL = SM::W4 * SM::W4;
  constexpr int RS = RING4 ? 5 * PL : SM::RING;   // one ring plane
  const int c = (j + 2) * SM::W4 + (i + 2);
  const R *p0 = ring + s0 * RS;
#pragma unroll
  for (int v = 0; v < NF; ++v) W0[v] = p0[ring_comp(v) * PL + c];
  const R ir = RING4 ? div_r(R(1), W0[0]) : p0[5 * PL + c];
  // the cell's gamma: the mesh's, or its mixture gamma (species)
  const R gc = NS > 0 ? p0[(6 + NS) * PL + c] : g;
#pragma unroll
  for (int v = 0; v < NF; ++v) {
    const R *q = p0 + ring_comp(v) * PL + c;
    h[0][v] = mc_half(W0[v] - q[-1], q[1] - W0[v]);
    h[1][v] = mc_half(W0[v] - q[-SM::W4], q[SM::W4] - W0[v]);
    if (NDIM == 3) {
      const R wm = ring[sm * RS + ring_comp(v) * PL + c];
      const R wp = ring[sp * RS + ring_comp(v) * PL + c];
      h[2][v] = mc_half(W0[v] - wm, wp - W0[v]);
    } else {
      h[2][v] = R(0);
    }
  }
  if constexpr (PRED) {
    // primitive quasi-linear form: sum_d A_d(W) dW_d / dx_d
    R acc[NF];
#pragma unroll
    for (int v = 0; v < NF; ++v) acc[v] = R(0);
    const R r = W0[0], gp = gc * W0[4];
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
      const int n = 1 + d;
      const R un = W0[n];
      R a[NF];
      a[0] = un * h[d][0] + r * h[d][n];
#pragma unroll
      for (int t = 0; t < 3; ++t) a[1 + t] = un * h[d][1 + t];
      a[n] = a[n] + h[d][4] * ir;
      a[4] = gp * h[d][n] + un * h[d][4];
#pragma unroll
      for (int k = 0; k < NS; ++k) a[5 + k] = un * h[d][5 + k];   // advected X_k
#pragma unroll
      for (int v = 0; v < NF; ++v) acc[v] = acc[v] + a[v] * idx2[d];
    }
#pragma unroll
    for (int v = 0; v < NF; ++v) Wh[v] = W0[v] - hdt * acc[v];
  } else {
    // plain PLM face states: no half step
#pragma unroll
    for (int v = 0; v < NF; ++v) Wh[v] = W0[v];
  }
}

// Returns the lower/upper face states per direction in fm/fp (the cell's
// primitives in all of them when one has non-positive density or pressure).
template <int NDIM, int T, typename R, bool PRED = true, int NS = 0, bool RING4 = false>
__device__ __forceinline__ void predict(const R *__restrict__ ring, int sm, int s0, int sp, int i,
                                        int j, R hdt, const R (&idx2)[3], R g,
                                        R (&fm)[3][5 + NS], R (&fp)[3][5 + NS]) {
  constexpr int NF = 5 + NS;
  R W0[NF], h[3][NF], Wh[NF];
  predict_wh<NDIM, T, R, PRED, NS, RING4>(ring, sm, s0, sp, i, j, hdt, idx2, g, W0, h, Wh);
  bool ok = true;
#pragma unroll
  for (int d = 0; d < NDIM; ++d) {
#pragma unroll
    for (int v = 0; v < NF; ++v) {
      fm[d][v] = Wh[v] - h[d][v];
      fp[d][v] = Wh[v] + h[d][v];
    }
    ok = ok && positive(fm[d][0]) && positive(fm[d][4]) && positive(fp[d][0]) &&
         positive(fp[d][4]);
  }
  if (!ok) {
#pragma unroll
    for (int d = 0; d < NDIM; ++d)
#pragma unroll
      for (int v = 0; v < NF; ++v) { fm[d][v] = W0[v]; fp[d][v] = W0[v]; }
  }
}

// A cell of the tile's radius-1 halo ring feeds one face of the tile: only
// that face state -- direction dir (0 or 1), the upper one (Wh + h) if plus,
// else the lower -- with the positivity fallback decided on the density and
// pressure of all its face states, as in predict (the same values).
template <int NDIM, int T, typename R, bool PRED = true, int NS = 0, bool RING4 = false>
__device__ __forceinline__ void predict_face(const R *__restrict__ ring, int sm, int s0, int sp,
                                             int i, int j, R hdt, const R (&idx2)[3], R g,
                                             int dir, bool plus, R (&fs)[5 + NS]) {
  constexpr int NF = 5 + NS;
  R W0[NF], h[3][NF], Wh[NF];
  predict_wh<NDIM, T, R, PRED, NS, RING4>(ring, sm, s0, sp, i, j, hdt, idx2, g, W0, h, Wh);
  bool ok = true;
#pragma unroll
  for (int d = 0; d < NDIM; ++d)
    ok = ok && positive(Wh[0] - h[d][0]) && positive(Wh[4] - h[d][4]) &&
         positive(Wh[0] + h[d][0]) && positive(Wh[4] + h[d][4]);
#pragma unroll
  for (int v = 0; v < NF; ++v) {
    const R hv = dir == 0 ? h[0][v] : h[1][v];
    fs[v] = ok ? (plus ? Wh[v] + hv : Wh[v] - hv) : W0[v];
  }
}

// One T x T column tile of leaf block b, marched along z.  Called by the
// per-block-set kernel (one CTA per tile) and by the batched persistent
// kernel (each CTA loops over tiles of many block sets).
//   RK false  MUSCL-Hancock: Hancock half step, registers store F (st unused)
//   RK true   an SSP Runge-Kutta stage: plain PLM face states; st.Uavg null,
//             or Unew = st.wa Uavg + st.wb (U + dt L(U)) (Uavg may be Unew
//             itself: each cell is read before it is written by the same
//             thread, so neither pointer is declared restrict); registers
//             store or (st.reg_add) add st.reg_w F
template <int NDIM, int T, typename S, typename R, bool RK = false, int NS = 0>
__device__ __forceinline__ void hydro_tile(const DevMesh &m, const S *__restrict__ U,
                                           S *Unew, int b, int tile, int tiles,
                                           double dt, double *__restrict__ regs,
                                           int *__restrict__ status,
                                           unsigned long long *__restrict__ smax_out,
                                           const unsigned char *__restrict__ rmask,
                                           int cfl_form, const HydroStage &st = HydroStage()) {
  const S *Uavg = RK ? static_cast<const S *>(st.Uavg) : nullptr;
  using SM = Smem<T, NS>;
  constexpr int NF = 5 + NS;         // conserved variables, face-state components
  constexpr int NT = T * T;
  using RC = RingCfg<NDIM, R, RK, NS>;
  constexpr bool R4 = RC::four;
  constexpr int NPL = RC::planes;
  constexpr int RS = ring_plane_elems<NDIM, T, R, RK, NS>();   // one ring plane
  constexpr int NVR = R4 ? 5 : SM::NV;                          // components stored
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *ring = reinterpret_cast<R *>(smem_raw);
  R *fxm = ring + NPL * RS;         // x lower-face states, then x fluxes
  R *fxp = fxm + SM::FX;
  R *fym = fxp + SM::FX;            // y lower-face states, then y fluxes
  R *fyp = fym + SM::FY;
  // deferred z faces: [left state | right state, then flux][component][4T]
  constexpr bool kZD = ZDefer<NDIM, T, R, RK, NS>::on;
  constexpr int kZT = 4 * T;                 // halo-predictor threads
  constexpr int kZ0 = 4 * T + 32;            // their z faces: threads after the extra face round
  static_assert(!kZD || (2 * (T + 1) * T) % NT == 32,
                "the x/y face loop leaves one extra round of 32 faces on threads [4T, 4T + 32)");
  R *zbuf = fyp + SM::FY;
  (void)zbuf;

  // FP32 compute: the warp-level roles (the halo predictor on the first 4T
  // threads, the last partial rounds of the face and plane-load loops on
  // others) rotate by whole warps with the CTA index, so that the CTAs sharing
  // an SM -- whose warp w all run on the same SM sub-partition -- spread the
  // extra work over the four sub-partitions (measured 2 % faster at 256^3; the
  // FP64-pipe-bound update measured 1 % slower with it and keeps the plain
  // order).
  const int tid = std::is_same<R, float>::value
                      ? (int)((threadIdx.x + 32u * blockIdx.x) % (unsigned)NT)
                      : (int)threadIdx.x;
  __syncthreads();   // the previous tile of this CTA is done with shared memory
  const int x0 = (tile % tiles) * T, y0 = (tile / tiles) * T;
  const int n = m.nxb, ng = m.ng, P = m.P;
  const int lev = m.level[b];
  const long long vs = m.vstride;
  // FP32 compute: the per-tile constants are formed once in FP64 by one
  // thread and read from shared memory where used, so that no FP64
  // arithmetic or conversion is rematerialised inside the cell loops
  constexpr bool kF32c = std::is_same<R, float>::value;
  __shared__ float kcf[13];
  if (kF32c && tid == 32 % NT) {
    kcf[0] = float(dt * m.idx[lev][0]);
    kcf[1] = float(dt * m.idx[lev][1]);
    kcf[2] = float(dt * m.idx[lev][2]);
    kcf[3] = float(0.5 * dt);
    kcf[4] = float(2.0 * m.idx[lev][0]);
    kcf[5] = float(2.0 * m.idx[lev][1]);
    kcf[6] = float(2.0 * m.idx[lev][2]);
    kcf[7] = float(1.0 / (m.gamma - 1.0));
    kcf[8] = float(m.gamma);
    kcf[9] = float(m.gamma - 1.0);
    kcf[10] = float(m.idx[lev][0]);
    kcf[11] = float(m.idx[lev][1]);
    kcf[12] = float(m.idx[lev][2]);
  }
  if (kF32c) __syncthreads();
  auto kc = [&](int i, double v) -> R {
    if constexpr (kF32c) return R(kcf[i]);
    else return R(v);
  };
  const R g = kc(8, m.gamma), gm1 = kc(9, m.gamma - 1.0), igm1 = kc(7, 1.0 / (m.gamma - 1.0));
  const R hdt = kc(3, 0.5 * dt);
  R idx2[3];
  idx2[0] = kc(4, 2.0 * m.idx[lev][0]);
  idx2[1] = kc(5, 2.0 * m.idx[lev][1]);
  idx2[2] = kc(6, 2.0 * m.idx[lev][2]);
  const double didx = m.idx[lev][0], didy = m.idx[lev][1], didz = m.idx[lev][2];
  // the same in the compute type (FP64 and double-word updates)
  const R rdx = R(didx), rdy = R(didy), rdz = R(didz), rdt = R(dt);
  const S *Ub = U + (long long)b * m.bstride;
  S *Unb = Unew + (long long)b * m.bstride;   // may alias Uavg (see above)
  const int ti = tid % T, tj = tid / T;
  const int zoff = NDIM == 3 ? ng : 0;
  const int ridx = m.regidx[b];
  double *reg = ridx >= 0 ? regs + (long long)ridx * m.nfaces * NF * m.nface_cells : nullptr;
  const int nfc = m.nface_cells;

  // Guard sources of this block: a same-level slot is read straight from the
  // neighbour's interior (the value the guard copy would have written); a
  // slot covered by a coarser leaf is read from this block's own guards,
  // which the prolongation pass filled.
  // Work of one plane beyond one item per thread, spread over disjoint warps
  // so that no warp carries two extras into a barrier: the halo predictor
  // (4T cells) runs on threads [0, 4T), the last partial round of x/y faces
  // on the threads right after them, the last partial round of the plane
  // load on the highest threads.
  constexpr int kLoadTail = (SM::W4 * SM::W4) % NT;
  constexpr int kFaceShift = NT - 4 * T;
  __shared__ long long src_off[27];
  __shared__ int4 src_map[27];
  if (tid < 27) guard_source(m, b, tid, src_off[tid], src_map[tid]);
  __syncthreads();
  // plane p into ring slot `slot`, cells [first, ...) strided by `stride`
  auto load_cells = [&](int p, int slot, int first, int stride) {
    R *dst = ring + slot * RS;
    const int zpad = p + zoff;
    const int sz = NDIM == 3 ? (zpad < ng ? 0 : (zpad >= ng + n ? 2 : 1)) : 1;
    for (int c = first; c < SM::W4 * SM::W4; c += stride) {
      const int ii = c % SM::W4, jj = c / SM::W4;
      const int gx = x0 + ii - 2 + ng, gy = y0 + jj - 2 + ng;
      const int sx = gx < ng ? 0 : (gx >= ng + n ? 2 : 1);
      const int sy = gy < ng ? 0 : (gy >= ng + n ? 2 : 1);
      const int q = sx + 3 * sy + 9 * sz;
      const int4 mq = src_map[q];
      const S *src = U + (src_off[q] + (gx * mq.x + gy * mq.y + zpad * mq.z));
      const unsigned flip = (unsigned)mq.w;   // velocity components mirrored at a wall
      R w[SM::NV];
      prim<S, R, NS>(src, vs, gm1, m, w);
      if (flip) {
#pragma unroll
        for (int d = 0; d < 3; ++d)
          if ((flip >> d) & 1u) w[1 + d] = -w[1 + d];
      }
#pragma unroll
      for (int v = 0; v < NVR; ++v) dst[v * SM::W4 * SM::W4 + c] = w[v];
    }
  };
  auto load_plane = [&](int p, int slot) { load_cells(p, slot, (tid + kLoadTail) % NT, NT); };
  // FP64 tiles with the z-face move (ZDefer::on) load plane p + 2 in the flux
  // phase of plane p, into the ring slot plane p - 1 left when the predictor
  // phase ended, on the threads with two rounds of faces there: those of the
  // halo predictor and those after the deferred z faces.  The loop top then
  // loads nothing.
  constexpr bool kLF = ZDefer<NDIM, T, R, RK, NS>::on;
  constexpr int kLoaders = kZT + (NT - kZ0 - kZT);
  const bool loader = tid < kZT || tid >= kZ0 + kZT;
  const int lrank = tid < kZT ? tid : tid - (kZ0 + kZT) + kZT;
  (void)kLoaders; (void)loader; (void)lrank;
  auto slot_of = [&](int p) { return NDIM == 3 ? (R4 ? (p & 3) : ((p % 3) + 3) % 3) : 0; };

  // register state of the thread's column: pending update of the cell below
  // (x+y part of its flux divergence, flux through its lower z face)
  constexpr bool kF32 = std::is_same<R, float>::value;
  R txy[NF], fzl[NF];
  R zprev[NF];
#pragma unroll
  for (int v = 0; v < NF; ++v) { txy[v] = R(0); fzl[v] = R(0); zprev[v] = R(0); }
  // FP32 path: dt/dx per direction; FP64 path: 1/dx and dt separately
  float cx, cy, cz;
  if constexpr (kF32c) {
    cx = kcf[0]; cy = kcf[1]; cz = kcf[2];
  } else {
    cx = float(dt * m.idx[lev][0]); cy = float(dt * m.idx[lev][1]); cz = float(dt * m.idx[lev][2]);
  }
  (void)cx; (void)cy; (void)cz;
  // Signal speed of the new state, for the next step's CFL dt (same formula
  // and precision as the standalone reduction).  Cells that the flux
  // correction will still change (on a face in rmask) are left to it.
  const unsigned fmask = rmask ? rmask[b] : 0u;
  R smax_t = R(0);
  SignalConsts<R> sconst(m, lev);
  if constexpr (kF32c) {
    sconst.g = kcf[8];
    sconst.gm1 = kcf[9];
    sconst.idx[0] = kcf[10];
    sconst.idx[1] = kcf[11];
    sconst.idx[2] = kcf[12];
  }
  // FP64 state with FP32 arithmetic (S = double, R = float): the flux
  // divergence, formed in FP32, is added to the FP64 state in FP64, and the
  // new state's signal speed is taken in FP64 from the stored values -- the
  // computation of the standalone reduction of an FP64 block set, so that
  // the fused dt equals a fresh one
  constexpr bool kAbl = std::is_same<S, double>::value && std::is_same<R, float>::value;
  [[maybe_unused]] const SignalConsts<double> sconst_d(m, lev);
  [[maybe_unused]] double smax_d = 0.0;
  auto masked = [&](int ci, int cj, int ck) {
    if (fmask) {
      const int cc[3] = {ci, cj, ck};
      for (int d = 0; d < NDIM; ++d) {
        if (((fmask >> (2 * d)) & 1u) && cc[d] == 0) return true;
        if (((fmask >> (2 * d + 1)) & 1u) && cc[d] == n - 1) return true;
      }
    }
    return false;
  };
  auto signal = [&](const R (&u)[NF], int ci, int cj, int ck) {
    if (masked(ci, cj, ck)) return;
    // FP32: the direction loop unrolled; FP64 (at its register limit) keeps
    // it rolled, which measured faster there
    constexpr int kSigDim = std::is_same<R, float>::value ? NDIM : 0;
    const R sg = cell_signal<R, kSigDim>(m, u, NS, sconst, cfl_form);
    smax_t = sig_max(smax_t, sg);   // a NaN stays
  };
  [[maybe_unused]] auto signal_d = [&](const double (&u)[NF], int ci, int cj, int ck) {
    if (masked(ci, cj, ck)) return;
    smax_d = sig_max(smax_d, cell_signal<double, 0>(m, u, NS, sconst_d, cfl_form));
  };


  const int pstart = NDIM == 3 ? -1 : 0;
  const int pend = NDIM == 3 ? n : 0;   // inclusive
  if (NDIM == 3) {
    load_plane(-2, slot_of(-2));
    load_plane(-1, slot_of(-1));
    if (R4 || kLF) load_plane(0, slot_of(0));
  }
  for (int p = pstart; p <= pend; ++p) {
    const bool inner = p >= 0 && p < (NDIM == 3 ? n : 1);
    const int s0 = slot_of(p), sm = slot_of(p - 1), sp = slot_of(p + 1);
    if (R4 || kLF) {
      // four-plane ring: plane p + 1 is already in; plane p + 2 goes into the
      // slot plane p - 2 left, in the same phase as the predictor below
      // (FP64 with kLF: plane p + 1 came in the flux phase of plane p - 1)
      __syncthreads();
    } else {
      if (NDIM == 3) load_plane(p + 1, sp);
      else load_plane(0, 0);
      __syncthreads();
    }

    // ---- predictor: own column cell, then (inner planes) the radius-1 ring
    R zm[NF], zp[NF];
    {
      R fm[3][NF], fp[3][NF];
      predict<NDIM, T, R, !RK, NS, R4>(ring, sm, s0, sp, ti, tj, hdt, idx2, g, fm, fp);
      if (inner) {
#pragma unroll
        for (int v = 0; v < NF; ++v) {
          fxm[v * T * SM::W2 + tj * SM::W2 + ti + 1] = fm[0][v];
          fxp[v * T * SM::W2 + tj * SM::W2 + ti + 1] = fp[0][v];
          fym[v * SM::W2 * T + (tj + 1) * T + ti] = fm[1][v];
          fyp[v * SM::W2 * T + (tj + 1) * T + ti] = fp[1][v];
        }
      }
#pragma unroll
      for (int v = 0; v < NF; ++v) { zm[v] = fm[2][v]; zp[v] = fp[2][v]; }
    }
    R Fz[NF];
    if constexpr (kZD) {
      if (p >= 0) {
        if (inner && tid < kZT) {
#pragma unroll
          for (int v = 0; v < NF; ++v) {
            zbuf[v * kZT + tid] = zprev[v];
            zbuf[(NF + v) * kZT + tid] = zm[v];
          }
        } else {
          hllc<2, R, NS>(zprev, zm, g, igm1, m, Fz);
          if (reg && (p == 0 || p == n)) {
            const int face = p == 0 ? 4 : 5;
#pragma unroll
            for (int v = 0; v < NF; ++v) put_reg<RK>(reg[(face * NF + v) * nfc + (y0 + tj) * n + (x0 + ti)], Fz[v], st);
          }
        }
      }
    }
    if (inner) {
      for (int c = tid; c < 4 * T; c += NT) {
        const int side = c / T, e = c % T;
        int i, j;
        if (side == 0) { i = -1; j = e; }
        else if (side == 1) { i = T; j = e; }
        else if (side == 2) { i = e; j = -1; }
        else { i = e; j = T; }
        if constexpr (std::is_same<R, dw>::value && NS == 0) {
          // single-gas double-word tile: the one predictor body the kernel
          // already inlines (a second one, for the face state alone, measured
          // slower in this instruction-fetch-sensitive kernel)
          R fm[3][NF], fp[3][NF];
          predict<NDIM, T, R, !RK, NS, R4>(ring, sm, s0, sp, i, j, hdt, idx2, g, fm, fp);
          if (side < 2) {
#pragma unroll
            for (int v = 0; v < NF; ++v) {
              fxm[v * T * SM::W2 + j * SM::W2 + i + 1] = fm[0][v];
              fxp[v * T * SM::W2 + j * SM::W2 + i + 1] = fp[0][v];
            }
          } else {
#pragma unroll
            for (int v = 0; v < NF; ++v) {
              fym[v * SM::W2 * T + (j + 1) * T + i] = fm[1][v];
              fyp[v * SM::W2 * T + (j + 1) * T + i] = fp[1][v];
            }
          }
        } else {
          // the one face state the tile's faces read: the upper one of the
          // lower rings (x face 0, y face 0), the lower one of the upper rings
          R fs[NF];
          predict_face<NDIM, T, R, !RK, NS, R4>(ring, sm, s0, sp, i, j, hdt, idx2, g, side >> 1,
                                                (side & 1) == 0, fs);
          R *dst = side == 0 ? fxp + j * SM::W2
                             : (side == 1 ? fxm + j * SM::W2 + T + 1
                                          : (side == 2 ? fyp + i : fym + (T + 1) * T + i));
#pragma unroll
          for (int v = 0; v < NF; ++v) dst[v * T * SM::W2] = fs[v];
        }
      }
    }
    if (R4 && p + 2 <= pend + 1) load_plane(p + 2, slot_of(p + 2));
    __syncthreads();

    // ---- fluxes: x and y faces of inner planes (in place over the lower-face
    // state), z face below the thread's own cell
    const int zglob = p;  // interior z index of this plane
    if constexpr (std::is_same<R, dw>::value) {
      // double-word tile: one inlined Riemann solver serves every face of the
      // thread -- its x/y faces of inner planes, then its z face below -- with
      // the normal velocity swapped into the x slot, to keep the code size down
      constexpr int VS = T * SM::W2;                   // component stride of the face arrays
      const int nxy = inner ? 2 * (T + 1) * T : 0;
      int f = (tid + kFaceShift) % NT;
      bool zpend = NDIM == 3 && p >= 0;
      while (f < nxy || zpend) {
        const bool zf = f >= nxy;
        int dir = 2, a = 0, e = 0;
        R *sr = nullptr;
        R WL[NF], WR[NF], F[NF];
        if (!zf) {
          dir = f >= (T + 1) * T;
          const int ff = dir ? f - (T + 1) * T : f;
          if (ff < T * T) {
            if (!dir) { a = ff % T; e = ff / T; }
            else { a = ff / T; e = ff % T; }
          } else {
            a = T; e = ff - T * T;
          }
          const R *sl = dir ? fyp + a * T + e : fxp + e * SM::W2 + a;
          sr = dir ? fym + (a + 1) * T + e : fxm + e * SM::W2 + a + 1;
#pragma unroll
          for (int v = 0; v < NF; ++v) {
            WL[v] = sl[v * VS];
            WR[v] = sr[v * VS];
          }
        } else {
#pragma unroll
          for (int v = 0; v < NF; ++v) {
            WL[v] = zprev[v];
            WR[v] = zm[v];
          }
        }
        auto swap_normal = [&](R (&w)[NF]) {
          if (dir == 1) { const R t = w[1]; w[1] = w[2]; w[2] = t; }
          else if (dir == 2) { const R t = w[1]; w[1] = w[3]; w[3] = t; }
        };
        swap_normal(WL);
        swap_normal(WR);
        hllc<0, R, NS>(WL, WR, g, igm1, m, F);
        swap_normal(F);
        if (!zf) {
#pragma unroll
          for (int v = 0; v < NF; ++v) sr[v * VS] = F[v];
          const int o0 = dir ? y0 : x0;
          if (reg && ((a == 0 && o0 == 0) || (a == T && o0 + T == n))) {
            const int face = 2 * dir + (a == 0 ? 0 : 1);
            const int t1 = (dir ? x0 : y0) + e, t2 = NDIM == 3 ? zglob : 0;
#pragma unroll
            for (int v = 0; v < NF; ++v) put_reg<RK>(reg[(face * NF + v) * nfc + t2 * n + t1], F[v], st);
          }
          f += NT;
        } else {
#pragma unroll
          for (int v = 0; v < NF; ++v) Fz[v] = F[v];
          if (reg && (p == 0 || p == n)) {
            const int face = p == 0 ? 4 : 5;
#pragma unroll
            for (int v = 0; v < NF; ++v) put_reg<RK>(reg[(face * NF + v) * nfc + (y0 + tj) * n + (x0 + ti)], Fz[v], st);
          }
          zpend = false;
        }
      }
    } else {
      if (inner) {
        for (int f = (tid + kFaceShift) % NT; f < 2 * (T + 1) * T; f += NT) {
          const int dir = f >= (T + 1) * T;
          const int ff = dir ? f - (T + 1) * T : f;
          // a: face index along the normal (0..T), e: transverse index; the
          // lanes of a warp take consecutive x so shared-memory rows stay
          // contiguous for both directions
          int a, e;
          if (ff < T * T) {
            if (!dir) { a = ff % T; e = ff / T; }
            else { a = ff / T; e = ff % T; }
          } else {
            a = T; e = ff - T * T;
          }
          R WL[NF], WR[NF], F[NF];
          if (!dir) {
#pragma unroll
            for (int v = 0; v < NF; ++v) {
              WL[v] = fxp[v * T * SM::W2 + e * SM::W2 + a];
              WR[v] = fxm[v * T * SM::W2 + e * SM::W2 + a + 1];
            }
            hllc<0, R, NS>(WL, WR, g, igm1, m, F);
#pragma unroll
            for (int v = 0; v < NF; ++v) fxm[v * T * SM::W2 + e * SM::W2 + a + 1] = F[v];
            if (reg && ((a == 0 && x0 == 0) || (a == T && x0 + T == n))) {
              const int face = a == 0 ? 0 : 1;
              const int t1 = y0 + e, t2 = NDIM == 3 ? zglob : 0;
#pragma unroll
              for (int v = 0; v < NF; ++v) put_reg<RK>(reg[(face * NF + v) * nfc + t2 * n + t1], F[v], st);
            }
          } else {
#pragma unroll
            for (int v = 0; v < NF; ++v) {
              WL[v] = fyp[v * SM::W2 * T + a * T + e];
              WR[v] = fym[v * SM::W2 * T + (a + 1) * T + e];
            }
            hllc<1, R, NS>(WL, WR, g, igm1, m, F);
#pragma unroll
            for (int v = 0; v < NF; ++v) fym[v * SM::W2 * T + (a + 1) * T + e] = F[v];
            if (reg && ((a == 0 && y0 == 0) || (a == T && y0 + T == n))) {
              const int face = a == 0 ? 2 : 3;
              const int t1 = x0 + e, t2 = NDIM == 3 ? zglob : 0;
#pragma unroll
              for (int v = 0; v < NF; ++v) put_reg<RK>(reg[(face * NF + v) * nfc + t2 * n + t1], F[v], st);
            }
          }
        }
      }
      if constexpr (kZD) {
        // the halo-predictor threads' z faces
        const int dz = tid - kZ0;
        if (inner && p >= 0 && dz >= 0 && dz < kZT) {
          R WL[NF], WR[NF], F[NF];
#pragma unroll
          for (int v = 0; v < NF; ++v) {
            WL[v] = zbuf[v * kZT + dz];
            WR[v] = zbuf[(NF + v) * kZT + dz];
          }
          hllc<2, R, NS>(WL, WR, g, igm1, m, F);
#pragma unroll
          for (int v = 0; v < NF; ++v) zbuf[(NF + v) * kZT + dz] = F[v];
          if (reg && (p == 0 || p == n)) {
            const int face = p == 0 ? 4 : 5;
            const int ci = x0 + dz % T, cj = y0 + dz / T;
#pragma unroll
            for (int v = 0; v < NF; ++v) put_reg<RK>(reg[(face * NF + v) * nfc + cj * n + ci], F[v], st);
          }
        }
      } else if (NDIM == 3 && p >= 0) {
        hllc<2, R, NS>(zprev, zm, g, igm1, m, Fz);
        if (reg && (p == 0 || p == n)) {
          const int face = p == 0 ? 4 : 5;
#pragma unroll
          for (int v = 0; v < NF; ++v) put_reg<RK>(reg[(face * NF + v) * nfc + (y0 + tj) * n + (x0 + ti)], Fz[v], st);
        }
      }
      if constexpr (kLF) {
        if (loader && p + 2 <= pend + 1) load_cells(p + 2, slot_of(p + 2), lrank, kLoaders);
      }
    }
    __syncthreads();
    if constexpr (kZD) {
      if (inner && p >= 0 && tid < kZT) {
#pragma unroll
        for (int v = 0; v < NF; ++v) Fz[v] = zbuf[(NF + v) * kZT + tid];
      }
    }

    // ---- update: finish the cell below (3D), start this plane's cell.
    // FP64: U + dt ((Fx- - Fx+)/dx + (Fy- - Fy+)/dy + (Fz- - Fz+)/dz).
    // FP32 storage: exact flux differences scaled by dt/dx, summed, one
    // rounding when added to U.
    if (NDIM == 3 && p >= 1) {
      const long long o = ((long long)(p - 1 + ng) * P + (y0 + tj + ng)) * P + (x0 + ti + ng);
      R un[NF];
      [[maybe_unused]] double ud[NF];
#pragma unroll
      for (int v = 0; v < NF; ++v) {
        if constexpr (kF32) {
          const float d = txy[v] + scaled_diff(fzl[v], Fz[v], cz);
          if constexpr (kAbl) {
            ud[v] = Ub[o + v * vs] + double(d);
            un[v] = float(ud[v]);
          } else {
            un[v] = float(Ub[o + v * vs]) + d;
          }
        } else {
          const R div = txy[v] + (fzl[v] - Fz[v]) * rdz;
          un[v] = R(Ub[o + v * vs]) + rdt * div;
        }
        if constexpr (RK) {
          if (Uavg)
            un[v] = fma(R(st.wa), R(Uavg[(long long)b * m.bstride + o + v * vs]), R(st.wb) * un[v]);
        }
        if constexpr (kAbl) Unb[o + v * vs] = ud[v];
        else Unb[o + v * vs] = S(un[v]);
      }
      if (!(un[0] > R(0)) || !(R(2) * un[4] * un[0] > un[1] * un[1] + un[2] * un[2] + un[3] * un[3]))
        atomicOr(status, 1);
      if (smax_out) {
        if constexpr (kAbl) signal_d(ud, x0 + ti, y0 + tj, p - 1);
        else signal(un, x0 + ti, y0 + tj, p - 1);
      }
    }
    if (inner) {
      const R *Fx = fxm + tj * SM::W2 + ti + 1;
      const R *Fy = fym + (tj + 1) * T + ti;
#pragma unroll
      for (int v = 0; v < NF; ++v) {
        const R fxl = Fx[v * T * SM::W2], fxr = Fx[v * T * SM::W2 + 1];
        const R fyl = Fy[v * SM::W2 * T], fyr = Fy[v * SM::W2 * T + T];
        if constexpr (kF32) {
          txy[v] = scaled_diff(fxl, fxr, cx) + scaled_diff(fyl, fyr, cy);
        } else {
          txy[v] = (fxl - fxr) * rdx + (fyl - fyr) * rdy;
        }
        if (NDIM == 3) fzl[v] = Fz[v];
      }
      if (NDIM == 2) {
        const long long o = (long long)(y0 + tj + ng) * P + (x0 + ti + ng);
        R un[NF];
        [[maybe_unused]] double ud[NF];
#pragma unroll
        for (int v = 0; v < NF; ++v) {
          if constexpr (kAbl) {
            ud[v] = Ub[o + v * vs] + double(txy[v]);
            un[v] = float(ud[v]);
          } else if constexpr (kF32) {
            un[v] = float(Ub[o + v * vs]) + txy[v];
          } else {
            un[v] = R(Ub[o + v * vs]) + rdt * txy[v];
          }
          if constexpr (RK) {
            if (Uavg)
              un[v] = fma(R(st.wa), R(Uavg[(long long)b * m.bstride + o + v * vs]), R(st.wb) * un[v]);
          }
          if constexpr (kAbl) Unb[o + v * vs] = ud[v];
          else Unb[o + v * vs] = S(un[v]);
        }
        if (!(un[0] > R(0)) ||
            !(R(2) * un[4] * un[0] > un[1] * un[1] + un[2] * un[2] + un[3] * un[3]))
          atomicOr(status, 1);
        if (smax_out) {
          if constexpr (kAbl) signal_d(ud, x0 + ti, y0 + tj, 0);
          else signal(un, x0 + ti, y0 + tj, 0);
        }
      }
    }
#pragma unroll
    for (int v = 0; v < NF; ++v) zprev[v] = zp[v];
  }
  if (smax_out) {
    // maximum over the CTA on the bit patterns of non-negative doubles
    unsigned long long bits = __double_as_longlong(kAbl ? smax_d : double(smax_t));
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long other = __shfl_down_sync(0xffffffffu, bits, o);
      bits = other > bits ? other : bits;
    }
    if ((tid & 31) == 0) atomicMax(smax_out, bits);
  }
}

}  // namespace
}  // namespace fx
