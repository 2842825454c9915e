// fx_internal.h -- types and kernel launchers shared by the libfx host code
// and its CUDA translation units.  Not part of the public ABI (include/fx.h).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "fx.h"

#define FX_MAXLEV 16
#define FX_MAXSPEC 4                 // species of the multispecies perfect gas
#define FX_MAXVAR (5 + FX_MAXSPEC)   // conserved variables per cell, at most

namespace fx {

// Guard-cell source of one neighbour slot of a leaf block.  Slot index
// (sx+1) + 3 (sy+1) + 9 (sz+1) for sx, sy, sz in {-1, 0, 1}.
enum SlotKind : int { SLOT_NONE = -1, SLOT_COPY = 0, SLOT_PROLONG = 1 };

// Everything a kernel needs to know about a block set, passed by value.
struct DevMesh {
  int ndim, nxb, ng, P, PZ, nb, lmax;
  long long vstride;             // elements of one variable of one block: PZ*P*P
  long long bstride;             // elements of one block: nvar*vstride
  int nvar, nspec;               // variables per cell (5 + nspec); species
  double spa[FX_MAXSPEC];        // 1 / A_k
  double spb[FX_MAXSPEC];        // 1 / (A_k (gamma_k - 1))
  int bc[3][2];                  // FX_BC_* per axis and side
  int ncell[FX_MAXLEV][3];       // cells per axis at each level
  double dx[FX_MAXLEV][3];       // cell widths at each level
  double idx[FX_MAXLEV][3];      // reciprocal cell widths
  double gamma;
  const int *level;              // [nb]
  const int *origin;             // [nb][3], cell index in the block's level lattice
  const int2 *slots;             // [nb][27] (kind, source block)
  const int *child;              // [nb][8], -1 if none
  const int *regidx;             // [nb] flux-register slot, -1 if none
  int nfaces;                    // 2*ndim
  int nface_cells;               // nxb^(ndim-1)
};

// Reflux work item: a coarse leaf with at least one face on a finer
// neighbour.  fine[f][q] = register slot of the fine child that covers
// transverse quarter q (q = h1 + 2 h2) of face f, -1 if the face is not
// corrected.
struct RefluxItem {
  int block;
  int fine[6][4];
};

// One block set inside a batch (device-resident; kernels of the batched step
// read it, the step-end kernel flips `cur` and counts `steps_left` down).
struct BatchReq {
  DevMesh m;
  void *U[2];
  int cur;                        // index of the current state buffer
  int steps_left;                 // > 0: advanced by the next batched step
  int prec;                       // 0 FP64, 1 FP32-bulk
  int form;                       // CFL form
  int reflux;                     // apply flux correction
  int nrefl;                      // reflux work items
  double cfl;
  double *dt;                     // this request's dt (device)
  double *regs;                   // flux registers (or null)
  int *status;                    // device status word
  unsigned long long *scratch;    // [2] = signal-speed max of the current state
  const unsigned char *rmask;     // faces corrected by reflux, per block (or null)
  const RefluxItem *refl;         // reflux work items (or null)
};

// Launchers.  Each returns the launch status (cudaGetLastError).  live (the
// coarse-fine launchers, may be null): every CTA returns at once while
// *live <= 0 -- the steps-left counter of a batched request whose step runs
// these per-block-set kernels.
cudaError_t launch_prim_to_cons(const DevMesh &m, const double *W, void *U, int prec,
                                cudaStream_t s);
cudaError_t launch_restrict(const DevMesh &m, void *U, int prec, const int *parents, int n,
                            cudaStream_t s, const int *live = nullptr);
// Interior cells of blocks [b0, b0 + nblk): dir 0 scatters a packed array
// [block][var][z][y][x] (relative to b0) into the padded layout, dir 1
// gathers them into it.
cudaError_t launch_pack(const DevMesh &m, void *U, int prec, void *packed, int b0, int nblk,
                        int dir, cudaStream_t s);
// Guard fills touch only guard cells within `depth` (Chebyshev distance) of
// the interior; prolongation of FP32 state computes in FP32 when
// state_precision_math is set (else FP64).
cudaError_t launch_guard_copy(const DevMesh &m, void *U, int prec, const int *leaves, int n,
                              int depth, cudaStream_t s, const int *live = nullptr);
// Prolonged guards of (leaf, slot) items -- slots covered by a coarser leaf
// -- within `depth`; the work is proportional to the prolonged cells.
cudaError_t launch_guard_prolong_slots(const DevMesh &m, void *U, int prec, const int2 *items,
                                       int n, int depth, int state_precision_math,
                                       cudaStream_t s, const int *live = nullptr);
// Guard depth the fused update reads (radius-2 stencil).
constexpr int kHydroGuardDepth = 2;
// Time-integration stage of one update launch (defaults: MUSCL-Hancock).
// Unew = wa Uavg + wb (U + dt L(U)) when Uavg is set (an SSP Runge-Kutta
// stage), else U + dt L(U); flux registers receive reg_w F, stored or (reg_add)
// added.
struct HydroStage {
  int pred = 1;               // 1: Hancock predictor; 0: PLM face states (SSP-RK)
  const void *Uavg = nullptr; // state blended into the stage result (or null)
  double wa = 0.5, wb = 0.5;  // blend weights
  double reg_w = 1.0;         // weight of the fluxes in the registers
  int reg_add = 0;            // 0 store, 1 add to the registers
  int dword = 0;              // FP64 state: 1 double-word arithmetic (MUSCL-Hancock only),
                              // 2 FP32 arithmetic (single gas, MUSCL-Hancock only)
  const int *live = nullptr;  // single-gas MUSCL-Hancock update of a batched request: every
                              // CTA returns at once while *live <= 0 (no steps left)
};

// smax (may be null): receives atomicMax of the bit patterns of the new
// state's CFL signal speeds (form 0 = sum over directions, 1 = max); cells on
// the faces flagged in rmask[block] (bit 2d+s) are left to the reflux kernel.
// The MUSCL-Hancock update, the multispecies update and the SSP-RK stages
// of an FP64 block set in double-word arithmetic (k_hydro_dw.cu,
// k_hydro_sp_dw.cu).
cudaError_t launch_hydro_dw(const DevMesh &m, const void *U, void *Unew, const int *leaves, int n,
                            const double *dt, double *regs, int *status,
                            unsigned long long *smax, const unsigned char *rmask, int form,
                            cudaStream_t s, const int *live = nullptr);
cudaError_t launch_hydro_species_dw(const DevMesh &m, const void *U, void *Unew,
                                    const int *leaves, int n, const double *dt, double *regs,
                                    int *status, unsigned long long *smax,
                                    const unsigned char *rmask, int form, cudaStream_t s);
cudaError_t launch_hydro_rk_dw(const DevMesh &m, const void *U, void *Unew, const int *leaves,
                               int n, const double *dt, double *regs, int *status,
                               unsigned long long *smax, const unsigned char *rmask, int form,
                               cudaStream_t s, const HydroStage &st);
cudaError_t launch_hydro(const DevMesh &m, const void *U, void *Unew, int prec, const int *leaves,
                         int n, const double *dt, double *regs, int *status,
                         unsigned long long *smax, const unsigned char *rmask, int form,
                         cudaStream_t s, const HydroStage &st = HydroStage());
// CTAs per SM of the per-block-set single-gas MUSCL-Hancock kernel that
// launch_hydro picks for blocks of edge nxb (compute class as for
// hydro_batch_fit), setting its shared-memory attribute on first use.
cudaError_t hydro_set_fit(int ndim, int nxb, int cls, int *fit);
cudaError_t hydro_set_fit_dw(int ndim, int nxb, int *fit);
// Regridding: per-leaf maximum of the Loehner indicator on density and
// pressure (filter eps) into err_bits[i] for leaves[i] (bit patterns, zeroed
// by the caller; guards filled); and the state transfer onto a new mesh,
// map[j] = (kind 0 copy / 1 prolong, old block, octant, -) per new block.
cudaError_t launch_regrid_err(const DevMesh &m, const void *U, int prec, const int *leaves, int n,
                              double eps, unsigned long long *err_bits, cudaStream_t s);
cudaError_t launch_regrid_transfer(const DevMesh &mo, const void *Uold, const DevMesh &mn,
                                   void *Unew, int prec, const int4 *map, cudaStream_t s);
// The multispecies MUSCL-Hancock kernels behind launch_hydro (m.nspec > 0).
cudaError_t launch_hydro_species(const DevMesh &m, const void *U, void *Unew, int prec,
                                 const int *leaves, int n, const double *dt, double *regs,
                                 int *status, unsigned long long *smax,
                                 const unsigned char *rmask, int form, cudaStream_t s);
// The SSP Runge-Kutta stage kernels behind launch_hydro (st.pred == 0).
cudaError_t launch_hydro_rk(const DevMesh &m, const void *U, void *Unew, int prec,
                            const int *leaves, int n, const double *dt, double *regs, int *status,
                            unsigned long long *smax, const unsigned char *rmask, int form,
                            cudaStream_t s, const HydroStage &st);
cudaError_t launch_reflux(const DevMesh &m, void *Unew, int prec, const RefluxItem *items, int n,
                          const double *dt, const double *regs, int *status,
                          unsigned long long *smax, int form, cudaStream_t s,
                          const int *live = nullptr);
// dt = cfl / (maximum held in *smax), then re-arms *smax to zero.
cudaError_t launch_dt_finalize(unsigned long long *smax, double cfl, double *dt_out,
                               cudaStream_t s);
cudaError_t launch_dt(const DevMesh &m, const void *U, int prec, const int *leaves, int n,
                      double cfl, int form, double *dt_out, unsigned long long *scratch,
                      cudaStream_t s);
cudaError_t launch_totals(const DevMesh &m, const void *U, int prec, const int *leaves, int n,
                          double *out, cudaStream_t s);

// Phases of the batched step (see k_batch.cu).
enum BatchPhase : int {
  BATCH_COPY = 1,
  BATCH_PROLONG = 2,
  BATCH_REFLUX = 3,
  BATCH_RESTRICT = 4
};
cudaError_t launch_batch_begin(BatchReq *reqs, int n, cudaStream_t s);
cudaError_t launch_batch_end(BatchReq *reqs, int n, cudaStream_t s);
cudaError_t launch_batch_phase(int phase, int prec, const BatchReq *reqs, const int4 *items, int n,
                               cudaStream_t s);
// Signal-speed maximum of a state (bit pattern) into *max_out, without
// forming dt; scratch as for launch_dt.
// accumulate: atomicMax into *max_out instead of storing (several ranges).
cudaError_t launch_signal_max(const DevMesh &m, const void *U, int prec, const int *leaves, int n,
                              int form, unsigned long long *max_out, unsigned long long *scratch,
                              cudaStream_t s, int accumulate = 0);
// Occupancy of the batched hydro kernel (CTAs per SM), setting its shared
// memory attribute on first use.  prec is the compute class of the update:
// 0 FP64, 1 FP32-bulk, 2 FP64 state in double-word arithmetic.
cudaError_t hydro_batch_fit(int ndim, int tile, int prec, int *fit);
cudaError_t hydro_batch_fit_dw(int ndim, int tile, int *fit);

// Batched persistent hydro kernel over (request, block, tile, tiles) items
// of one compute class (as above).  ctas_per_sm <= 0 means as many as fit.
cudaError_t launch_hydro_batch(int ndim, int tile, int prec, const BatchReq *reqs,
                               const int4 *items, int nitems, unsigned int *counter,
                               int ctas_per_sm, int nsm, cudaStream_t s);
cudaError_t launch_hydro_batch_dw(int ndim, int tile, const BatchReq *reqs, const int4 *items,
                                  int nitems, unsigned int *counter, int ctas_per_sm, int nsm,
                                  cudaStream_t s);

// Host plan of a regrid (regrid.cpp): the new mesh sorted by (level, z, y,
// x) and, per new block, (kind 0 keep / 1 new child, old block or old
// parent, octant, 0).  Returns FX_OK or FX_ERR_MESH with *msg set.
struct RegridPlan {
  std::vector<int> level, parent;
  std::vector<long long> origin;   // [n][3]
  std::vector<int4> map;
};
int regrid_plan(int ndim, int nxb, const int nroot[3], const int bc[6], int nb,
                const std::vector<int> &level, const std::vector<int> &origin,
                const std::vector<int> &parent, const std::vector<double> &err, double rc,
                double dc, int max_level, RegridPlan *out, std::string *msg);

// Element-wise double-word operation for fx_dword_selftest (k_dword_test.cu).
cudaError_t launch_dword_test(int op, const double *a, const double *b, double *out, int n,
                              cudaStream_t s);

// Raises the dynamic shared-memory limit of kernel `func` to `bytes` on the
// current device, once per device: the attribute belongs to that device's
// context, so one flag per process would skip a second device and its launch
// would fail.  `done` holds one bit per device ordinal (ordinals >= 64 set the
// attribute on every call); two threads that race on a first call both set
// the same value, which is harmless.
cudaError_t set_smem_once(const void *func, size_t bytes, std::atomic<unsigned long long> &done);

// Process-wide count of kernels launched by the library.
void count_launch(int n = 1);
long long launch_count();

}  // namespace fx
