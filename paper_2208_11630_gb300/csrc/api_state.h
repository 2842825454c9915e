// api_state.h -- private to the host side of libfx: the structures behind
// the opaque handles of fx.h (a context, a block set) and the error helpers
// shared by the files that implement the entry points (fx_api.cpp: contexts,
// block sets and steps; host_io.cpp: host round trips; regrid_api.cpp:
// regridding; batch_api.cpp: batched stepping).
#pragma once

#include "../../include/fx.h"
#include "fx_internal.h"

#include <string>
#include <vector>

using fx::DevMesh;
using fx::RefluxItem;


struct fx_ctx {
  double gamma = 1.4;
  int nxb = 16, ng = 4;
  int cfl_form = 0;
  int reflux = 1;
  int integrator = 0;   // 0 MUSCL-Hancock, 1 SSP-RK2, 2 SSP-RK3
  int f64_arith = 0;    // MUSCL-Hancock update of FP64 sets: 0 FP64, 1 double-word, 2 FP32
  int nspec = 0;        // multispecies perfect gas: species and their constants
  double spa[FX_MAXSPEC] = {0, 0, 0, 0}, spb[FX_MAXSPEC] = {0, 0, 0, 0};
  int device = 0;
  std::string err;
};

struct fx_blocks {
  fx_ctx *ctx = nullptr;
  int ndim = 3, nb = 0, nxb = 16, ng = 4, P = 24, PZ = 24, lmax = 0, prec = 0;
  int nvar = 5;                             // variables per cell (5 + species)
  size_t elsize = 8;
  void *U[2] = {nullptr, nullptr};
  int cur = 0;
  DevMesh dm{};
  // host copies
  std::vector<int> level, parent, leaf, child, origin;
  // device tables
  int *d_level = nullptr, *d_origin = nullptr, *d_child = nullptr, *d_regidx = nullptr;
  int2 *d_slots = nullptr;
  int *d_lists = nullptr;     // concatenated work lists
  int leaves_off = 0, nleaves = 0;
  std::vector<int> par_off, par_cnt;        // parents per level
  int2 *d_pslots = nullptr;                 // (leaf, slot) items covered by a coarser leaf
  std::vector<int> pslot_off, pslot_cnt;    // per level
  std::vector<int2> h_pslots;
  int src_off = 0, nsrc = 0;                // coarse leaves that feed a prolongation
  double *d_regs = nullptr;
  int nreg = 0;
  std::vector<int> regidx;
  RefluxItem *d_refl = nullptr;
  int nrefl = 0;
  unsigned long long *d_scratch = nullptr;  // [0] dt max bits, [1] CTA counter,
                                            // [2] signal-speed max of the last update
  unsigned char *d_rmask = nullptr;         // [nb] faces (bit 2d+s) the reflux corrects
  std::vector<int> h_lists;                 // host copy of the work lists
  std::vector<RefluxItem> h_refl;
  int in_batch = 0;                         // owned by a batch: stepped only through it
  long long epoch = 0;                      // bumped on every write of the current state
  long long next_epoch = -1;                // epoch described by d_scratch[2]
  long long restricted_epoch = -1;          // epoch whose parents are restricted
  int next_form = 0;
  int *d_status = nullptr;
  double *d_dt = nullptr;                   // dt scratch for fx_run_host
  double *d_totals = nullptr;               // [nleaves][nvar]; also the regrid indicator words
  // fx_run_host_interior: packed interior staging buffer and the streams and
  // events of the overlapped download (created on first use)
  void *d_pack = nullptr;
  void *d_U3 = nullptr;                     // third state buffer of SSP-RK3 (first use)
  // creation arguments kept for regridding, and the pending regrid plan
  int nroot[3] = {1, 1, 1};
  double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
  int bc[6] = {0, 0, 0, 0, 0, 0};
  int plan_valid = 0;
  fx::RegridPlan plan;
  std::vector<double> plan_err;             // indicator per block (-1: parent)
  cudaStream_t aux[2] = {nullptr, nullptr}, cpy = nullptr;
  cudaEvent_t ev_ready = nullptr, ev_done = nullptr, ev_chunk[8] = {}, ev_up[8] = {};
};

namespace fxapi {

// Stores msg as the context's last error and returns code.
int fail(fx_ctx *ctx, int code, const std::string &msg);
// fail() with FX_ERR_CUDA and the CUDA error string after where.
int cuda_fail(fx_ctx *ctx, cudaError_t e, const char *where);

}  // namespace fxapi

// Returns FX_ERR_CUDA from the enclosing entry point (whose block set is bs)
// when call does not succeed.
// The stage of a MUSCL-Hancock update of block set bs under context ctx
// (also the base of the SSP-RK stages): the arithmetic of its update.
inline fx::HydroStage muscl_stage(const fx_ctx *ctx, const fx_blocks *bs) {
  fx::HydroStage st;
  st.dword = bs->prec == 0 ? ctx->f64_arith : 0;
  return st;
}

#define FX_CUDA(call, where)                                         \
  do {                                                               \
    cudaError_t e_ = (call);                                         \
    if (e_ != cudaSuccess) return fxapi::cuda_fail(bs->ctx, e_, where); \
  } while (0)
