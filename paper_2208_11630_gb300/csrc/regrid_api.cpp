// regrid_api.cpp -- the regridding entry points: evaluate the refinement
// indicator on the device, plan the new octree on the host, and move the state
// onto the new blocks (copy or conservative prolongation, then restriction).
//
// Paper: Flash-X (arXiv 2208.11630), Section 2 -- the Grid unit refines and
// derefines PARAMESH blocks as the solution evolves.
#include "api_state.h"

#include <cstring>
#include <utility>

using fxapi::cuda_fail;
using fxapi::fail;

extern "C" {


int fx_regrid_plan(fx_ctx *ctx, fx_blocks *bs, double refine_cutoff, double derefine_cutoff,
                   double filter, int max_level, void *stream, int *nblocks_new) {
  if (!ctx || !bs || !nblocks_new || max_level < 0 || max_level >= FX_MAXLEV - 1 ||
      !(filter >= 0.0))
    return FX_ERR_ARG;
  if (bs->in_batch) return fail(ctx, FX_ERR_STATE, "block set is owned by a batch");
  cudaStream_t s = (cudaStream_t)stream;
  bs->plan_valid = 0;
  // parents restricted and every guard layer filled (no leaf interior changes)
  int rc = fx_guardcell_fill(ctx, bs, stream);
  if (rc) return rc;
  // the per-leaf indicator words use the totals scratch (nvar >= 5 doubles per leaf)
  unsigned long long *d_err = reinterpret_cast<unsigned long long *>(bs->d_totals);
  std::vector<unsigned long long> h(bs->nleaves);
  cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(unsigned long long) * bs->nleaves, s);
  if (e == cudaSuccess)
    e = fx::launch_regrid_err(bs->dm, bs->U[bs->cur], bs->prec, bs->d_lists + bs->leaves_off,
                              bs->nleaves, filter, d_err, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), d_err, sizeof(unsigned long long) * bs->nleaves,
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "regrid indicator");
  bs->plan_err.assign(bs->nb, -1.0);
  for (int i = 0; i < bs->nleaves; ++i) {
    double v;
    std::memcpy(&v, &h[i], sizeof v);
    bs->plan_err[bs->h_lists[bs->leaves_off + i]] = v;
  }
  std::string msg;
  rc = fx::regrid_plan(bs->ndim, bs->nxb, bs->nroot, bs->bc, bs->nb, bs->level, bs->origin,
                       bs->parent, bs->plan_err, refine_cutoff, derefine_cutoff, max_level,
                       &bs->plan, &msg);
  if (rc) return fail(ctx, rc, msg);
  bs->plan_valid = 1;
  *nblocks_new = (int)bs->plan.level.size();
  return FX_OK;
}

int fx_regrid_errors(const fx_blocks *bs, double *err_host) {
  if (!bs || !err_host) return FX_ERR_ARG;
  if (!bs->plan_valid) return FX_ERR_STATE;
  std::memcpy(err_host, bs->plan_err.data(), sizeof(double) * bs->nb);
  return FX_OK;
}

int fx_regrid_mesh(const fx_blocks *bs, int *level, int64_t *origin, int *parent) {
  if (!bs || !level || !origin || !parent) return FX_ERR_ARG;
  if (!bs->plan_valid) return FX_ERR_STATE;
  const size_t n = bs->plan.level.size();
  for (size_t j = 0; j < n; ++j) {
    level[j] = bs->plan.level[j];
    parent[j] = bs->plan.parent[j];
    for (int d = 0; d < 3; ++d) origin[3 * j + d] = bs->plan.origin[3 * j + d];
  }
  return FX_OK;
}

int fx_regrid_apply(fx_ctx *ctx, fx_blocks *bs, void *U0_new, void *U1_new, void *stream) {
  if (!ctx || !bs || !U0_new || !U1_new) return FX_ERR_ARG;
  if (bs->in_batch) return fail(ctx, FX_ERR_STATE, "block set is owned by a batch");
  if (!bs->plan_valid) return fail(ctx, FX_ERR_STATE, "no regrid plan");
  if (5 + ctx->nspec != bs->nvar)
    return fail(ctx, FX_ERR_STATE, "the context's species changed since the block set was made");
  cudaStream_t s = (cudaStream_t)stream;
  const int n = (int)bs->plan.level.size();
  fx_blocks *nbs = nullptr;
  int rc = fx_blocks_create(ctx, bs->ndim, n, bs->nxb, bs->nroot, bs->plan.level.data(),
                            reinterpret_cast<const int64_t *>(bs->plan.origin.data()),
                            bs->plan.parent.data(), bs->lo, bs->hi, bs->bc, bs->prec, U0_new,
                            U1_new, &nbs);
  if (rc) return rc;
  int4 *d_map = nullptr;
  cudaError_t e = cudaMalloc(&d_map, sizeof(int4) * n);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_map, bs->plan.map.data(), sizeof(int4) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = fx::launch_regrid_transfer(bs->dm, bs->U[bs->cur], nbs->dm, U0_new, bs->prec, d_map, s);
  for (int l = nbs->lmax; l >= 0 && e == cudaSuccess; --l)
    e = fx::launch_restrict(nbs->dm, U0_new, nbs->prec, nbs->d_lists + nbs->par_off[l],
                            nbs->par_cnt[l], s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_map);
  if (e != cudaSuccess) {
    fx_blocks_destroy(nbs);
    return cuda_fail(ctx, e, "regrid transfer");
  }
  // the handle keeps its identity: swap in the new mesh, free the old one
  std::swap(*bs, *nbs);
  fx_blocks_destroy(nbs);
  return FX_OK;
}

}  // extern "C"
