// regrid_api.cpp -- the regridding entry points: evaluate the refinement
// indicator on the device, plan the new octree on the host, and move the state
// onto the new blocks (copy or conservative prolongation, then restriction).
//
// Paper: Flash-X (arXiv 2208.11630), Section 2 -- the Grid unit refines and
// derefines PARAMESH blocks as the solution evolves.
#include "api_state.h"

#include <algorithm>
#include <array>
#include <cstdio>
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

int fx_regrid_plan_host(int ndim, int nxb, const int nroot[3], const int bc[6], int nblocks,
                        const int *level, const int64_t *origin, const int *parent,
                        const double *err, double refine_cutoff, double derefine_cutoff,
                        int max_level, int cap, int *nblocks_new, int *level_new,
                        int64_t *origin_new, int *parent_new, int *map_new, char *msg,
                        int msg_len) {
  auto bad = [&](int code, const char *text) {
    if (msg && msg_len > 0) std::snprintf(msg, (size_t)msg_len, "%s", text);
    return code;
  };
  if (msg && msg_len > 0) msg[0] = '\0';
  if (nblocks_new) *nblocks_new = 0;
  if ((ndim != 2 && ndim != 3) || nblocks < 1 || !nroot || !bc || !level || !origin || !parent ||
      !err || !nblocks_new || cap < 0 || max_level < 0 || max_level >= FX_MAXLEV - 1)
    return bad(FX_ERR_ARG, "null or out-of-range argument");
  if (cap > 0 && (!level_new || !origin_new || !parent_new || !map_new))
    return bad(FX_ERR_ARG, "null output array");
  if (nxb < 8 || nxb > 64 || nxb % 8) return bad(FX_ERR_ARG, "nxb must be a multiple of 8 in [8, 64]");
  int root[3], bcs[6];
  for (int d = 0; d < 3; ++d) {
    root[d] = d < ndim ? nroot[d] : 1;
    if (root[d] < 1) return bad(FX_ERR_ARG, "bad nroot");
  }
  for (int i = 0; i < 6; ++i) bcs[i] = i < 2 * ndim ? bc[i] : FX_BC_OUTFLOW;
  for (int d = 0; d < ndim; ++d) {
    for (int s = 0; s < 2; ++s)
      if (bcs[2 * d + s] != FX_BC_OUTFLOW && bcs[2 * d + s] != FX_BC_PERIODIC &&
          bcs[2 * d + s] != FX_BC_REFLECT)
        return bad(FX_ERR_ARG, "bad boundary kind");
    if ((bcs[2 * d] == FX_BC_PERIODIC) != (bcs[2 * d + 1] == FX_BC_PERIODIC))
      return bad(FX_ERR_ARG, "periodic boundaries must be set on both sides of an axis");
  }
  // the mesh: the same rules as fx_blocks_create (levels, origins on the
  // block lattice of their level, distinct positions, parents one level up
  // with every child present)
  const int nb = nblocks, nch = 1 << ndim;
  int lmax = 0;
  for (int b = 0; b < nb; ++b) {
    if (level[b] < 0 || level[b] >= FX_MAXLEV) return bad(FX_ERR_MESH, "level out of range");
    lmax = std::max(lmax, level[b]);
  }
  for (int d = 0; d < 3; ++d)
    if ((((long long)root[d] * nxb) << lmax) > (1LL << 30)) return bad(FX_ERR_MESH, "lattice too large");
  std::vector<int> lv(level, level + nb), pa(parent, parent + nb), org(3 * (size_t)nb);
  std::vector<std::array<long long, 4>> at(nb);
  for (int b = 0; b < nb; ++b) {
    at[b][0] = level[b];
    for (int d = 0; d < 3; ++d) {
      const long long o = d < ndim ? origin[3 * b + d] : 0;
      const long long N = d < ndim ? ((long long)root[d] * nxb) << level[b] : 1;
      if (o % nxb || o < 0 || o >= N)
        return bad(FX_ERR_MESH, "block origin not on the block lattice of its level");
      org[3 * b + d] = (int)o;
      at[b][1 + d] = o;
    }
  }
  std::sort(at.begin(), at.end());
  if (std::adjacent_find(at.begin(), at.end()) != at.end())
    return bad(FX_ERR_MESH, "two blocks at the same position");
  std::vector<int> child(8 * (size_t)nb, -1), leaf(nb, 1);
  for (int b = 0; b < nb; ++b) {
    const int p = parent[b];
    if (p < 0) {
      if (p != -1 || level[b] != 0) return bad(FX_ERR_MESH, "block above level 0 without a parent");
      continue;
    }
    if (p >= nb || level[p] != level[b] - 1) return bad(FX_ERR_MESH, "parent on the wrong level");
    int oct = 0;
    for (int d = 0; d < ndim; ++d) {
      const int rel = org[3 * b + d] - 2 * org[3 * p + d];
      if (rel != 0 && rel != nxb) return bad(FX_ERR_MESH, "child outside its parent");
      if (rel) oct |= 1 << d;
    }
    if (child[8 * p + oct] >= 0) return bad(FX_ERR_MESH, "duplicate child");
    child[8 * p + oct] = b;
    leaf[p] = 0;
  }
  for (int b = 0; b < nb; ++b)
    if (!leaf[b])
      for (int c = 0; c < nch; ++c)
        if (child[8 * b + c] < 0) return bad(FX_ERR_MESH, "parent with a missing child");
  fx::RegridPlan plan;
  std::string text;
  const int rc = fx::regrid_plan(ndim, nxb, root, bcs, nb, lv, org, pa,
                                 std::vector<double>(err, err + nb), refine_cutoff,
                                 derefine_cutoff, max_level, &plan, &text);
  if (rc) return bad(rc, text.c_str());
  const int n = (int)plan.level.size();
  *nblocks_new = n;
  if (n > cap) return bad(FX_ERR_ARG, "capacity below the planned block count");
  for (int j = 0; j < n; ++j) {
    level_new[j] = plan.level[j];
    parent_new[j] = plan.parent[j];
    for (int d = 0; d < 3; ++d) origin_new[3 * j + d] = plan.origin[3 * j + d];
    map_new[3 * j] = plan.map[j].x;
    map_new[3 * j + 1] = plan.map[j].y;
    map_new[3 * j + 2] = plan.map[j].z;
  }
  return FX_OK;
}

}  // extern "C"
