// fx_api.cpp -- host side of libfx: contexts, block-set metadata (neighbour
// slots, level lists, flux-register map) and the C entry points of fx.h.
//
// Paper: Flash-X (arXiv 2208.11630), Section 2 -- the Grid unit owns the mesh
// (uniform grid or PARAMESH octree of blocks) and the fine-coarse boundary
// resolution; physics updates blocks one by one.  This file is the Grid's
// bookkeeping: it resolves, once per block set, where every guard region of
// every leaf comes from (same-level block, physical boundary, or a leaf one
// level coarser), which coarse faces need flux correction, and which blocks
// need flux registers.  Kernels then run from flat device tables.

#include "api_state.h"

#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>


namespace fx {
static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

cudaError_t set_smem_once(const void *func, size_t bytes, std::atomic<unsigned long long> &done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = (dev >= 0 && dev < 64) ? 1ull << dev : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  if (bit) done.fetch_or(bit, std::memory_order_release);
  return cudaSuccess;
}
}  // namespace fx

namespace fxapi {

int fail(fx_ctx *ctx, int code, const std::string &msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int cuda_fail(fx_ctx *ctx, cudaError_t e, const char *where) {
  return fail(ctx, FX_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

}  // namespace fxapi

using fxapi::cuda_fail;
using fxapi::fail;

namespace {

template <typename T>
int upload(fx_blocks *bs, T **dst, const std::vector<T> &src) {
  if (src.empty()) { *dst = nullptr; return FX_OK; }
  cudaError_t e = cudaMalloc((void **)dst, sizeof(T) * src.size());
  if (e != cudaSuccess) return fail(bs->ctx, FX_ERR_OOM, "cudaMalloc of a mesh table failed");
  e = cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(bs->ctx, e, "upload of a mesh table");
  return FX_OK;
}

void free_blocks(fx_blocks *bs) {
  cudaFree(bs->d_level); cudaFree(bs->d_origin); cudaFree(bs->d_child);
  cudaFree(bs->d_regidx); cudaFree(bs->d_slots); cudaFree(bs->d_lists);
  cudaFree(bs->d_regs); cudaFree(bs->d_refl); cudaFree(bs->d_scratch);
  cudaFree(bs->d_status); cudaFree(bs->d_dt); cudaFree(bs->d_totals); cudaFree(bs->d_rmask);
  cudaFree(bs->d_pslots);
  if (bs->cpy) cudaStreamSynchronize(bs->cpy);
  for (cudaStream_t a : bs->aux)
    if (a) { cudaStreamSynchronize(a); cudaStreamDestroy(a); }
  if (bs->cpy) cudaStreamDestroy(bs->cpy);
  if (bs->ev_ready) cudaEventDestroy(bs->ev_ready);
  if (bs->ev_done) cudaEventDestroy(bs->ev_done);
  for (cudaEvent_t e : bs->ev_chunk)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : bs->ev_up)
    if (e) cudaEventDestroy(e);
  cudaFree(bs->d_pack);
  cudaFree(bs->d_U3);
}

struct Lattice {
  // (level, bx, by, bz) -> block; block indices are below 2^30 per axis
  struct Key {
    int l, x, y, z;
    bool operator==(const Key &o) const { return l == o.l && x == o.x && y == o.y && z == o.z; }
  };
  struct Hash {
    size_t operator()(const Key &k) const {
      uint64_t h = (uint64_t)(uint32_t)k.x * 0x9E3779B97F4A7C15ull;
      h ^= ((uint64_t)(uint32_t)k.y + ((uint64_t)(uint32_t)k.l << 40)) * 0xC2B2AE3D27D4EB4Full;
      h ^= (uint64_t)(uint32_t)k.z * 0x165667B19E3779F9ull;
      return (size_t)(h ^ (h >> 29));
    }
  };
  std::unordered_map<Key, int, Hash> map;
  static Key key(int l, const long long bc[3]) { return Key{l, (int)bc[0], (int)bc[1], (int)bc[2]}; }
  int find(int l, const long long bc[3]) const {
    auto it = map.find(key(l, bc));
    return it == map.end() ? -1 : it->second;
  }
};

}  // namespace

extern "C" {

int fx_init(double gamma, int nxb, int nguard, fx_ctx **out) {
  if (!out) return FX_ERR_ARG;
  *out = nullptr;
  if (!(gamma > 1.0) || nxb < 8 || nxb > 64 || nxb % 8 || nguard < 2 || nguard > nxb / 2)
    return FX_ERR_ARG;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return FX_ERR_CUDA;
  int ndev = 0;
  e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) return FX_ERR_CUDA;
  fx_ctx *c = new (std::nothrow) fx_ctx;
  if (!c) return FX_ERR_OOM;
  c->gamma = gamma;
  c->nxb = nxb;
  c->ng = nguard;
  c->device = dev;
  *out = c;
  return FX_OK;
}

int fx_finalize(fx_ctx *ctx) {
  delete ctx;
  return FX_OK;
}

int fx_set_species(fx_ctx *ctx, int nspec, const double *gamma_k, const double *A_k) {
  if (!ctx || nspec < 0 || nspec > FX_MAXSPEC || (nspec && (!gamma_k || !A_k)))
    return FX_ERR_ARG;
  for (int k = 0; k < nspec; ++k)
    if (!(gamma_k[k] > 1.0) || !(A_k[k] > 0.0))
      return fail(ctx, FX_ERR_ARG, "species need gamma_k > 1 and A_k > 0");
  ctx->nspec = nspec;
  for (int k = 0; k < FX_MAXSPEC; ++k) {
    ctx->spa[k] = k < nspec ? 1.0 / A_k[k] : 0.0;
    ctx->spb[k] = k < nspec ? 1.0 / (A_k[k] * (gamma_k[k] - 1.0)) : 0.0;
  }
  return FX_OK;
}

int fx_set_option(fx_ctx *ctx, const char *key, double value) {
  if (!ctx || !key) return FX_ERR_ARG;
  if (!strcmp(key, "cfl_form")) {
    if (value != 0.0 && value != 1.0) return fail(ctx, FX_ERR_ARG, "cfl_form must be 0 or 1");
    ctx->cfl_form = (int)value;
    return FX_OK;
  }
  if (!strcmp(key, "reflux")) {
    if (value != 0.0 && value != 1.0) return fail(ctx, FX_ERR_ARG, "reflux must be 0 or 1");
    ctx->reflux = (int)value;
    return FX_OK;
  }
  if (!strcmp(key, "f64_arith")) {
    if (value != 0.0 && value != 1.0 && value != 2.0)
      return fail(ctx, FX_ERR_ARG, "f64_arith must be 0, 1 or 2");
    ctx->f64_arith = (int)value;
    return FX_OK;
  }
  if (!strcmp(key, "integrator")) {
    if (value != 0.0 && value != 1.0 && value != 2.0)
      return fail(ctx, FX_ERR_ARG, "integrator must be 0, 1 or 2");
    ctx->integrator = (int)value;
    return FX_OK;
  }
  return fail(ctx, FX_ERR_ARG, std::string("unknown option ") + key);
}

const char *fx_last_error(const fx_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int fx_blocks_create(fx_ctx *ctx, int ndim, int nblocks, int nxb, const int nroot[3],
                     const int *level, const int64_t *origin, const int *parent,
                     const double lo[3], const double hi[3], const int bc[6], int precision,
                     void *U0, void *U1, fx_blocks **out) {
  if (!ctx || !out) return FX_ERR_ARG;
  *out = nullptr;
  if (nxb == 0) nxb = ctx->nxb;
  if ((ndim != 2 && ndim != 3) || nblocks < 1 || !nroot || !level || !origin || !parent || !lo ||
      !hi || !bc || !U0 || !U1)
    return fail(ctx, FX_ERR_ARG, "null or out-of-range argument");
  if (nxb < 8 || nxb > 64 || nxb % 8 || ctx->ng > nxb / 2)
    return fail(ctx, FX_ERR_ARG, "nxb must be a multiple of 8 in [8, 64] with nguard <= nxb/2");
  if (precision != FX_F64 && precision != FX_F32BULK)
    return fail(ctx, FX_ERR_ARG, "precision must be FX_F64 or FX_F32BULK");
  if (((uintptr_t)U0 | (uintptr_t)U1) & 15) return fail(ctx, FX_ERR_ARG, "state buffers must be 16-byte aligned");
  for (int d = 0; d < ndim; ++d) {
    if (nroot[d] < 1 || !(hi[d] > lo[d])) return fail(ctx, FX_ERR_ARG, "bad nroot or domain");
    for (int s = 0; s < 2; ++s)
      if (bc[2 * d + s] != FX_BC_OUTFLOW && bc[2 * d + s] != FX_BC_PERIODIC &&
          bc[2 * d + s] != FX_BC_REFLECT)
        return fail(ctx, FX_ERR_ARG, "bad boundary kind");
    if ((bc[2 * d] == FX_BC_PERIODIC) != (bc[2 * d + 1] == FX_BC_PERIODIC))
      return fail(ctx, FX_ERR_ARG, "periodic boundaries must be set on both sides of an axis");
  }
  fx_blocks *bs = new (std::nothrow) fx_blocks;
  if (!bs) return fail(ctx, FX_ERR_OOM, "host allocation failed");
  bs->ctx = ctx;
  bs->ndim = ndim;
  bs->nb = nblocks;
  bs->nxb = nxb;
  bs->ng = ctx->ng;
  bs->P = nxb + 2 * ctx->ng;
  bs->PZ = ndim == 3 ? bs->P : 1;
  bs->prec = precision;
  bs->elsize = precision == FX_F64 ? 8 : 4;
  bs->nvar = 5 + ctx->nspec;
  bs->U[0] = U0;
  bs->U[1] = U1;
  for (int d = 0; d < 3; ++d) {
    bs->nroot[d] = d < ndim ? nroot[d] : 1;
    bs->lo[d] = d < ndim ? lo[d] : 0.0;
    bs->hi[d] = d < ndim ? hi[d] : 1.0;
  }
  for (int i = 0; i < 6; ++i) bs->bc[i] = i < 2 * ndim ? bc[i] : FX_BC_OUTFLOW;
  const int nb = nblocks, n = nxb;
  auto bail = [&](int code, const std::string &msg) {
    free_blocks(bs);
    delete bs;
    return fail(ctx, code, msg);
  };

  // ---- host metadata
  bs->level.assign(level, level + nb);
  bs->parent.assign(parent, parent + nb);
  bs->origin.assign(3 * nb, 0);
  bs->leaf.assign(nb, 1);
  bs->child.assign(8 * nb, -1);
  int lmax = 0;
  for (int b = 0; b < nb; ++b) {
    if (level[b] < 0 || level[b] >= FX_MAXLEV) return bail(FX_ERR_MESH, "level out of range");
    lmax = std::max(lmax, level[b]);
  }
  bs->lmax = lmax;
  long long ncell[FX_MAXLEV][3];
  for (int l = 0; l <= lmax; ++l)
    for (int d = 0; d < 3; ++d) ncell[l][d] = d < ndim ? ((long long)nroot[d] * n) << l : 1;
  if (ncell[lmax][0] > (1LL << 30) || ncell[lmax][1] > (1LL << 30) || ncell[lmax][2] > (1LL << 30))
    return bail(FX_ERR_MESH, "lattice too large");
  Lattice lat;
  lat.map.reserve(2 * (size_t)nb);
  for (int b = 0; b < nb; ++b) {
    long long bcd[3];
    for (int d = 0; d < 3; ++d) {
      long long o = d < ndim ? origin[3 * b + d] : 0;
      if (o % n || o < 0 || o >= ncell[level[b]][d])
        return bail(FX_ERR_MESH, "block origin not on the block lattice of its level");
      bs->origin[3 * b + d] = (int)o;
      bcd[d] = o / n;
    }
    if (!lat.map.emplace(Lattice::key(level[b], bcd), b).second)
      return bail(FX_ERR_MESH, "two blocks at the same position");
  }
  for (int b = 0; b < nb; ++b) {
    int p = parent[b];
    if (p < 0) {
      if (level[b] != 0) return bail(FX_ERR_MESH, "block above level 0 without a parent");
      continue;
    }
    if (p >= nb || level[p] != level[b] - 1) return bail(FX_ERR_MESH, "parent on the wrong level");
    int oct = 0;
    for (int d = 0; d < ndim; ++d) {
      int rel = bs->origin[3 * b + d] - 2 * bs->origin[3 * p + d];
      if (rel != 0 && rel != n) return bail(FX_ERR_MESH, "child outside its parent");
      if (rel) oct |= 1 << d;
    }
    if (bs->child[8 * p + oct] >= 0) return bail(FX_ERR_MESH, "duplicate child");
    bs->child[8 * p + oct] = b;
    bs->leaf[p] = 0;
  }
  for (int b = 0; b < nb; ++b)
    if (!bs->leaf[b])
      for (int c = 0; c < (1 << ndim); ++c)
        if (bs->child[8 * b + c] < 0) return bail(FX_ERR_MESH, "parent with a missing child");

  // ---- guard slots of every leaf
  std::vector<int2> slots(27 * nb, make_int2(fx::SLOT_NONE, -1));
  std::vector<std::vector<int2>> pslots_by_level(lmax + 1);
  for (int b = 0; b < nb; ++b) {
    if (!bs->leaf[b]) continue;
    const int l = level[b];
    for (int sz = (ndim == 3 ? -1 : 0); sz <= (ndim == 3 ? 1 : 0); ++sz)
      for (int sy = -1; sy <= 1; ++sy)
        for (int sx = -1; sx <= 1; ++sx) {
          if (!sx && !sy && !sz) continue;
          const int s[3] = {sx, sy, sz};
          long long g[3];
          for (int d = 0; d < 3; ++d) {
            if (d >= ndim) { g[d] = 0; continue; }
            g[d] = bs->origin[3 * b + d] + (s[d] < 0 ? -1 : (s[d] > 0 ? n : 0));
            const long long N = ncell[l][d];
            if (g[d] < 0 || g[d] >= N) {
              const int kind = bc[2 * d + (g[d] < 0 ? 0 : 1)];
              if (kind == FX_BC_PERIODIC) g[d] = ((g[d] % N) + N) % N;
              else if (kind == FX_BC_REFLECT) g[d] = g[d] < 0 ? -1 - g[d] : 2 * N - 1 - g[d];
              else g[d] = g[d] < 0 ? 0 : N - 1;
            }
          }
          long long bcd[3] = {g[0] / n, g[1] / n, g[2] / n};
          int2 sl;
          int src = lat.find(l, bcd);
          if (src >= 0) {
            sl = make_int2(fx::SLOT_COPY, src);
          } else {
            long long cb[3] = {(g[0] / 2) / n, (g[1] / 2) / n, ndim == 3 ? (g[2] / 2) / n : 0};
            int c = l > 0 ? lat.find(l - 1, cb) : -1;
            if (c < 0 || !bs->leaf[c])
              return bail(FX_ERR_MESH, "guard region of block " + std::to_string(b) +
                                           " not covered by a same-level block or a coarser "
                                           "leaf (mesh not 2:1 balanced)");
            sl = make_int2(fx::SLOT_PROLONG, c);
            pslots_by_level[l].push_back(make_int2(b, (sx + 1) + 3 * (sy + 1) + 9 * (sz + 1)));
          }
          slots[27 * b + (sx + 1) + 3 * (sy + 1) + 9 * (sz + 1)] = sl;
        }
  }

  // ---- flux correction: coarse leaf faces on a refined same-level block
  std::vector<RefluxItem> refl;
  bs->regidx.assign(nb, -1);
  auto reg = [&](int b) {
    if (bs->regidx[b] < 0) bs->regidx[b] = bs->nreg++;
    return bs->regidx[b];
  };
  for (int c = 0; c < nb; ++c) {
    if (!bs->leaf[c] || level[c] >= lmax) continue;
    RefluxItem it;
    it.block = c;
    bool any = false;
    for (int f = 0; f < 6; ++f)
      for (int q = 0; q < 4; ++q) it.fine[f][q] = -1;
    for (int d = 0; d < ndim; ++d) {
      const int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;
      for (int s = 0; s < 2; ++s) {
        long long bcd[3] = {bs->origin[3 * c] / n, bs->origin[3 * c + 1] / n,
                            bs->origin[3 * c + 2] / n};
        bcd[d] += s ? 1 : -1;
        const long long NB = ncell[level[c]][d] / n;
        if (bcd[d] < 0 || bcd[d] >= NB) {
          if (bc[2 * d + s] != FX_BC_PERIODIC) continue;
          bcd[d] = (bcd[d] + NB) % NB;
        }
        const int nbk = lat.find(level[c], bcd);
        if (nbk < 0 || bs->leaf[nbk]) continue;
        any = true;
        for (int h2 = 0; h2 < (ndim == 3 ? 2 : 1); ++h2)
          for (int h1 = 0; h1 < 2; ++h1) {
            int oct = (s ? 0 : 1) << d;
            oct |= h1 << a1;
            if (ndim == 3) oct |= h2 << a2;
            const int ch = bs->child[8 * nbk + oct];
            if (ch < 0 || !bs->leaf[ch])
              return bail(FX_ERR_MESH, "coarse-fine face spans more than one level");
            it.fine[2 * d + s][h1 + 2 * h2] = ch;
          }
      }
    }
    if (any) refl.push_back(it);
  }
  for (auto &it : refl) {
    reg(it.block);
    for (int f = 0; f < 6; ++f)
      for (int q = 0; q < 4; ++q)
        if (it.fine[f][q] >= 0) it.fine[f][q] = reg(it.fine[f][q]);
  }
  bs->nrefl = (int)refl.size();
  std::vector<unsigned char> rmask(nb, 0);
  for (auto &it : refl)
    for (int f = 0; f < 6; ++f)
      if (it.fine[f][0] >= 0) rmask[it.block] |= (unsigned char)(1u << f);

  // ---- work lists: leaves | parents per level | coarse leaves feeding prolongation
  std::vector<int> lists;
  for (int b = 0; b < nb; ++b)
    if (bs->leaf[b]) lists.push_back(b);
  bs->leaves_off = 0;
  bs->nleaves = (int)lists.size();
  bs->par_off.assign(lmax + 1, 0);
  bs->par_cnt.assign(lmax + 1, 0);
  for (int l = 0; l <= lmax; ++l) {
    bs->par_off[l] = (int)lists.size();
    for (int b = 0; b < nb; ++b)
      if (!bs->leaf[b] && level[b] == l) lists.push_back(b);
    bs->par_cnt[l] = (int)lists.size() - bs->par_off[l];
  }
  {
    std::vector<char> is_src(nb, 0);
    for (int b = 0; b < nb; ++b)
      for (int q = 0; q < 27; ++q)
        if (slots[27 * b + q].x == fx::SLOT_PROLONG) is_src[slots[27 * b + q].y] = 1;
    bs->src_off = (int)lists.size();
    for (int b = 0; b < nb; ++b)
      if (is_src[b]) lists.push_back(b);
    bs->nsrc = (int)lists.size() - bs->src_off;
  }

  // ---- device tables
  int rc;
  if ((rc = upload(bs, &bs->d_level, bs->level))) return bail(rc, ctx->err);
  if ((rc = upload(bs, &bs->d_origin, bs->origin))) return bail(rc, ctx->err);
  if ((rc = upload(bs, &bs->d_child, bs->child))) return bail(rc, ctx->err);
  if ((rc = upload(bs, &bs->d_regidx, bs->regidx))) return bail(rc, ctx->err);
  if ((rc = upload(bs, &bs->d_slots, slots))) return bail(rc, ctx->err);
  if ((rc = upload(bs, &bs->d_lists, lists))) return bail(rc, ctx->err);
  bs->h_lists = lists;
  bs->pslot_off.assign(lmax + 1, 0);
  bs->pslot_cnt.assign(lmax + 1, 0);
  bs->h_pslots.clear();
  for (int l = 0; l <= lmax; ++l) {
    bs->pslot_off[l] = (int)bs->h_pslots.size();
    bs->h_pslots.insert(bs->h_pslots.end(), pslots_by_level[l].begin(), pslots_by_level[l].end());
    bs->pslot_cnt[l] = (int)bs->h_pslots.size() - bs->pslot_off[l];
  }
  if ((rc = upload(bs, &bs->d_pslots, bs->h_pslots))) return bail(rc, ctx->err);
  bs->h_refl = refl;
  if ((rc = upload(bs, &bs->d_refl, refl))) return bail(rc, ctx->err);
  if (bs->nrefl > 0 && (rc = upload(bs, &bs->d_rmask, rmask))) return bail(rc, ctx->err);
  const int nfc = ndim == 3 ? n * n : n;
  if (bs->nreg > 0) {
    if (cudaMalloc(&bs->d_regs, sizeof(double) * (size_t)bs->nreg * 2 * ndim * bs->nvar * nfc) != cudaSuccess)
      return bail(FX_ERR_OOM, "cudaMalloc of flux registers failed");
  }
  if (cudaMalloc(&bs->d_scratch, 3 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&bs->d_status, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&bs->d_dt, sizeof(double)) != cudaSuccess ||
      cudaMalloc(&bs->d_totals, sizeof(double) * bs->nvar * (size_t)bs->nleaves) != cudaSuccess)
    return bail(FX_ERR_OOM, "cudaMalloc of scratch failed");
  if (cudaMemset(bs->d_scratch, 0, 3 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(bs->d_status, 0, sizeof(int)) != cudaSuccess)
    return bail(FX_ERR_CUDA, "cudaMemset of scratch failed");

  DevMesh &m = bs->dm;
  m.ndim = ndim; m.nxb = n; m.ng = bs->ng; m.P = bs->P; m.PZ = bs->PZ; m.nb = nb; m.lmax = lmax;
  m.vstride = (long long)bs->PZ * bs->P * bs->P;
  m.bstride = (long long)bs->nvar * m.vstride;
  m.nvar = bs->nvar;
  m.nspec = bs->nvar - 5;
  for (int k = 0; k < FX_MAXSPEC; ++k) {
    m.spa[k] = ctx->spa[k];
    m.spb[k] = ctx->spb[k];
  }
  for (int d = 0; d < 3; ++d)
    for (int s = 0; s < 2; ++s) m.bc[d][s] = d < ndim ? bc[2 * d + s] : FX_BC_OUTFLOW;
  for (int l = 0; l < FX_MAXLEV; ++l)
    for (int d = 0; d < 3; ++d) {
      if (l <= lmax && d < ndim) {
        m.ncell[l][d] = (int)ncell[l][d];
        m.dx[l][d] = (hi[d] - lo[d]) / (double)ncell[l][d];
        m.idx[l][d] = 1.0 / m.dx[l][d];
      } else {
        m.ncell[l][d] = 1; m.dx[l][d] = 1.0; m.idx[l][d] = 1.0;
      }
    }
  m.gamma = ctx->gamma;
  m.level = bs->d_level;
  m.origin = bs->d_origin;
  m.slots = bs->d_slots;
  m.child = bs->d_child;
  m.regidx = bs->d_regidx;
  m.nfaces = 2 * ndim;
  m.nface_cells = nfc;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return bail(FX_ERR_CUDA, std::string("sync: ") + cudaGetErrorString(e));
  *out = bs;
  return FX_OK;
}

int fx_blocks_destroy(fx_blocks *bs) {
  if (!bs) return FX_ERR_ARG;
  free_blocks(bs);
  delete bs;
  return FX_OK;
}

int fx_blocks_current(const fx_blocks *bs) { return bs ? bs->cur : FX_ERR_ARG; }

int fx_prim_to_cons(fx_ctx *ctx, fx_blocks *bs, const double *W_dev, void *stream) {
  if (!ctx || !bs || !W_dev) return FX_ERR_ARG;
  FX_CUDA(fx::launch_prim_to_cons(bs->dm, W_dev, bs->U[bs->cur], bs->prec, (cudaStream_t)stream),
          "prim_to_cons launch");
  ++bs->epoch;
  return FX_OK;
}

int fx_guardcell_fill(fx_ctx *ctx, fx_blocks *bs, void *stream) {
  if (!ctx || !bs) return FX_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  void *U = bs->U[bs->cur];
  for (int l = bs->lmax; l >= 0; --l)
    FX_CUDA(fx::launch_restrict(bs->dm, U, bs->prec, bs->d_lists + bs->par_off[l], bs->par_cnt[l], s),
            "restrict launch");
  FX_CUDA(fx::launch_guard_copy(bs->dm, U, bs->prec, bs->d_lists + bs->leaves_off, bs->nleaves,
                                bs->ng, s),
          "guard copy launch");
  for (int l = 1; l <= bs->lmax; ++l)
    FX_CUDA(fx::launch_guard_prolong_slots(bs->dm, U, bs->prec, bs->d_pslots + bs->pslot_off[l],
                                           bs->pslot_cnt[l], bs->ng, 0, s),
            "guard prolong launch");
  return FX_OK;
}

int fx_compute_dt(fx_ctx *ctx, fx_blocks *bs, double cfl, double *dt_dev, void *stream) {
  if (!ctx || !bs || !dt_dev || !(cfl > 0.0)) return FX_ERR_ARG;
  if (bs->nleaves == 0) return fail(ctx, FX_ERR_STATE, "no leaves");
  if (bs->next_epoch == bs->epoch && bs->next_form == ctx->cfl_form) {
    // the last update already reduced this state's signal speeds
    FX_CUDA(fx::launch_dt_finalize(bs->d_scratch + 2, cfl, dt_dev, (cudaStream_t)stream),
            "dt finalize launch");
    bs->next_epoch = -1;
    return FX_OK;
  }
  FX_CUDA(fx::launch_dt(bs->dm, bs->U[bs->cur], bs->prec, bs->d_lists + bs->leaves_off, bs->nleaves,
                        cfl, ctx->cfl_form, dt_dev, bs->d_scratch, (cudaStream_t)stream),
          "dt launch");
  return FX_OK;
}

int fx_blocks_mark_dirty(fx_blocks *bs) {
  if (!bs) return FX_ERR_ARG;
  ++bs->epoch;
  return FX_OK;
}

static int fill_for_fused_advance(fx_ctx *ctx, fx_blocks *bs, cudaStream_t s, void *U);

int fx_hydro_advance(fx_ctx *ctx, fx_blocks *bs, const double *dt_dev, void *stream) {
  if (!ctx || !bs || !dt_dev) return FX_ERR_ARG;
  if (bs->in_batch) return fail(ctx, FX_ERR_STATE, "block set is owned by a batch");
  cudaStream_t s = (cudaStream_t)stream;
  void *Uo = bs->U[bs->cur], *Un = bs->U[1 - bs->cur];
  unsigned long long *smax = bs->d_scratch + 2;
  const bool refl = ctx->reflux && bs->nrefl > 0;
  const int *leaves = bs->d_lists + bs->leaves_off;
  if ((ctx->integrator == 1 || ctx->integrator == 2) && bs->nvar > 5)
    return fail(ctx, FX_ERR_ARG, "the SSP-RK integrators step a single gas only");
  if (ctx->f64_arith == 2 && bs->prec == 0 && (ctx->integrator != 0 || bs->nvar > 5))
    return fail(ctx, FX_ERR_ARG,
                "FP32 arithmetic on FP64 state (f64_arith = 2) is the single-gas MUSCL-Hancock update only");
  if (ctx->integrator == 1 || ctx->integrator == 2) {
    // SSP-RK2: U1 = U + dt L(U) into the other buffer; coarse-fine fill of
    // U1; U = (U + (U1 + dt L(U1))) / 2 in place; registers hold the stage
    // average of the fluxes for the correction.
    // SSP-RK3: U1 as above; U2 = 3/4 U + 1/4 (U1 + dt L(U1)) into a third
    // buffer; U = 1/3 U + 2/3 (U2 + dt L(U2)) in place; register weights
    // 1/6, 1/6, 2/3.
    const bool rk3 = ctx->integrator == 2;
    if (rk3 && !bs->d_U3) {
      const size_t bytes = (size_t)bs->nb * bs->dm.bstride * bs->elsize;
      if (cudaMalloc(&bs->d_U3, bytes) != cudaSuccess) {
        bs->d_U3 = nullptr;
        cudaGetLastError();
        return fail(ctx, FX_ERR_OOM, "cudaMalloc of the SSP-RK3 stage buffer failed");
      }
      FX_CUDA(cudaMemsetAsync(bs->d_U3, 0, bytes, s), "stage buffer clear");
    }
    fx::HydroStage s1 = muscl_stage(ctx, bs), s2 = s1, s3 = s1;   // arithmetic (f64_arith)
    s1.pred = 0; s1.reg_w = rk3 ? 1.0 / 6.0 : 0.5;
    s2.pred = 0; s2.Uavg = Uo; s2.reg_add = 1;
    if (rk3) { s2.wa = 0.75; s2.wb = 0.25; s2.reg_w = 1.0 / 6.0; }
    else { s2.wa = 0.5; s2.wb = 0.5; s2.reg_w = 0.5; }
    s3.pred = 0; s3.Uavg = Uo; s3.reg_add = 1;
    s3.wa = 1.0 / 3.0; s3.wb = 2.0 / 3.0; s3.reg_w = 2.0 / 3.0;
    FX_CUDA(fx::launch_hydro(bs->dm, Uo, Un, bs->prec, leaves, bs->nleaves, dt_dev, bs->d_regs,
                             bs->d_status, nullptr, nullptr, ctx->cfl_form, s, s1),
            "hydro stage 1 launch");
    int rc = fill_for_fused_advance(ctx, bs, s, Un);
    if (rc) return rc;
    void *Ulast = Un;
    if (rk3) {
      FX_CUDA(fx::launch_hydro(bs->dm, Un, bs->d_U3, bs->prec, leaves, bs->nleaves, dt_dev,
                               bs->d_regs, bs->d_status, nullptr, nullptr, ctx->cfl_form, s, s2),
              "hydro stage 2 launch");
      rc = fill_for_fused_advance(ctx, bs, s, bs->d_U3);
      if (rc) return rc;
      Ulast = bs->d_U3;
    }
    FX_CUDA(cudaMemsetAsync(smax, 0, sizeof(unsigned long long), s), "signal max reset");
    FX_CUDA(fx::launch_hydro(bs->dm, Ulast, Uo, bs->prec, leaves, bs->nleaves, dt_dev, bs->d_regs,
                             bs->d_status, smax, refl ? bs->d_rmask : nullptr, ctx->cfl_form, s,
                             rk3 ? s3 : s2),
            "hydro final stage launch");
    if (refl)
      FX_CUDA(fx::launch_reflux(bs->dm, Uo, bs->prec, bs->d_refl, bs->nrefl, dt_dev, bs->d_regs,
                                bs->d_status, smax, ctx->cfl_form, s),
              "reflux launch");
    for (int l = bs->lmax; l >= 0; --l)
      FX_CUDA(fx::launch_restrict(bs->dm, Uo, bs->prec, bs->d_lists + bs->par_off[l],
                                  bs->par_cnt[l], s),
              "restrict launch");
    ++bs->epoch;                      // the new state is in the same buffer
    bs->next_epoch = bs->epoch;
    bs->restricted_epoch = bs->epoch;
    bs->next_form = ctx->cfl_form;
    return FX_OK;
  }
  FX_CUDA(cudaMemsetAsync(smax, 0, sizeof(unsigned long long), s), "signal max reset");
  FX_CUDA(fx::launch_hydro(bs->dm, Uo, Un, bs->prec, leaves, bs->nleaves,
                           dt_dev, bs->d_regs, bs->d_status, smax, refl ? bs->d_rmask : nullptr,
                           ctx->cfl_form, s, muscl_stage(ctx, bs)),
          "hydro launch");
  if (refl)
    FX_CUDA(fx::launch_reflux(bs->dm, Un, bs->prec, bs->d_refl, bs->nrefl, dt_dev, bs->d_regs,
                              bs->d_status, smax, ctx->cfl_form, s),
            "reflux launch");
  for (int l = bs->lmax; l >= 0; --l)
    FX_CUDA(fx::launch_restrict(bs->dm, Un, bs->prec, bs->d_lists + bs->par_off[l], bs->par_cnt[l], s),
            "restrict launch");
  bs->cur = 1 - bs->cur;
  ++bs->epoch;
  bs->next_epoch = bs->epoch;
  bs->next_form = ctx->cfl_form;
  bs->restricted_epoch = bs->epoch;   // the update ends with the restriction
  return FX_OK;
}

// The part of the guard fill that the fused hydro kernel still needs: parents
// restricted (they are same-level sources), the guards of coarse leaves that
// feed a prolongation, and the prolonged guards themselves.  Same-level guards
// of every other leaf are read by the hydro kernel from the neighbours.  The
// restriction is skipped for the current state when the update that wrote it
// already restricted it and nothing has written it since (state epochs).
static int fill_for_fused_advance(fx_ctx *ctx, fx_blocks *bs, cudaStream_t s, void *U) {
  const bool restricted = U == bs->U[bs->cur] && bs->restricted_epoch == bs->epoch;
  for (int l = bs->lmax; l >= 0 && !restricted; --l)
    FX_CUDA(fx::launch_restrict(bs->dm, U, bs->prec, bs->d_lists + bs->par_off[l], bs->par_cnt[l], s),
            "restrict launch");
  FX_CUDA(fx::launch_guard_copy(bs->dm, U, bs->prec, bs->d_lists + bs->src_off, bs->nsrc,
                                fx::kHydroGuardDepth, s),
          "guard copy launch");
  for (int l = 1; l <= bs->lmax; ++l)
    FX_CUDA(fx::launch_guard_prolong_slots(bs->dm, U, bs->prec,
                                           bs->d_pslots + bs->pslot_off[l], bs->pslot_cnt[l],
                                           fx::kHydroGuardDepth, 1, s),
            "guard prolong launch");
  (void)ctx;
  return FX_OK;
}

int fx_guardcell_fill_amr(fx_ctx *ctx, fx_blocks *bs, void *stream) {
  if (!ctx || !bs) return FX_ERR_ARG;
  return fill_for_fused_advance(ctx, bs, (cudaStream_t)stream, bs->U[bs->cur]);
}

int fx_step(fx_ctx *ctx, fx_blocks *bs, double cfl, double *dt_dev, void *stream) {
  int rc = fx_compute_dt(ctx, bs, cfl, dt_dev, stream);
  if (rc) return rc;
  rc = fx_guardcell_fill_amr(ctx, bs, stream);
  if (rc) return rc;
  return fx_hydro_advance(ctx, bs, dt_dev, stream);
}

int fx_conserved_totals(fx_ctx *ctx, fx_blocks *bs, double *out_host, void *stream) {
  if (!ctx || !bs || !out_host) return FX_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  FX_CUDA(fx::launch_totals(bs->dm, bs->U[bs->cur], bs->prec, bs->d_lists + bs->leaves_off,
                            bs->nleaves, bs->d_totals, s),
          "totals launch");
  const int nv = bs->nvar;
  std::vector<double> h(nv * (size_t)bs->nleaves);
  FX_CUDA(cudaMemcpyAsync(h.data(), bs->d_totals, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s),
          "totals copy");
  FX_CUDA(cudaStreamSynchronize(s), "totals sync");
  for (int v = 0; v < nv; ++v) {
    double sum = 0.0, comp = 0.0;
    for (int i = 0; i < bs->nleaves; ++i) {
      double y = h[nv * (size_t)i + v] - comp;
      double t = sum + y;
      comp = (t - sum) - y;
      sum = t;
    }
    out_host[v] = sum;
  }
  return FX_OK;
}

int fx_status(fx_ctx *ctx, fx_blocks *bs) {
  if (!ctx || !bs) return FX_ERR_ARG;
  int h = 0;
  FX_CUDA(cudaDeviceSynchronize(), "status sync");
  FX_CUDA(cudaMemcpy(&h, bs->d_status, sizeof(int), cudaMemcpyDeviceToHost), "status copy");
  FX_CUDA(cudaMemset(bs->d_status, 0, sizeof(int)), "status reset");
  if (h) return fail(ctx, FX_ERR_UNPHYSICAL, "non-positive density or pressure after an update");
  return FX_OK;
}

long long fx_kernel_launches(void) { return fx::launch_count(); }

int fx_dword_selftest(int op, const double *a_dev, const double *b_dev, double *out_dev, int n,
                      void *stream) {
  if (op < 0 || op > 7 || n < 0 || !a_dev || !out_dev || ((op <= 3 || op == 7) && !b_dev))
    return FX_ERR_ARG;
  return fx::launch_dword_test(op, a_dev, b_dev, out_dev, n, (cudaStream_t)stream) == cudaSuccess
             ? FX_OK
             : FX_ERR_CUDA;
}

const double *fx_block_fluxes(const fx_blocks *bs, int b) {
  if (!bs || b < 0 || b >= bs->nb || bs->regidx[b] < 0 || !bs->d_regs) return nullptr;
  const int nfc = bs->ndim == 3 ? bs->nxb * bs->nxb : bs->nxb;
  return bs->d_regs + (size_t)bs->regidx[b] * 2 * bs->ndim * bs->nvar * nfc;
}

}  // extern "C"
