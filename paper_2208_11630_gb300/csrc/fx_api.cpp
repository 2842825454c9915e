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
#include "../../include/fx.h"
#include "fx_internal.h"

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

using fx::DevMesh;
using fx::RefluxItem;

struct fx_ctx {
  double gamma = 1.4;
  int nxb = 16, ng = 4;
  int cfl_form = 0;
  int reflux = 1;
  int integrator = 0;   // 0 MUSCL-Hancock, 1 SSP-RK2, 2 SSP-RK3
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
  int next_form = 0;
  int *d_status = nullptr;
  double *d_dt = nullptr;                   // dt scratch for fx_run_host
  double *d_totals = nullptr;               // [nleaves][nvar]
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

namespace fx {
static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace fx

namespace {

int fail(fx_ctx *ctx, int code, const std::string &msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int cuda_fail(fx_ctx *ctx, cudaError_t e, const char *where) {
  return fail(ctx, FX_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define FX_CUDA(call, where)                                         \
  do {                                                               \
    cudaError_t e_ = (call);                                         \
    if (e_ != cudaSuccess) return cuda_fail(bs->ctx, e_, where);     \
  } while (0)

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
  // (level, bx, by, bz) -> block
  std::map<std::tuple<int, long long, long long, long long>, int> map;
  int find(int l, const long long bc[3]) const {
    auto it = map.find(std::make_tuple(l, bc[0], bc[1], bc[2]));
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
  for (int b = 0; b < nb; ++b) {
    long long bcd[3];
    for (int d = 0; d < 3; ++d) {
      long long o = d < ndim ? origin[3 * b + d] : 0;
      if (o % n || o < 0 || o >= ncell[level[b]][d])
        return bail(FX_ERR_MESH, "block origin not on the block lattice of its level");
      bs->origin[3 * b + d] = (int)o;
      bcd[d] = o / n;
    }
    auto key = std::make_tuple(level[b], bcd[0], bcd[1], bcd[2]);
    if (lat.map.count(key)) return bail(FX_ERR_MESH, "two blocks at the same position");
    lat.map[key] = b;
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
    fx::HydroStage s1, s2, s3;
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
    bs->next_form = ctx->cfl_form;
    return FX_OK;
  }
  FX_CUDA(cudaMemsetAsync(smax, 0, sizeof(unsigned long long), s), "signal max reset");
  FX_CUDA(fx::launch_hydro(bs->dm, Uo, Un, bs->prec, leaves, bs->nleaves,
                           dt_dev, bs->d_regs, bs->d_status, smax, refl ? bs->d_rmask : nullptr,
                           ctx->cfl_form, s),
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
  return FX_OK;
}

// The part of the guard fill that the fused hydro kernel still needs: parents
// restricted (they are same-level sources), the guards of coarse leaves that
// feed a prolongation, and the prolonged guards themselves.  Same-level guards
// of every other leaf are read by the hydro kernel from the neighbours.
static int fill_for_fused_advance(fx_ctx *ctx, fx_blocks *bs, cudaStream_t s, void *U) {
  for (int l = bs->lmax; l >= 0; --l)
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

int fx_run_host(fx_ctx *ctx, fx_blocks *bs, const void *U_host_in, void *U_host_out, int nsteps,
                double cfl, double *t_host, void *stream) {
  if (!ctx || !bs || !U_host_in || !U_host_out || nsteps < 0) return FX_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)bs->nb * bs->dm.bstride * bs->elsize;
  FX_CUDA(cudaMemcpyAsync(bs->U[bs->cur], U_host_in, bytes, cudaMemcpyHostToDevice, s), "state upload");
  ++bs->epoch;
  double t = 0.0;
  for (int i = 0; i < nsteps; ++i) {
    int rc = fx_step(ctx, bs, cfl, bs->d_dt, stream);
    if (rc) return rc;
    if (t_host) {
      double dt = 0.0;
      FX_CUDA(cudaMemcpyAsync(&dt, bs->d_dt, sizeof(double), cudaMemcpyDeviceToHost, s), "dt copy");
      FX_CUDA(cudaStreamSynchronize(s), "dt sync");
      t += dt;
    }
  }
  FX_CUDA(cudaMemcpyAsync(U_host_out, bs->U[bs->cur], bytes, cudaMemcpyDeviceToHost, s), "state download");
  FX_CUDA(cudaStreamSynchronize(s), "run sync");
  if (t_host) *t_host = t;
  return FX_OK;
}

}  // extern "C"

namespace {

constexpr int kPipeChunks = 8;

// Bytes of one block's interior cells (all five variables).
size_t interior_block_bytes(const fx_blocks *bs) {
  return (size_t)bs->nvar * bs->nxb * bs->nxb * (bs->ndim == 3 ? bs->nxb : 1) * bs->elsize;
}

int ensure_pipeline(fx_blocks *bs) {
  if (bs->d_pack) return FX_OK;
  // streams and events first; the staging buffer last marks completion
  for (cudaStream_t &a : bs->aux)
    if (!a) FX_CUDA(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking), "stream create");
  if (!bs->cpy) FX_CUDA(cudaStreamCreateWithFlags(&bs->cpy, cudaStreamNonBlocking), "stream create");
  if (!bs->ev_ready)
    FX_CUDA(cudaEventCreateWithFlags(&bs->ev_ready, cudaEventDisableTiming), "event create");
  if (!bs->ev_done)
    FX_CUDA(cudaEventCreateWithFlags(&bs->ev_done, cudaEventDisableTiming), "event create");
  for (cudaEvent_t &e : bs->ev_chunk)
    if (!e) FX_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event create");
  for (cudaEvent_t &e : bs->ev_up)
    if (!e) FX_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event create");
  if (cudaMalloc(&bs->d_pack, interior_block_bytes(bs) * bs->nb) != cudaSuccess) {
    bs->d_pack = nullptr;
    cudaGetLastError();
    return fail(bs->ctx, FX_ERR_OOM, "cudaMalloc of the interior staging buffer failed");
  }
  return FX_OK;
}

// Update of a single-level block set whose leaves are all its blocks, in
// chunks of consecutive blocks on two alternating streams (so that one
// chunk's last CTAs overlap the next chunk's first); each chunk's interior
// is gathered and copied to the host as soon as it is done, overlapping the
// download with the rest of the update.  Same kernels and results as
// fx_hydro_advance.
int advance_and_download(fx_ctx *ctx, fx_blocks *bs, cudaStream_t s, void *W_out) {
  void *Uo = bs->U[bs->cur], *Un = bs->U[1 - bs->cur];
  unsigned long long *smax = bs->d_scratch + 2;
  const size_t pb = interior_block_bytes(bs);
  const int K = bs->nleaves < kPipeChunks ? bs->nleaves : kPipeChunks;
  FX_CUDA(cudaMemsetAsync(smax, 0, sizeof(unsigned long long), s), "signal max reset");
  FX_CUDA(cudaEventRecord(bs->ev_ready, s), "event record");
  for (int c = 0; c < K; ++c) {
    const int b0 = (int)((long long)bs->nleaves * c / K);
    const int b1 = (int)((long long)bs->nleaves * (c + 1) / K);
    cudaStream_t a = bs->aux[c & 1];
    if (c < 2) FX_CUDA(cudaStreamWaitEvent(a, bs->ev_ready, 0), "stream wait");
    FX_CUDA(fx::launch_hydro(bs->dm, Uo, Un, bs->prec, bs->d_lists + bs->leaves_off + b0, b1 - b0,
                             bs->d_dt, bs->d_regs, bs->d_status, smax, nullptr, ctx->cfl_form, a),
            "hydro launch");
    char *pk = static_cast<char *>(bs->d_pack) + pb * b0;
    FX_CUDA(fx::launch_pack(bs->dm, Un, bs->prec, pk, b0, b1 - b0, 1, a), "pack launch");
    FX_CUDA(cudaEventRecord(bs->ev_chunk[c], a), "event record");
    FX_CUDA(cudaStreamWaitEvent(bs->cpy, bs->ev_chunk[c], 0), "stream wait");
    FX_CUDA(cudaMemcpyAsync(static_cast<char *>(W_out) + pb * b0, pk, pb * (b1 - b0),
                            cudaMemcpyDeviceToHost, bs->cpy),
            "state download");
  }
  FX_CUDA(cudaEventRecord(bs->ev_done, bs->cpy), "event record");
  FX_CUDA(cudaStreamWaitEvent(s, bs->ev_done, 0), "stream wait");
  bs->cur = 1 - bs->cur;
  ++bs->epoch;
  bs->next_epoch = bs->epoch;
  bs->next_form = ctx->cfl_form;
  return FX_OK;
}

// Upload of a single-level block set's packed interiors in chunks of
// consecutive blocks on the copy stream; each chunk is scattered into the
// padded layout and its CFL signal maximum reduced on `s` as soon as it
// lands, so the dt reduction overlaps the rest of the upload.  Leaves
// dt = cfl / max in bs->d_dt.
int upload_and_reduce(fx_ctx *ctx, fx_blocks *bs, cudaStream_t s, const void *W_in, double cfl) {
  const size_t pb = interior_block_bytes(bs);
  const int K = bs->nb < kPipeChunks ? bs->nb : kPipeChunks;
  unsigned long long *smax = bs->d_scratch + 2;
  FX_CUDA(cudaMemsetAsync(smax, 0, sizeof(unsigned long long), s), "signal max reset");
  FX_CUDA(cudaEventRecord(bs->ev_ready, s), "event record");
  FX_CUDA(cudaStreamWaitEvent(bs->cpy, bs->ev_ready, 0), "stream wait");
  for (int c = 0; c < K; ++c) {
    const int b0 = (int)((long long)bs->nb * c / K), b1 = (int)((long long)bs->nb * (c + 1) / K);
    char *pk = static_cast<char *>(bs->d_pack) + pb * b0;
    FX_CUDA(cudaMemcpyAsync(pk, static_cast<const char *>(W_in) + pb * b0, pb * (b1 - b0),
                            cudaMemcpyHostToDevice, bs->cpy),
            "state upload");
    FX_CUDA(cudaEventRecord(bs->ev_up[c], bs->cpy), "event record");
    FX_CUDA(cudaStreamWaitEvent(s, bs->ev_up[c], 0), "stream wait");
    FX_CUDA(fx::launch_pack(bs->dm, bs->U[bs->cur], bs->prec, pk, b0, b1 - b0, 0, s),
            "unpack launch");
    FX_CUDA(fx::launch_signal_max(bs->dm, bs->U[bs->cur], bs->prec,
                                  bs->d_lists + bs->leaves_off + b0, b1 - b0, ctx->cfl_form, smax,
                                  bs->d_scratch, s, 1),
            "signal max launch");
  }
  FX_CUDA(fx::launch_dt_finalize(smax, cfl, bs->d_dt, s), "dt finalize launch");
  ++bs->epoch;
  return FX_OK;
}

}  // namespace

extern "C" {

int fx_run_host_interior(fx_ctx *ctx, fx_blocks *bs, const void *W_in, void *W_out, int nsteps,
                         double cfl, double *t_host, void *stream) {
  if (!ctx || !bs || !W_in || !W_out || nsteps < 0 || !(cfl > 0.0)) return FX_ERR_ARG;
  if (bs->in_batch) return fail(ctx, FX_ERR_STATE, "block set is owned by a batch");
  int rc = ensure_pipeline(bs);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = interior_block_bytes(bs) * bs->nb;
  const bool single_level = bs->lmax == 0 && bs->nrefl == 0 && bs->nleaves == bs->nb &&
                            ctx->integrator == 0;
  bool have_dt = false;
  if (single_level && nsteps > 0) {
    rc = upload_and_reduce(ctx, bs, s, W_in, cfl);   // dt of the uploaded state in d_dt
    if (rc) return rc;
    have_dt = true;
  } else {
    FX_CUDA(cudaMemcpyAsync(bs->d_pack, W_in, bytes, cudaMemcpyHostToDevice, s), "state upload");
    FX_CUDA(fx::launch_pack(bs->dm, bs->U[bs->cur], bs->prec, bs->d_pack, 0, bs->nb, 0, s),
            "unpack launch");
    ++bs->epoch;
  }
  bool downloaded = false;
  double t = 0.0;
  for (int i = 0; i < nsteps; ++i) {
    if (i == 0 && have_dt) {
      rc = fx_guardcell_fill_amr(ctx, bs, stream);
      if (!rc) {
        if (i == nsteps - 1) {
          rc = advance_and_download(ctx, bs, s, W_out);
          downloaded = true;
        } else {
          rc = fx_hydro_advance(ctx, bs, bs->d_dt, stream);
        }
      }
    } else if (i == nsteps - 1 && single_level) {
      rc = fx_compute_dt(ctx, bs, cfl, bs->d_dt, stream);
      if (!rc) rc = fx_guardcell_fill_amr(ctx, bs, stream);
      if (!rc) rc = advance_and_download(ctx, bs, s, W_out);
      downloaded = true;
    } else {
      rc = fx_step(ctx, bs, cfl, bs->d_dt, stream);
    }
    if (rc) return rc;
    if (t_host) {
      double dt = 0.0;
      FX_CUDA(cudaMemcpyAsync(&dt, bs->d_dt, sizeof(double), cudaMemcpyDeviceToHost, s), "dt copy");
      FX_CUDA(cudaStreamSynchronize(s), "dt sync");
      t += dt;
    }
  }
  if (!downloaded) {
    FX_CUDA(fx::launch_pack(bs->dm, bs->U[bs->cur], bs->prec, bs->d_pack, 0, bs->nb, 1, s),
            "pack launch");
    FX_CUDA(cudaMemcpyAsync(W_out, bs->d_pack, bytes, cudaMemcpyDeviceToHost, s), "state download");
  }
  FX_CUDA(cudaStreamSynchronize(s), "run sync");
  if (t_host) *t_host = t;
  return FX_OK;
}

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
  unsigned long long *d_err = nullptr;
  if (cudaMalloc(&d_err, sizeof(unsigned long long) * bs->nleaves) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, FX_ERR_OOM, "cudaMalloc of the indicator buffer failed");
  }
  std::vector<unsigned long long> h(bs->nleaves);
  cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(unsigned long long) * bs->nleaves, s);
  if (e == cudaSuccess)
    e = fx::launch_regrid_err(bs->dm, bs->U[bs->cur], bs->prec, bs->d_lists + bs->leaves_off,
                              bs->nleaves, filter, d_err, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), d_err, sizeof(unsigned long long) * bs->nleaves,
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_err);
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

long long fx_kernel_launches(void) { return fx::launch_count(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// batched, graph-replayed stepping of many block sets
// ---------------------------------------------------------------------------

using fx::BatchReq;

namespace {

struct Range {
  int off = 0, n = 0;
};

struct HydroGroup {
  int ndim, tile, prec;
  Range r;
  int ctas;   // CTAs per SM (0 = as many as fit)
};

// Tuned launch choice for one (ndim, precision) group of block sets whose
// nxb allows 16x16 tiles: the tile edge and the CTAs per SM.
struct Choice {
  int tile = 16;
  int ctas = 0;
};

// (ndim, prec, SM count, mask of the 16-capable block edges in the group)
std::map<std::tuple<int, int, int, int>, Choice> g_tune_cache;

}  // namespace

struct fx_batch {
  fx_ctx *ctx = nullptr;
  int max_req = 0, nsm = 0;
  std::vector<fx_blocks *> slot;
  std::vector<BatchReq> h_req;
  BatchReq *d_req = nullptr;
  double *d_dt = nullptr;
  int4 *d_items = nullptr;
  size_t items_cap = 0;
  unsigned int *d_ctr = nullptr;     // work counters, one per hydro group
  cudaStream_t cap = nullptr;        // private capture stream
  cudaGraphExec_t exec = nullptr;
  bool dirty = true;
  int lmax = 0;
  Range rst[2][FX_MAXLEV], cpy[2], pro[2][FX_MAXLEV], rfx[2];
  std::vector<HydroGroup> groups;
  Choice choice[2][2];               // [ndim - 2][prec]
  bool tuned[2][2] = {{false, false}, {false, false}};
};

namespace {

constexpr int kMaxGroups = 8;

// Work lists of the batched step for the current composition.
int build_lists(fx_batch *b, const Choice (&ch)[2][2]) {
  std::vector<int4> rst[2][FX_MAXLEV], cpy[2], pro[2][FX_MAXLEV], rfx[2];
  std::map<std::tuple<int, int, int>, std::vector<int4>> hyd;
  b->lmax = 0;
  for (int r = 0; r < b->max_req; ++r) {
    fx_blocks *bs = b->slot[r];
    if (!bs) continue;
    const int pr = bs->prec, nd = bs->ndim, n = bs->nxb;
    const std::vector<int> &L = bs->h_lists;
    const int ncell = n * n * (nd == 3 ? n : 1);
    const int chunks = (ncell + 255) / 256;
    b->lmax = std::max(b->lmax, bs->lmax);
    for (int l = 0; l <= bs->lmax; ++l) {
      for (int q = 0; q < bs->par_cnt[l]; ++q)
        for (int c = 0; c < chunks; ++c) rst[pr][l].push_back(make_int4(r, L[bs->par_off[l] + q], c, 0));
      for (int q = 0; q < bs->pslot_cnt[l]; ++q) {
        const int2 it = bs->h_pslots[bs->pslot_off[l] + q];
        pro[pr][l].push_back(make_int4(r, it.x, it.y, 0));
      }
    }
    for (int q = 0; q < bs->nsrc; ++q)
      for (int k = 0; k < bs->PZ; ++k) cpy[pr].push_back(make_int4(r, L[bs->src_off + q], k, 0));
    for (int q = 0; q < bs->nrefl; ++q)
      for (int c = 0; c < chunks; ++c) rfx[pr].push_back(make_int4(r, q, c, chunks));
    const int T = (n % 16 == 0) ? ch[nd - 2][pr].tile : 8;
    const int tiles = n / T;
    auto &H = hyd[std::make_tuple(nd, T, pr)];
    for (int q = 0; q < bs->nleaves; ++q)
      for (int t = 0; t < tiles * tiles; ++t)
        H.push_back(make_int4(r, L[bs->leaves_off + q], t, tiles));
  }
  std::vector<int4> all;
  auto put = [&](std::vector<int4> &v, Range &rg) {
    rg.off = (int)all.size();
    rg.n = (int)v.size();
    all.insert(all.end(), v.begin(), v.end());
  };
  for (int p = 0; p < 2; ++p) {
    for (int l = 0; l < FX_MAXLEV; ++l) {
      put(rst[p][l], b->rst[p][l]);
      put(pro[p][l], b->pro[p][l]);
    }
    put(cpy[p], b->cpy[p]);
    put(rfx[p], b->rfx[p]);
  }
  b->groups.clear();
  for (auto &kv : hyd) {
    HydroGroup g;
    g.ndim = std::get<0>(kv.first);
    g.tile = std::get<1>(kv.first);
    g.prec = std::get<2>(kv.first);
    g.ctas = g.tile == 16 || true ? ch[g.ndim - 2][g.prec].ctas : 0;
    put(kv.second, g.r);
    b->groups.push_back(g);
  }
  if ((int)b->groups.size() > kMaxGroups) return FX_ERR_STATE;
  if (all.size() > b->items_cap) {
    cudaFree(b->d_items);
    b->d_items = nullptr;
    size_t cap = std::max<size_t>(all.size(), 2 * b->items_cap);
    if (cudaMalloc(&b->d_items, cap * sizeof(int4)) != cudaSuccess) return FX_ERR_OOM;
    b->items_cap = cap;
  }
  if (!all.empty() &&
      cudaMemcpy(b->d_items, all.data(), all.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess)
    return FX_ERR_CUDA;
  return FX_OK;
}

cudaError_t record_step(fx_batch *b, cudaStream_t s) {
  cudaError_t e;
#define FXB(call) do { e = (call); if (e != cudaSuccess) return e; } while (0)
  FXB(fx::launch_batch_begin(b->d_req, b->max_req, s));
  for (int l = b->lmax - 1; l >= 0; --l)
    for (int p = 0; p < 2; ++p)
      FXB(fx::launch_batch_phase(fx::BATCH_RESTRICT_PRE, p, b->d_req, b->d_items + b->rst[p][l].off,
                                 b->rst[p][l].n, s));
  for (int p = 0; p < 2; ++p)
    FXB(fx::launch_batch_phase(fx::BATCH_COPY, p, b->d_req, b->d_items + b->cpy[p].off, b->cpy[p].n, s));
  for (int l = 1; l <= b->lmax; ++l)
    for (int p = 0; p < 2; ++p)
      FXB(fx::launch_batch_phase(fx::BATCH_PROLONG, p, b->d_req, b->d_items + b->pro[p][l].off,
                                 b->pro[p][l].n, s));
  for (size_t g = 0; g < b->groups.size(); ++g) {
    const HydroGroup &G = b->groups[g];
    FXB(cudaMemsetAsync(b->d_ctr + g, 0, sizeof(unsigned int), s));
    FXB(fx::launch_hydro_batch(G.ndim, G.tile, G.prec, b->d_req, b->d_items + G.r.off, G.r.n,
                               b->d_ctr + g, G.ctas, b->nsm, s));
  }
  for (int p = 0; p < 2; ++p)
    FXB(fx::launch_batch_phase(fx::BATCH_REFLUX, p, b->d_req, b->d_items + b->rfx[p].off, b->rfx[p].n, s));
  for (int l = b->lmax - 1; l >= 0; --l)
    for (int p = 0; p < 2; ++p)
      FXB(fx::launch_batch_phase(fx::BATCH_RESTRICT_POST, p, b->d_req, b->d_items + b->rst[p][l].off,
                                 b->rst[p][l].n, s));
  FXB(fx::launch_batch_end(b->d_req, b->max_req, s));
#undef FXB
  return cudaSuccess;
}

// The coarse-fine fill of the current buffers (restriction, copies feeding
// prolongation, prolongation): what an update needs to read valid guards.
cudaError_t record_fill(fx_batch *b, cudaStream_t s) {
  cudaError_t e;
  for (int l = b->lmax - 1; l >= 0; --l)
    for (int p = 0; p < 2; ++p)
      if ((e = fx::launch_batch_phase(fx::BATCH_RESTRICT_PRE, p, b->d_req, b->d_items + b->rst[p][l].off,
                                      b->rst[p][l].n, s)) != cudaSuccess)
        return e;
  for (int p = 0; p < 2; ++p)
    if ((e = fx::launch_batch_phase(fx::BATCH_COPY, p, b->d_req, b->d_items + b->cpy[p].off,
                                    b->cpy[p].n, s)) != cudaSuccess)
      return e;
  for (int l = 1; l <= b->lmax; ++l)
    for (int p = 0; p < 2; ++p)
      if ((e = fx::launch_batch_phase(fx::BATCH_PROLONG, p, b->d_req, b->d_items + b->pro[p][l].off,
                                      b->pro[p][l].n, s)) != cudaSuccess)
        return e;
  return cudaSuccess;
}

int capture(fx_batch *b) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  int rc = build_lists(b, b->choice);
  if (rc) return fail(b->ctx, rc, "building the batch work lists failed");
  for (const HydroGroup &G : b->groups) {   // attributes before capture
    int fit = 0;
    cudaError_t e = fx::hydro_batch_fit(G.ndim, G.tile, G.prec, &fit);
    if (e != cudaSuccess) return cuda_fail(b->ctx, e, "batched kernel set-up");
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(b->ctx, e, "begin capture");
  cudaError_t er = record_step(b, b->cap);
  e = cudaStreamEndCapture(b->cap, &g);
  if (er != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(b->ctx, er, "recording the batched step");
  }
  if (e != cudaSuccess) return cuda_fail(b->ctx, e, "end capture");
  e = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(b->ctx, e, "graph instantiate");
  b->dirty = false;
  return FX_OK;
}

}  // namespace

extern "C" {

int fx_batch_create(fx_ctx *ctx, int max_requests, fx_batch **out) {
  if (!ctx || !out || max_requests < 1 || max_requests > (1 << 20)) return FX_ERR_ARG;
  *out = nullptr;
  fx_batch *b = new (std::nothrow) fx_batch;
  if (!b) return fail(ctx, FX_ERR_OOM, "host allocation failed");
  b->ctx = ctx;
  b->max_req = max_requests;
  b->slot.assign(max_requests, nullptr);
  b->h_req.assign(max_requests, BatchReq{});
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaMalloc(&b->d_req, sizeof(BatchReq) * max_requests) != cudaSuccess ||
      cudaMalloc(&b->d_dt, sizeof(double) * max_requests) != cudaSuccess ||
      cudaMalloc(&b->d_ctr, sizeof(unsigned int) * kMaxGroups) != cudaSuccess ||
      cudaMemset(b->d_req, 0, sizeof(BatchReq) * max_requests) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFree(b->d_req); cudaFree(b->d_dt); cudaFree(b->d_ctr);
    delete b;
    return fail(ctx, FX_ERR_OOM, "batch allocation failed");
  }
  *out = b;
  return FX_OK;
}

int fx_batch_destroy(fx_batch *b) {
  if (!b) return FX_ERR_ARG;
  cudaDeviceSynchronize();
  for (fx_blocks *bs : b->slot)
    if (bs) bs->in_batch = 0;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  cudaFree(b->d_req); cudaFree(b->d_dt); cudaFree(b->d_ctr); cudaFree(b->d_items);
  delete b;
  return FX_OK;
}

int fx_batch_add(fx_batch *b, fx_blocks *bs, double cfl, int nsteps, void *stream, int *slot_out) {
  if (!b || !bs || !(cfl > 0.0) || nsteps < 1) return FX_ERR_ARG;
  if (bs->in_batch) return fail(b->ctx, FX_ERR_STATE, "block set already in a batch");
  if (bs->ctx->integrator != 0)
    return fail(b->ctx, FX_ERR_ARG, "batches step MUSCL-Hancock block sets only");
  if (bs->nvar != 5) return fail(b->ctx, FX_ERR_ARG, "batches step single-gas block sets only");
  int s = -1;
  for (int r = 0; r < b->max_req; ++r)
    if (!b->slot[r]) { s = r; break; }
  if (s < 0) return fail(b->ctx, FX_ERR_STATE, "batch is full");
  cudaStream_t st = (cudaStream_t)stream;
  BatchReq &q = b->h_req[s];
  q = BatchReq{};
  q.m = bs->dm;
  q.U[0] = bs->U[0];
  q.U[1] = bs->U[1];
  q.cur = bs->cur;
  q.steps_left = nsteps;
  q.prec = bs->prec;
  q.form = bs->ctx->cfl_form;
  q.reflux = (bs->ctx->reflux && bs->nrefl > 0) ? 1 : 0;
  q.nrefl = bs->nrefl;
  q.cfl = cfl;
  q.dt = b->d_dt + s;
  q.regs = bs->d_regs;
  q.status = bs->d_status;
  q.scratch = bs->d_scratch;
  q.rmask = q.reflux ? bs->d_rmask : nullptr;
  q.refl = bs->d_refl;
  // the first batched step needs the signal-speed maximum of the current state
  if (!(bs->next_epoch == bs->epoch && bs->next_form == q.form)) {
    FX_CUDA(fx::launch_signal_max(bs->dm, bs->U[bs->cur], bs->prec, bs->d_lists + bs->leaves_off,
                                  bs->nleaves, q.form, bs->d_scratch + 2, bs->d_scratch, st),
            "signal max launch");
  }
  FX_CUDA(cudaMemcpyAsync(b->d_req + s, &q, sizeof(BatchReq), cudaMemcpyHostToDevice, st),
          "batch descriptor upload");
  FX_CUDA(cudaStreamSynchronize(st), "batch add sync");
  b->slot[s] = bs;
  bs->in_batch = 1;
  b->dirty = true;
  if (slot_out) *slot_out = s;
  return FX_OK;
}

int fx_batch_run(fx_batch *b, int nsteps, void *stream) {
  if (!b || nsteps < 0) return FX_ERR_ARG;
  if (b->dirty) {
    // the new composition is captured after everything already queued
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(b->ctx, e, "batch sync");
    int rc = capture(b);
    if (rc) return rc;
  }
  for (int i = 0; i < nsteps; ++i) {
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(b->ctx, e, "graph launch");
  }
  return FX_OK;
}

int fx_batch_poll(fx_batch *b, int *steps_left, void *stream) {
  if (!b || !steps_left) return FX_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int> h(b->max_req, 0);
  cudaError_t e = cudaMemcpy2DAsync(h.data(), sizeof(int), &b->d_req[0].steps_left, sizeof(BatchReq),
                                    sizeof(int), b->max_req, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(b->ctx, e, "poll copy");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(b->ctx, e, "poll sync");
  for (int r = 0; r < b->max_req; ++r) steps_left[r] = b->slot[r] ? h[r] : -1;
  return FX_OK;
}

int fx_batch_remove(fx_batch *b, int slot, void *stream) {
  if (!b || slot < 0 || slot >= b->max_req || !b->slot[slot]) return FX_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  fx_blocks *bs = b->slot[slot];
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(b->ctx, e, "remove sync");
  BatchReq q;
  e = cudaMemcpy(&q, b->d_req + slot, sizeof(BatchReq), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(b->ctx, e, "descriptor read");
  // a request still running is cancelled: the captured graph skips it
  const int zero = 0;
  e = cudaMemcpy(&b->d_req[slot].steps_left, &zero, sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(b->ctx, e, "descriptor write");
  bs->cur = q.cur;
  ++bs->epoch;
  bs->next_epoch = bs->epoch;        // the last update left its signal maximum
  bs->next_form = q.form;
  bs->in_batch = 0;
  b->slot[slot] = nullptr;           // free for reuse (a new occupant recaptures)
  return FX_OK;
}

int fx_batch_tune(fx_batch *b, void *stream, int *report) {
  if (!b) return FX_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(b->ctx, e, "tune sync");
  // dt = 0 makes every timed update leave the state unchanged: the new
  // buffer receives a copy of the current one and the signal maximum of the
  // current state is reproduced; the next batched step recomputes dt
  e = cudaMemset(b->d_dt, 0, sizeof(double) * b->max_req);
  if (e != cudaSuccess) return cuda_fail(b->ctx, e, "tune dt reset");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // valid guards for every request before any timed update
  if (build_lists(b, b->choice)) return fail(b->ctx, FX_ERR_OOM, "tuning work lists");
  e = record_fill(b, st);
  if (e != cudaSuccess) return cuda_fail(b->ctx, e, "tuning guard fill");
  int nrep = 0;
  for (int nd = 2; nd <= 3; ++nd)
    for (int pr = 0; pr < 2; ++pr) {
      // is there a group of 16-capable block sets of this kind?
      int mask = 0;
      for (fx_blocks *bs : b->slot)
        if (bs && bs->ndim == nd && bs->prec == pr && bs->nxb % 16 == 0) mask |= 1 << (bs->nxb / 16);
      if (!mask) continue;
      auto key = std::make_tuple(nd, pr, b->nsm, mask);
      auto hit = g_tune_cache.find(key);
      if (hit != g_tune_cache.end()) {
        b->choice[nd - 2][pr] = hit->second;
        b->tuned[nd - 2][pr] = true;
        continue;
      }
      float best = 1e30f;
      Choice bestc;
      for (int tile : {16, 8}) {
        int fit = 0;
        e = fx::hydro_batch_fit(nd, tile, pr, &fit);
        if (e != cudaSuccess) break;
        for (int ctas = 1; ctas <= fit; ++ctas) {
          Choice ch[2][2];
          for (int a = 0; a < 2; ++a)
            for (int c = 0; c < 2; ++c) ch[a][c] = b->choice[a][c];
          ch[nd - 2][pr].tile = tile;
          ch[nd - 2][pr].ctas = ctas;
          if (build_lists(b, ch)) break;
          const HydroGroup *G = nullptr;
          int gi = 0;
          for (size_t g = 0; g < b->groups.size(); ++g)
            if (b->groups[g].ndim == nd && b->groups[g].prec == pr && b->groups[g].tile == tile) {
              G = &b->groups[g];
              gi = (int)g;
            }
          if (!G) continue;
          // time on a bounded sample: a dozen waves of the persistent grid,
          // in work per item (the 8x8 variant has four times the items); the
          // fastest of four launches after a warm-up one, so that a single
          // disturbed launch cannot decide the choice
          const int per_wave = ctas * b->nsm;
          int nsample = std::min(G->r.n, 12 * per_wave * (tile == 8 ? 4 : 1));
          nsample = std::max(nsample, std::min(G->r.n, per_wave));
          float best_ms = 1e30f;
          for (int rep = 0; rep < 5; ++rep) {
            cudaMemsetAsync(b->d_ctr + gi, 0, sizeof(unsigned int), st);
            cudaEventRecord(e0, st);
            fx::launch_hydro_batch(nd, tile, pr, b->d_req, b->d_items + G->r.off, nsample,
                                   b->d_ctr + gi, ctas, b->nsm, st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best_ms) best_ms = ms;   // first launch warms up
          }
          // normalise to the whole group: time per item times items
          const float est = best_ms * (float)G->r.n / (float)nsample;
          if (report && nrep < 64) {
            report[3 * nrep] = tile;
            report[3 * nrep + 1] = ctas;
            report[3 * nrep + 2] = std::max(1, (int)(est * 1000.f));   // microseconds
            ++nrep;
          }
          if (est < best) { best = est; bestc.tile = tile; bestc.ctas = ctas; }
        }
      }
      b->choice[nd - 2][pr] = bestc;
      b->tuned[nd - 2][pr] = true;
      g_tune_cache[key] = bestc;
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(b->ctx, e, "tuning");
  if (report) report[3 * nrep] = 0;
  b->dirty = true;
  return FX_OK;
}

int fx_batch_choice(const fx_batch *b, int ndim, int precision, int *tile, int *ctas_per_sm) {
  if (!b || (ndim != 2 && ndim != 3) || (precision != 0 && precision != 1)) return FX_ERR_ARG;
  if (tile) *tile = b->choice[ndim - 2][precision].tile;
  if (ctas_per_sm) *ctas_per_sm = b->choice[ndim - 2][precision].ctas;
  return FX_OK;
}

}  // extern "C"

extern "C" {

const double *fx_block_fluxes(const fx_blocks *bs, int b) {
  if (!bs || b < 0 || b >= bs->nb || bs->regidx[b] < 0 || !bs->d_regs) return nullptr;
  const int nfc = bs->ndim == 3 ? bs->nxb * bs->nxb : bs->nxb;
  return bs->d_regs + (size_t)bs->regidx[b] * 2 * bs->ndim * bs->nvar * nfc;
}

}  // extern "C"
