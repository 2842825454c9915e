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
  int device = 0;
  std::string err;
};

struct fx_blocks {
  fx_ctx *ctx = nullptr;
  int ndim = 3, nb = 0, nxb = 16, ng = 4, P = 24, PZ = 24, lmax = 0, prec = 0;
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
  std::vector<int> pro_off, pro_cnt;        // leaves with prolongation slots per level
  int src_off = 0, nsrc = 0;                // coarse leaves that feed a prolongation
  double *d_regs = nullptr;
  int nreg = 0;
  std::vector<int> regidx;
  RefluxItem *d_refl = nullptr;
  int nrefl = 0;
  unsigned long long *d_scratch = nullptr;  // [0] dt max bits, [1] CTA counter,
                                            // [2] signal-speed max of the last update
  unsigned char *d_rmask = nullptr;         // [nb] faces (bit 2d+s) the reflux corrects
  long long epoch = 0;                      // bumped on every write of the current state
  long long next_epoch = -1;                // epoch described by d_scratch[2]
  int next_form = 0;
  int *d_status = nullptr;
  double *d_dt = nullptr;                   // dt scratch for fx_run_host
  double *d_totals = nullptr;               // [nleaves][5]
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
      if (bc[2 * d + s] != FX_BC_OUTFLOW && bc[2 * d + s] != FX_BC_PERIODIC)
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
  bs->U[0] = U0;
  bs->U[1] = U1;
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
  std::vector<std::vector<int>> pro_by_level(lmax + 1);
  for (int b = 0; b < nb; ++b) {
    if (!bs->leaf[b]) continue;
    const int l = level[b];
    bool has_pro = false;
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
              g[d] = kind == FX_BC_PERIODIC ? ((g[d] % N) + N) % N : (g[d] < 0 ? 0 : N - 1);
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
            has_pro = true;
          }
          slots[27 * b + (sx + 1) + 3 * (sy + 1) + 9 * (sz + 1)] = sl;
        }
    if (has_pro) pro_by_level[l].push_back(b);
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

  // ---- work lists: leaves | parents per level | prolong leaves per level
  std::vector<int> lists;
  for (int b = 0; b < nb; ++b)
    if (bs->leaf[b]) lists.push_back(b);
  bs->leaves_off = 0;
  bs->nleaves = (int)lists.size();
  bs->par_off.assign(lmax + 1, 0);
  bs->par_cnt.assign(lmax + 1, 0);
  bs->pro_off.assign(lmax + 1, 0);
  bs->pro_cnt.assign(lmax + 1, 0);
  for (int l = 0; l <= lmax; ++l) {
    bs->par_off[l] = (int)lists.size();
    for (int b = 0; b < nb; ++b)
      if (!bs->leaf[b] && level[b] == l) lists.push_back(b);
    bs->par_cnt[l] = (int)lists.size() - bs->par_off[l];
  }
  for (int l = 0; l <= lmax; ++l) {
    bs->pro_off[l] = (int)lists.size();
    for (int b : pro_by_level[l]) lists.push_back(b);
    bs->pro_cnt[l] = (int)lists.size() - bs->pro_off[l];
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
  if ((rc = upload(bs, &bs->d_refl, refl))) return bail(rc, ctx->err);
  if (bs->nrefl > 0 && (rc = upload(bs, &bs->d_rmask, rmask))) return bail(rc, ctx->err);
  const int nfc = ndim == 3 ? n * n : n;
  if (bs->nreg > 0) {
    if (cudaMalloc(&bs->d_regs, sizeof(double) * (size_t)bs->nreg * 2 * ndim * 5 * nfc) != cudaSuccess)
      return bail(FX_ERR_OOM, "cudaMalloc of flux registers failed");
  }
  if (cudaMalloc(&bs->d_scratch, 3 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&bs->d_status, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&bs->d_dt, sizeof(double)) != cudaSuccess ||
      cudaMalloc(&bs->d_totals, sizeof(double) * 5 * (size_t)bs->nleaves) != cudaSuccess)
    return bail(FX_ERR_OOM, "cudaMalloc of scratch failed");
  if (cudaMemset(bs->d_scratch, 0, 3 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(bs->d_status, 0, sizeof(int)) != cudaSuccess)
    return bail(FX_ERR_CUDA, "cudaMemset of scratch failed");

  DevMesh &m = bs->dm;
  m.ndim = ndim; m.nxb = n; m.ng = bs->ng; m.P = bs->P; m.PZ = bs->PZ; m.nb = nb; m.lmax = lmax;
  m.vstride = (long long)bs->PZ * bs->P * bs->P;
  m.bstride = 5 * m.vstride;
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
  FX_CUDA(fx::launch_guard_copy(bs->dm, U, bs->prec, bs->d_lists + bs->leaves_off, bs->nleaves, s),
          "guard copy launch");
  for (int l = 1; l <= bs->lmax; ++l)
    FX_CUDA(fx::launch_guard_prolong(bs->dm, U, bs->prec, bs->d_lists + bs->pro_off[l],
                                     bs->pro_cnt[l], s),
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

int fx_hydro_advance(fx_ctx *ctx, fx_blocks *bs, const double *dt_dev, void *stream) {
  if (!ctx || !bs || !dt_dev) return FX_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  void *Uo = bs->U[bs->cur], *Un = bs->U[1 - bs->cur];
  unsigned long long *smax = bs->d_scratch + 2;
  const bool refl = ctx->reflux && bs->nrefl > 0;
  FX_CUDA(cudaMemsetAsync(smax, 0, sizeof(unsigned long long), s), "signal max reset");
  FX_CUDA(fx::launch_hydro(bs->dm, Uo, Un, bs->prec, bs->d_lists + bs->leaves_off, bs->nleaves,
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
static int fill_for_fused_advance(fx_ctx *ctx, fx_blocks *bs, cudaStream_t s) {
  void *U = bs->U[bs->cur];
  for (int l = bs->lmax; l >= 0; --l)
    FX_CUDA(fx::launch_restrict(bs->dm, U, bs->prec, bs->d_lists + bs->par_off[l], bs->par_cnt[l], s),
            "restrict launch");
  FX_CUDA(fx::launch_guard_copy(bs->dm, U, bs->prec, bs->d_lists + bs->src_off, bs->nsrc, s),
          "guard copy launch");
  for (int l = 1; l <= bs->lmax; ++l)
    FX_CUDA(fx::launch_guard_prolong(bs->dm, U, bs->prec, bs->d_lists + bs->pro_off[l],
                                     bs->pro_cnt[l], s),
            "guard prolong launch");
  (void)ctx;
  return FX_OK;
}

int fx_guardcell_fill_amr(fx_ctx *ctx, fx_blocks *bs, void *stream) {
  if (!ctx || !bs) return FX_ERR_ARG;
  return fill_for_fused_advance(ctx, bs, (cudaStream_t)stream);
}

int fx_step(fx_ctx *ctx, fx_blocks *bs, double cfl, double *dt_dev, void *stream) {
  int rc = fx_compute_dt(ctx, bs, cfl, dt_dev, stream);
  if (rc) return rc;
  rc = fx_guardcell_fill_amr(ctx, bs, stream);
  if (rc) return rc;
  return fx_hydro_advance(ctx, bs, dt_dev, stream);
}

int fx_conserved_totals(fx_ctx *ctx, fx_blocks *bs, double out_host[5], void *stream) {
  if (!ctx || !bs || !out_host) return FX_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  FX_CUDA(fx::launch_totals(bs->dm, bs->U[bs->cur], bs->prec, bs->d_lists + bs->leaves_off,
                            bs->nleaves, bs->d_totals, s),
          "totals launch");
  std::vector<double> h(5 * (size_t)bs->nleaves);
  FX_CUDA(cudaMemcpyAsync(h.data(), bs->d_totals, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s),
          "totals copy");
  FX_CUDA(cudaStreamSynchronize(s), "totals sync");
  for (int v = 0; v < 5; ++v) {
    double sum = 0.0, comp = 0.0;
    for (int i = 0; i < bs->nleaves; ++i) {
      double y = h[5 * (size_t)i + v] - comp;
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

long long fx_kernel_launches(void) { return fx::launch_count(); }

const double *fx_block_fluxes(const fx_blocks *bs, int b) {
  if (!bs || b < 0 || b >= bs->nb || bs->regidx[b] < 0 || !bs->d_regs) return nullptr;
  const int nfc = bs->ndim == 3 ? bs->nxb * bs->nxb : bs->nxb;
  return bs->d_regs + (size_t)bs->regidx[b] * 2 * bs->ndim * 5 * nfc;
}

}  // extern "C"
