// batch_api.cpp -- batched, graph-replayed stepping of many block sets
// (requests): one persistent kernel per phase over the work items of all
// requests, captured once into a CUDA graph and replayed per step, with the
// tile and CTAs-per-SM choice made by timing the candidates on the device.
//
// Paper: Flash-X (arXiv 2208.11630), Section 2 -- each request is a Grid of
// blocks advanced by the unsplit hydro step; a batch advances many of them
// together.
#include "api_state.h"

#include <algorithm>
#include <map>
#include <new>
#include <tuple>
#include <vector>

using fxapi::cuda_fail;
using fxapi::fail;
using fx::BatchReq;

namespace {

struct Range {
  int off = 0, n = 0;
};

struct HydroGroup {
  int ndim, tile, prec;   // prec: compute class (0 FP64, 1 FP32-bulk, 2 double-word)
  Range r;
  int ctas;   // CTAs per SM (0 = as many as fit)
};

// Tuned launch choice for one (ndim, compute class) group of block sets
// whose nxb allows 16x16 tiles: the tile edge and the CTAs per SM.
struct Choice {
  int tile = 16;
  int ctas = 0;
};

// (ndim, compute class, SM count, mask of the 16-capable block edges in the group)
std::map<std::tuple<int, int, int, int>, Choice> g_tune_cache;

constexpr int kClasses = 3;

// Compute class of a block set's update: its precision, or 2 for an FP64 set
// whose context asks for double-word arithmetic.
int compute_class(const fx_blocks *bs) {
  return bs->prec == 0 && bs->ctx->f64_arith == 1 ? 2 : bs->prec;
}

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
  Choice choice[2][kClasses];        // [ndim - 2][compute class]
  bool tuned[2][kClasses] = {};
};

namespace {

constexpr int kMaxGroups = 8;

// Work lists of the batched step for the current composition.
int build_lists(fx_batch *b, const Choice (&ch)[2][kClasses]) {
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
    const int hc = compute_class(bs);
    const int T = (n % 16 == 0) ? ch[nd - 2][hc].tile : 8;
    const int tiles = n / T;
    auto &H = hyd[std::make_tuple(nd, T, hc)];
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
  if (bs->prec == 0 && bs->ctx->f64_arith == 2)
    return fail(b->ctx, FX_ERR_ARG, "FP32 arithmetic on FP64 state (f64_arith = 2) is not batched");
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
    for (int pr = 0; pr < kClasses; ++pr) {
      // is there a group of 16-capable block sets of this kind?
      int mask = 0;
      for (fx_blocks *bs : b->slot)
        if (bs && bs->ndim == nd && compute_class(bs) == pr && bs->nxb % 16 == 0)
          mask |= 1 << (bs->nxb / 16);
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
          Choice ch[2][kClasses];
          for (int a = 0; a < 2; ++a)
            for (int c = 0; c < kClasses; ++c) ch[a][c] = b->choice[a][c];
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
  if (!b || (ndim != 2 && ndim != 3) || precision < 0 || precision >= kClasses) return FX_ERR_ARG;
  if (tile) *tile = b->choice[ndim - 2][precision].tile;
  if (ctas_per_sm) *ctas_per_sm = b->choice[ndim - 2][precision].ctas;
  return FX_OK;
}

}  // extern "C"
