// batch_api.cpp -- batched, graph-replayed stepping of many block sets
// (requests): one kernel per phase over the work items of all requests,
// captured once into a CUDA graph and replayed per step, with the tile and
// CTAs-per-SM choice of the persistent update made by timing the candidates
// on the device.  A request with enough tiles to fill the GPU by itself is
// stepped by the per-block-set kernels instead (the launches of fx_step,
// with mesh and buffers as kernel parameters rather than loaded from its
// descriptor, each gated by its steps-left counter), on a branch of the
// graph beside the batched phases; its buffers alternate between steps, so
// the graph is captured twice, once per buffer parity, and the replays
// alternate.
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
constexpr int kSide = 4;   // capture streams for the updates of the large requests

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
  cudaStream_t side[kSide] = {};     // branches of the large requests' updates
  cudaEvent_t fork = nullptr, join[kSide] = {};
  cudaGraphExec_t exec[2] = {};      // the step from buffer parity 0 and from parity 1
  int phase = 0;                     // parity of the next replay (alternates if large requests)
  std::vector<int> big;              // requests updated by the per-block-set kernel
  std::vector<int> cur0;             // their current buffer when the graphs were captured
  bool dirty = true;
  int lmax = 0;
  Range rst[2][FX_MAXLEV], cpy[2], pro[2][FX_MAXLEV], rfx[2];
  std::vector<HydroGroup> groups;
  Choice choice[2][kClasses];        // [ndim - 2][compute class]
  bool tuned[2][kClasses] = {};
};

namespace {

constexpr int kMaxGroups = 8;

// Does the request fill the GPU by itself: at least one full wave of the
// per-block-set kernel's CTAs?
bool fills_gpu(const fx_batch *b, const fx_blocks *bs) {
  int fit = 0;
  if (fx::hydro_set_fit(bs->ndim, bs->nxb, compute_class(bs), &fit) != cudaSuccess || fit < 1)
    return false;
  const int tiles = bs->nxb % 16 == 0 ? bs->nxb / 16 : bs->nxb / 8;
  return (long long)bs->nleaves * tiles * tiles >= (long long)fit * b->nsm;
}

// Work lists of the batched step for the current composition.  split: leave
// the requests that fill the GPU out of the batched phases' lists and list
// them in b->big (the captured step); without it every request is in the
// lists (the tuner's timing).
int build_lists(fx_batch *b, const Choice (&ch)[2][kClasses], bool split) {
  std::vector<int4> rst[2][FX_MAXLEV], cpy[2], pro[2][FX_MAXLEV], rfx[2];
  std::map<std::tuple<int, int, int>, std::vector<int4>> hyd;
  b->lmax = 0;
  b->big.clear();
  for (int r = 0; r < b->max_req; ++r) {
    fx_blocks *bs = b->slot[r];
    if (!bs) continue;
    if (split && fills_gpu(b, bs)) {
      b->big.push_back(r);
      continue;
    }
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

#define FXB(call) do { e = (call); if (e != cudaSuccess) return e; } while (0)

// The step of a request that fills the GPU: the launches of fx_step after
// its dt (fx_guardcell_fill_amr, then fx_hydro_advance for the MUSCL-Hancock
// integrator), from buffer c into 1 - c, each kernel gated by the request's
// steps-left counter.  The signal-speed maximum was re-armed by the batch's
// begin kernel.
cudaError_t record_request(fx_batch *b, int r, int c, cudaStream_t s) {
  cudaError_t e;
  const fx_blocks *bs = b->slot[r];
  const BatchReq &q = b->h_req[r];
  const int *live = &b->d_req[r].steps_left;
  void *U = bs->U[c], *Un = bs->U[1 - c];
  FXB(fx::launch_guard_copy(bs->dm, U, bs->prec, bs->d_lists + bs->src_off, bs->nsrc,
                            fx::kHydroGuardDepth, s, live));
  for (int l = 1; l <= bs->lmax; ++l)
    FXB(fx::launch_guard_prolong_slots(bs->dm, U, bs->prec, bs->d_pslots + bs->pslot_off[l],
                                       bs->pslot_cnt[l], fx::kHydroGuardDepth, 1, s, live));
  fx::HydroStage st;
  st.dword = compute_class(bs) == 2 ? 1 : 0;
  st.live = live;
  FXB(fx::launch_hydro(bs->dm, U, Un, bs->prec, bs->d_lists + bs->leaves_off, bs->nleaves, q.dt,
                       q.regs, q.status, q.scratch + 2, q.rmask, q.form, s, st));
  if (q.reflux)
    FXB(fx::launch_reflux(bs->dm, Un, bs->prec, q.refl, q.nrefl, q.dt, q.regs, q.status,
                          q.scratch + 2, q.form, s, live));
  for (int l = bs->lmax; l >= 0; --l)
    FXB(fx::launch_restrict(bs->dm, Un, bs->prec, bs->d_lists + bs->par_off[l], bs->par_cnt[l], s,
                            live));
  return cudaSuccess;
}

// One batched step; parity 1 swaps the buffers of the large requests
// relative to b->cur0 (the other graph of the pair).
cudaError_t record_step(fx_batch *b, cudaStream_t s, int parity) {
  cudaError_t e;
  FXB(fx::launch_batch_begin(b->d_req, b->max_req, s));
  const int nside = std::min<int>(kSide, (int)b->big.size());
  if (nside > 0) {
    FXB(cudaEventRecord(b->fork, s));
    for (int j = 0; j < nside; ++j) FXB(cudaStreamWaitEvent(b->side[j], b->fork, 0));
  }
  for (size_t k = 0; k < b->big.size(); ++k)
    FXB(record_request(b, b->big[k], b->cur0[k] ^ parity, b->side[k % kSide]));
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
      FXB(fx::launch_batch_phase(fx::BATCH_RESTRICT, p, b->d_req, b->d_items + b->rst[p][l].off,
                                 b->rst[p][l].n, s));
  for (int j = 0; j < nside; ++j) {
    FXB(cudaEventRecord(b->join[j], b->side[j]));
    FXB(cudaStreamWaitEvent(s, b->join[j], 0));
  }
  FXB(fx::launch_batch_end(b->d_req, b->max_req, s));
  return cudaSuccess;
}
#undef FXB

// The coarse-fine fill of the current buffers (copies feeding prolongation,
// prolongation; parents are valid): what an update needs to read valid guards.
cudaError_t record_fill(fx_batch *b, cudaStream_t s) {
  cudaError_t e;
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

void drop_graphs(fx_batch *b) {
  for (cudaGraphExec_t &x : b->exec)
    if (x) {
      cudaGraphExecDestroy(x);
      x = nullptr;
    }
}

// Captures the batched step of the current composition (the caller has
// synchronised the stream the batch runs on).
int capture(fx_batch *b) {
  drop_graphs(b);
  int rc = build_lists(b, b->choice, true);
  if (rc) return fail(b->ctx, rc, "building the batch work lists failed");
  for (const HydroGroup &G : b->groups) {   // attributes before capture
    int fit = 0;
    cudaError_t e = fx::hydro_batch_fit(G.ndim, G.tile, G.prec, &fit);
    if (e != cudaSuccess) return cuda_fail(b->ctx, e, "batched kernel set-up");
  }
  b->cur0.assign(b->big.size(), 0);
  for (size_t k = 0; k < b->big.size(); ++k) {   // current buffers, as the device flipped them
    cudaError_t e = cudaMemcpy(&b->cur0[k], &b->d_req[b->big[k]].cur, sizeof(int),
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(b->ctx, e, "descriptor read");
  }
  const int nexec = b->big.empty() ? 1 : 2;
  for (int parity = 0; parity < nexec; ++parity) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(b->ctx, e, "begin capture");
    cudaError_t er = record_step(b, b->cap, parity);
    e = cudaStreamEndCapture(b->cap, &g);
    if (er != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      drop_graphs(b);
      return cuda_fail(b->ctx, er, "recording the batched step");
    }
    if (e != cudaSuccess) {
      drop_graphs(b);
      return cuda_fail(b->ctx, e, "end capture");
    }
    e = cudaGraphInstantiate(&b->exec[parity], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      drop_graphs(b);
      return cuda_fail(b->ctx, e, "graph instantiate");
    }
  }
  b->phase = 0;
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
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return fail(ctx, FX_ERR_OOM, "batch allocation failed");
  }
  bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int j = 0; j < kSide && ok; ++j)
    ok = cudaStreamCreateWithFlags(&b->side[j], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->join[j], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    fx_batch_destroy(b);
    cudaGetLastError();
    return fail(ctx, FX_ERR_CUDA, "batch stream set-up failed");
  }
  *out = b;
  return FX_OK;
}

int fx_batch_destroy(fx_batch *b) {
  if (!b) return FX_ERR_ARG;
  cudaDeviceSynchronize();
  for (fx_blocks *bs : b->slot)
    if (bs) bs->in_batch = 0;
  drop_graphs(b);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (int j = 0; j < kSide; ++j) {
    if (b->side[j]) cudaStreamDestroy(b->side[j]);
    if (b->join[j]) cudaEventDestroy(b->join[j]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
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
  // every batched step starts from restricted parents
  if (bs->restricted_epoch != bs->epoch) {
    for (int l = bs->lmax; l >= 0; --l)
      FX_CUDA(fx::launch_restrict(bs->dm, bs->U[bs->cur], bs->prec, bs->d_lists + bs->par_off[l],
                                  bs->par_cnt[l], st),
              "restrict launch");
    bs->restricted_epoch = bs->epoch;
  }
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
    cudaError_t e = cudaGraphLaunch(b->exec[b->phase], (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(b->ctx, e, "graph launch");
    if (b->exec[1]) b->phase ^= 1;
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
  bs->restricted_epoch = bs->epoch;  // restricted on admission and by every batched step
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
  if (build_lists(b, b->choice, false)) return fail(b->ctx, FX_ERR_OOM, "tuning work lists");
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
          if (build_lists(b, ch, false)) break;
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

int fx_batch_path(const fx_batch *b, int slot, int *path) {
  if (!b || !path || slot < 0 || slot >= b->max_req || !b->slot[slot]) return FX_ERR_ARG;
  *path = fills_gpu(b, b->slot[slot]) ? 1 : 0;
  return FX_OK;
}

int fx_batch_choice(const fx_batch *b, int ndim, int precision, int *tile, int *ctas_per_sm) {
  if (!b || (ndim != 2 && ndim != 3) || precision < 0 || precision >= kClasses) return FX_ERR_ARG;
  if (tile) *tile = b->choice[ndim - 2][precision].tile;
  if (ctas_per_sm) *ctas_per_sm = b->choice[ndim - 2][precision].ctas;
  return FX_OK;
}

}  // extern "C"
