// host_io.cpp -- entry points that take the state from host memory and return
// it there: fx_run_host (whole padded blocks) and fx_run_host_interior
// (interior cells only, packed on the device, with the upload, the CFL
// reduction, the update and the download of successive chunks overlapped on
// separate streams).
//
// Paper: Flash-X (arXiv 2208.11630), Section 2 -- the time loop advances the
// hydrodynamics on every leaf block with a step set by the CFL condition;
// these calls run that loop for a state that lives in host memory.
#include "api_state.h"

#include <cstring>

using fxapi::cuda_fail;
using fxapi::fail;

extern "C" {


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
                             bs->d_dt, bs->d_regs, bs->d_status, smax, nullptr, ctx->cfl_form, a,
                             muscl_stage(ctx, bs)),
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

}  // extern "C"
