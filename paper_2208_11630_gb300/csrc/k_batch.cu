// k_batch.cu -- the batched step: many block sets (requests) advanced
// together, every kernel reading its request's mesh, buffers and dt from a
// device-resident descriptor, so that one captured CUDA graph replays a step
// of the whole batch without host work.
//
// Order of one batched step (each phase one launch over a work list that
// spans all requests; items of requests with no steps left are skipped):
//   begin     dt = cfl / (signal-speed maximum of the current state)
//   copy      same-level guards of coarse leaves feeding a prolongation
//   prolong   guards of leaves next to a coarser leaf, level by level, one
//             CTA per (leaf, slot covered by the coarser leaf)
//   hydro     fused MUSCL-Hancock/HLLC update (k_hydro_batch, persistent)
//   reflux    fine-to-coarse flux correction                  (new buffer)
//   restrict  parents of the new state, finest level first
//   end       swap buffers, count the step
// The parents of the current state are valid at every step: a request's are
// restricted when it joins the batch, and each step ends by restricting them.
// A request that fills the GPU by itself runs the per-block-set kernels of
// these phases instead (batch_api.cpp), on a branch of the graph.
// Paper: Flash-X (arXiv 2208.11630), Section 2 (block-by-block physics update
// with Grid calls between updates); the batching across independent block
// sets is this library's GPU design, not the paper's.
#include "grid_ops.cuh"

namespace fx {
namespace {

__global__ void k_batch_begin(BatchReq *__restrict__ reqs, int n) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  BatchReq &q = reqs[r];
  if (q.steps_left <= 0) return;
  *q.dt = q.cfl / __longlong_as_double(q.scratch[2]);
  q.scratch[2] = 0ull;
}

__global__ void k_batch_end(BatchReq *__restrict__ reqs, int n) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  BatchReq &q = reqs[r];
  if (q.steps_left <= 0) return;
  q.cur = 1 - q.cur;
  q.steps_left -= 1;
}

// items: (request, parent, chunk, -); restricts the new buffer
template <typename S>
__global__ void k_batch_restrict(const BatchReq *__restrict__ reqs, const int4 *__restrict__ items) {
  const int4 w = items[blockIdx.x];
  const BatchReq &q = reqs[w.x];
  if (q.steps_left <= 0) return;
  S *U = static_cast<S *>(q.U[1 - q.cur]);
  ops::restrict_cells<S>(q.m, U, w.y, w.z);
}

// items: (request, leaf, padded z-plane, -)
template <typename S>
__global__ void k_batch_copy(const BatchReq *__restrict__ reqs, const int4 *__restrict__ items) {
  const int4 w = items[blockIdx.x];
  const BatchReq &q = reqs[w.x];
  if (q.steps_left <= 0) return;
  ops::guard_copy_plane<S>(q.m, static_cast<S *>(q.U[q.cur]), w.y, w.z, kHydroGuardDepth);
}

template <typename S>
__global__ void k_batch_prolong(const BatchReq *__restrict__ reqs, const int4 *__restrict__ items) {
  const int4 w = items[blockIdx.x];
  const BatchReq &q = reqs[w.x];
  if (q.steps_left <= 0) return;
  ops::guard_prolong_slot<S, S>(q.m, static_cast<S *>(q.U[q.cur]), w.y, w.z, kHydroGuardDepth,
                                threadIdx.x, blockDim.x);
}

// items: (request, reflux item, chunk, chunks)
template <typename S>
__global__ void k_batch_reflux(const BatchReq *__restrict__ reqs, const int4 *__restrict__ items) {
  const int4 w = items[blockIdx.x];
  const BatchReq &q = reqs[w.x];
  if (q.steps_left <= 0 || !q.reflux) return;
  __shared__ RefluxItem it;
  if (threadIdx.x == 0) it = q.refl[w.y];
  __syncthreads();
  ops::reflux_cells<S>(q.m, static_cast<S *>(q.U[1 - q.cur]), it, *q.dt, q.regs, q.status,
                       q.scratch + 2, q.form, w.z * blockDim.x + threadIdx.x, w.w * blockDim.x);
}

}  // namespace

cudaError_t launch_batch_begin(BatchReq *reqs, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_batch_begin<<<(n + 127) / 128, 128, 0, s>>>(reqs, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_batch_end(BatchReq *reqs, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_batch_end<<<(n + 127) / 128, 128, 0, s>>>(reqs, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_batch_phase(int phase, int prec, const BatchReq *reqs, const int4 *items, int n,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const bool f = prec != 0;
  switch (phase) {
    case BATCH_RESTRICT:
      if (f) k_batch_restrict<float><<<n, 256, 0, s>>>(reqs, items);
      else k_batch_restrict<double><<<n, 256, 0, s>>>(reqs, items);
      break;
    case BATCH_COPY:
      if (f) k_batch_copy<float><<<n, 256, 0, s>>>(reqs, items);
      else k_batch_copy<double><<<n, 256, 0, s>>>(reqs, items);
      break;
    case BATCH_PROLONG:
      if (f) k_batch_prolong<float><<<n, 128, 0, s>>>(reqs, items);
      else k_batch_prolong<double><<<n, 128, 0, s>>>(reqs, items);
      break;
    case BATCH_REFLUX:
      if (f) k_batch_reflux<float><<<n, 256, 0, s>>>(reqs, items);
      else k_batch_reflux<double><<<n, 256, 0, s>>>(reqs, items);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace fx
