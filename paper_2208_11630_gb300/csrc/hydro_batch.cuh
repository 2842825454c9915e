// hydro_batch.cuh -- the persistent batched form of the fused tile update
// and its launch helpers, shared by the FP64/FP32 instantiations
// (k_hydro.cu) and the double-word one (k_hydro_dw.cu).
//
// Paper: Flash-X (arXiv 2208.11630), Section 2 -- many block sets (requests)
// advanced by the unsplit hydro step of Section 2.2 in one launch.
#pragma once

#include "hydro_tile.cuh"

namespace fx {
namespace {

// Persistent batched kernel: the CTAs pull (request, leaf, tile) items from a
// shared counter until the list is exhausted; items of finished requests are
// skipped.  Each request brings its own mesh, buffers, dt and scratch.
template <int NDIM, int T, typename S, typename R>
__global__ void __launch_bounds__(T *T, (T == 16 ? (sizeof(R) == 4 ? 4 : 2) : 6))
k_hydro_batch(const BatchReq *__restrict__ reqs, const int4 *__restrict__ items, int nitems,
              unsigned int *__restrict__ counter) {
  __shared__ int item_s;
  for (;;) {
    if (threadIdx.x == 0) item_s = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int it = item_s;
    __syncthreads();
    if (it >= nitems) return;
    const int4 w = items[it];            // (request, block, tile, tiles per axis)
    const BatchReq &r = reqs[w.x];
    if (r.steps_left <= 0) continue;
    const int c = r.cur;
    hydro_tile<NDIM, T, S, R>(r.m, static_cast<const S *>(r.U[c]), static_cast<S *>(r.U[1 - c]),
                              w.y, w.z, w.w, *r.dt, r.regs, r.status, r.scratch + 2, r.rmask,
                              r.form);
  }
}

template <int NDIM, int T, typename S, typename R>
cudaError_t launch_batch_t(const BatchReq *reqs, const int4 *items, int nitems,
                           unsigned int *counter, int ctas_per_sm, int nsm, cudaStream_t s) {
  const size_t smem = tile_smem_bytes<NDIM, T, R>();
  auto kern = k_hydro_batch<NDIM, T, S, R>;
  static std::atomic<unsigned long long> attr_devs{0};
  if (cudaError_t e = set_smem_once((const void *)kern, smem, attr_devs); e != cudaSuccess)
    return e;
  int fit = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kern, T * T, smem);
  if (e != cudaSuccess) return e;
  int per_sm = ctas_per_sm > 0 ? (ctas_per_sm < fit ? ctas_per_sm : fit) : fit;
  if (per_sm < 1) per_sm = 1;
  int grid = per_sm * nsm;
  if (grid > nitems) grid = nitems;
  if (grid < 1) return cudaSuccess;
  kern<<<grid, T * T, smem, s>>>(reqs, items, nitems, counter);
  count_launch();
  return cudaGetLastError();
}

template <int NDIM, int T, typename S, typename R>
cudaError_t fit_t(int *fit) {
  const size_t smem = tile_smem_bytes<NDIM, T, R>();
  auto kern = k_hydro_batch<NDIM, T, S, R>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(fit, kern, T * T, smem);
}

}  // namespace
}  // namespace fx
