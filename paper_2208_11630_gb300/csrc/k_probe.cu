// k_probe.cu -- throughput probe of the fused multiply-add pipes (a
// measurement aid with no counterpart in the paper).
//
// The FP64 update is bound by this GPU's FP64 pipe, so its roofline needs the
// FP64 FMA rate; the benchmark measures it live with this kernel next to the
// update, under the same clocks.  Every thread runs kChains independent FMA
// chains (enough independent work per warp to cover the pipe latency) for
// `iters` iterations: 2 * kChains * iters flops per thread.  The chains
// converge to a fixed point, so no value overflows or underflows into slow
// paths; one result per CTA is written so that the work is not removed.
#include "../../include/fx.h"
#include "fx_internal.h"

namespace fx {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_probe(int iters, T *__restrict__ out) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
  const T b = T(0.999), c = T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s = s + a[k];
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

}  // namespace
}  // namespace fx

extern "C" int fx_fma_probe(int precision, int ctas, int iters, void *out_dev, void *stream,
                            double *flops) {
  if ((precision != FX_F64 && precision != FX_F32BULK) || ctas < 1 || iters < 1 || !out_dev)
    return FX_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == FX_F64)
    fx::k_fma_probe<double><<<ctas, fx::kThreads, 0, s>>>(iters, static_cast<double *>(out_dev));
  else
    fx::k_fma_probe<float><<<ctas, fx::kThreads, 0, s>>>(iters, static_cast<float *>(out_dev));
  fx::count_launch();
  if (flops) *flops = 2.0 * fx::kChains * (double)iters * (double)ctas * fx::kThreads;
  return cudaGetLastError() == cudaSuccess ? FX_OK : FX_ERR_CUDA;
}
