// k_noalloc.cu -- CFL time step for callers that must not allocate device
// memory.
//
// Who needs this: code that runs where cudaMalloc is off limits -- inside a
// host callback or a custom allocator's own bookkeeping, in a process whose
// device memory is carved up by another runtime, or in a real-time loop that
// forbids allocation after start-up.  Such a caller owns its state buffer and
// its output, and cannot let the library create a block set (which allocates
// mesh tables and reduction scratch).  fx_compute_dt_noalloc gives it the same
// time step as fx_compute_dt for a single-level array of blocks, using only a
// fixed scratch array that is part of the library image.
//
// The scratch is a file-scope __device__ array: every GPU that loads libfx
// holds it (FX_NOALLOC_MAX_BLOCKS + 1 words, 256 KB + 8 B) until the process
// exits.  Host code cannot use the array's name as a device address; its
// device address is looked up once per device with cudaGetSymbolAddress the
// first time the entry point runs on that device, with that device current.
// All calls share the array, so calls that overlap on the GPU (two streams, or
// two threads) race on it; the caller must order them.
#include "../../include/fx.h"
#include "eos.cuh"
#include "fx_internal.h"

#include <atomic>
#include <cstdio>

namespace {

constexpr int kMaxDevices = 64;

// [0, FX_NOALLOC_MAX_BLOCKS): one partial maximum per block (written before it
// is read in every call); [FX_NOALLOC_MAX_BLOCKS]: count of finished CTAs
// (cleared by the host at the start of every call).
static __device__ __align__(256) unsigned long long g_dt_scratch[FX_NOALLOC_MAX_BLOCKS + 1];

std::atomic<unsigned long long *> g_scratch_ptr[kMaxDevices];

void set_msg(char *errbuf, size_t errlen, const char *msg) {
  if (errbuf && errlen) snprintf(errbuf, errlen, "%s", msg);
}

// One CTA per block: the CTA's maximum signal speed goes to partial[b]; the
// last CTA to finish takes the maximum over all partials (exact, so the order
// does not matter), writes dt and re-arms the counter.
__global__ void k_dt_noalloc(const double *__restrict__ U, int ndim, int nxb, int ng,
                             double idx0, double idx1, double idx2, double gamma, double cfl,
                             int form, double *__restrict__ dt_out,
                             unsigned long long *__restrict__ scratch) {
  const int b = blockIdx.x;
  const int P = nxb + 2 * ng, PZ = ndim == 3 ? P : 1;
  const int nz = ndim == 3 ? nxb : 1;
  const int ncell = nxb * nxb * nz;
  const long long vs = (long long)PZ * P * P;
  const double *Ub = U + (long long)b * 5 * vs;
  const double idx[3] = {idx0, idx1, idx2};
  const double gm1 = gamma - 1.0;
  double smax = 0.0;
  for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
    const int i = c % nxb, j = (c / nxb) % nxb, k = c / (nxb * nxb);
    const double *u = Ub + ((long long)(ndim == 3 ? k + ng : 0) * P + (j + ng)) * P + (i + ng);
    const double r = u[0], mx = u[vs], my = u[2 * vs], mz = u[3 * vs], E = u[4 * vs];
    const double ir = 1.0 / r;
    const double p = gm1 * (E - 0.5 * (mx * mx + my * my + mz * mz) * ir);
    const double cs = sqrt(gamma * p * ir);
    const double vel[3] = {mx * ir, my * ir, mz * ir};
    double s = 0.0;
    for (int d = 0; d < ndim; ++d) {
      const double sd = (fabs(vel[d]) + cs) * idx[d];
      s = form == 0 ? s + sd : fx::sig_max(s, sd);
    }
    smax = fx::sig_max(smax, s);  // a NaN stays: dt comes out NaN
  }
  unsigned long long bits = __double_as_longlong(smax);
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_down_sync(0xffffffffu, bits, o);
    bits = other > bits ? other : bits;
  }
  __shared__ unsigned long long wmax[32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) wmax[warp] = bits;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = wmax[w] > m ? wmax[w] : m;
    scratch[b] = m;
    __threadfence();
    const unsigned long long done = atomicAdd(&scratch[FX_NOALLOC_MAX_BLOCKS], 1ull);
    last = done == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  unsigned long long m = 0;
  for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) {
    const unsigned long long v = *((volatile unsigned long long *)&scratch[q]);
    m = v > m ? v : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_down_sync(0xffffffffu, m, o);
    m = other > m ? other : m;
  }
  __syncthreads();
  if (lane == 0) wmax[warp] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long r = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = wmax[w] > r ? wmax[w] : r;
    *dt_out = cfl / __longlong_as_double(r);
    scratch[FX_NOALLOC_MAX_BLOCKS] = 0ull;
  }
}

}  // namespace

extern "C" int fx_compute_dt_noalloc(const double *U_dev, int ndim, int nblocks, int nxb,
                                     int nguard, const double dx[3], double gamma, double cfl,
                                     int cfl_form, double *dt_dev, void *stream, char *errbuf,
                                     size_t errlen) {
  if (!U_dev || !dt_dev || !dx || (ndim != 2 && ndim != 3) || nxb < 1 || nguard < 0 ||
      !(gamma > 1.0) || !(cfl > 0.0) || (cfl_form != 0 && cfl_form != 1)) {
    set_msg(errbuf, errlen, "fx_compute_dt_noalloc: invalid argument");
    return FX_ERR_ARG;
  }
  for (int d = 0; d < ndim; ++d)
    if (!(dx[d] > 0.0)) {
      set_msg(errbuf, errlen, "fx_compute_dt_noalloc: cell widths must be positive");
      return FX_ERR_ARG;
    }
  if (nblocks < 1 || nblocks > FX_NOALLOC_MAX_BLOCKS) {
    set_msg(errbuf, errlen,
            "fx_compute_dt_noalloc: nblocks must be in [1, FX_NOALLOC_MAX_BLOCKS]; the "
            "fixed scratch holds one partial maximum per block");
    return FX_ERR_ARG;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_msg(errbuf, errlen, "fx_compute_dt_noalloc: no usable current device");
    return FX_ERR_CUDA;
  }
  unsigned long long *scratch = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!scratch) {
    // one-time set-up on this device: resolve the array's device address
    e = cudaGetSymbolAddress((void **)&scratch, g_dt_scratch);
    if (e != cudaSuccess || !scratch) {
      set_msg(errbuf, errlen, "fx_compute_dt_noalloc: cudaGetSymbolAddress of the scratch failed");
      return FX_ERR_CUDA;
    }
    g_scratch_ptr[dev].store(scratch, std::memory_order_release);
  }
  cudaStream_t s = (cudaStream_t)stream;
  // the CTA counter must start at zero; the partials are written before use
  e = cudaMemsetAsync(scratch + FX_NOALLOC_MAX_BLOCKS, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) {
    set_msg(errbuf, errlen, "fx_compute_dt_noalloc: clearing the scratch counter failed");
    return FX_ERR_CUDA;
  }
  const double idx2 = ndim == 3 ? 1.0 / dx[2] : 1.0;
  k_dt_noalloc<<<nblocks, 256, 0, s>>>(U_dev, ndim, nxb, nguard, 1.0 / dx[0], 1.0 / dx[1], idx2,
                                       gamma, cfl, cfl_form, dt_dev, scratch);
  fx::count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_msg(errbuf, errlen, "fx_compute_dt_noalloc: kernel launch failed");
    return FX_ERR_CUDA;
  }
  return FX_OK;
}
