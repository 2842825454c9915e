// k_dword_test.cu -- element-wise kernel behind fx_dword_selftest: one
// double-word operation (dword.cuh) per element, for testing the arithmetic
// of the "f64_arith" option against FP64 and its error bounds.
#include "dword.cuh"
#include "fx_internal.h"

namespace fx {
namespace {

__global__ void k_dword_test(int op, const double *__restrict__ a, const double *__restrict__ b,
                             double *__restrict__ out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const dw x(a[i]);
  const dw y = op <= 3 || op == 7 ? dw(b[i]) : dw(0.0f, 0.0f);
  dw r;
  switch (op) {
    case 0: r = x + y; break;
    case 1: r = x - y; break;
    case 2: r = x * y; break;
    case 3: r = x / y; break;
    case 4: r = sqrt(x); break;
    case 5: r = rsqrt(x); break;
    case 6: r = x; break;
    default: r = fma(x, y, x); break;
  }
  out[i] = double(r);
}

}  // namespace

cudaError_t launch_dword_test(int op, const double *a, const double *b, double *out, int n,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_dword_test<<<(n + 255) / 256, 256, 0, s>>>(op, a, b, out, n);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fx
