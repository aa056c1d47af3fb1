// Measured FP64 fused-multiply-add rate of this GPU: the denominator of the
// FP64 pair kernel's roofline (its bound is the FP64 pipe, not HBM).  Not
// part of the MD interface: a separate library used by the benchmark.
//
// Each thread runs 8 independent chains of a = a * b + c (one DFMA, two
// FLOPs) for `iters` rounds; the grid fills every SM.  The result is written
// so that nothing is optimised away.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__global__ void __launch_bounds__(256) k_dfma(double *out, int iters, double b, double c) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1.0, x2 = x0 + 2.0, x3 = x0 + 3.0;
  double x4 = x0 + 4.0, x5 = x0 + 5.0, x6 = x0 + 6.0, x7 = x0 + 7.0;
  for (int k = 0; k < iters; k++) {
#pragma unroll
    for (int u = 0; u < 16; u++) {
      x0 = fma(x0, b, c); x1 = fma(x1, b, c); x2 = fma(x2, b, c); x3 = fma(x3, b, c);
      x4 = fma(x4, b, c); x5 = fma(x5, b, c); x6 = fma(x6, b, c); x7 = fma(x7, b, c);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}

}  // namespace

extern "C" {

// Launches blocks x 256 threads, each 8 x 16 x iters DFMAs, on `stream`;
// out: DEVICE double [blocks * 256].  Returns the FLOPs of the launch
// (2 per DFMA), or -1 on a launch error.
double mdrate_dfma(double *out, int32_t blocks, int32_t iters, void *stream) {
  if (!out || blocks < 1 || iters < 1) return -1.0;
  k_dfma<<<blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(out, iters, 0.999999, 1e-7);
  if (cudaGetLastError() != cudaSuccess) return -1.0;
  return 2.0 * 8.0 * 16.0 * (double)iters * (double)blocks * 256.0;
}

}  // extern "C"
