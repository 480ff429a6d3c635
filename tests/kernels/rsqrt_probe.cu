// Test harness: evaluates the library's FP64 Newton inverse square root on an
// array (compiled by the GPU test on the GPU host).
#include "../../paper_2412_12392_gb300/csrc/common.cuh"

__global__ void rsqrt_probe_kernel(const double* x, double* y, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = mslam::rsqrt_newton(x[i]);
}

extern "C" int rsqrt_probe(const double* x, double* y, int n) {
  rsqrt_probe_kernel<<<(n + 255) / 256, 256>>>(x, y, n);
  return (int)cudaDeviceSynchronize();
}
