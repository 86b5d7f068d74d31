// FP64 throughput probe: independent FMA chains on every SM.
//
// The SVD and GEMM kernels of this library are bound by the FP64 pipe, whose rate
// on GB300 is a small fraction of FP32.  This probe measures it on the device at
// hand so that roofline fractions can be read against a measured number next to
// the one derived from unit counts and clocks.
#include <cuda_runtime.h>

#include "mps_internal.h"

namespace {

__global__ void fma_chains(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
         x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

}  // namespace

extern "C" int mps_fp64_peak_probe(double* gflops, void* cuda_stream) {
  if (!gflops) return MPS_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MPS_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MPS_ECUDA;
  const int threads = 256, blocks = sms * 8, iters = 1024;
  double* out = nullptr;
  if (cudaMallocAsync(&out, sizeof(double) * blocks * threads, st) != cudaSuccess) return MPS_ENOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  mps::count_launch();
  fma_chains<<<blocks, threads, 0, st>>>(out, 16, 1.0000001, 1e-9);     // warm-up
  cudaEventRecord(e0, st);
  mps::count_launch();
  fma_chains<<<blocks, threads, 0, st>>>(out, iters, 1.0000001, 1e-9);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaFreeAsync(out, st);
  cudaStreamSynchronize(st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || ms <= 0.f) return MPS_ECUDA;
  *gflops = 2.0 * 64.0 * iters * (double)blocks * threads / (ms * 1e6);
  return MPS_OK;
}
