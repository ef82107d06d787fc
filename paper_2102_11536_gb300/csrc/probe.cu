// FP64 FMA throughput probe (measurement aid for the roofline of FP64-bound
// kernels): many independent FMA chains per thread, several blocks per SM.
#include "iga_internal.h"

namespace {

template <int CH>
__global__ void k_fma_chain(double* out, int iters, double a, double b) {
  double acc[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) acc[c] = (double)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = fma(acc[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += acc[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

}  // namespace

extern "C" int iga_probe_fp64_fma(int device, double* tflops, double* sm_clock_ghz) {
  if (!tflops) return IGA_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return IGA_ECUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return IGA_ECUDA;
  const int blocks = prop.multiProcessorCount * 4, threads = 256, iters = 1 << 14, reps = 5;
  constexpr int CH = 8;
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * blocks * threads) != cudaSuccess) return IGA_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int w = 0; w < 2; ++w) k_fma_chain<CH><<<blocks, threads>>>(d, iters, 0.999, 0.001);
  cudaEventRecord(e0);
  for (int r = 0; r < reps; ++r) k_fma_chain<CH><<<blocks, threads>>>(d, iters, 0.999, 0.001);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (err != cudaSuccess || ms <= 0.0f) return IGA_ECUDA;
  const double flops = 2.0 * CH * (double)iters * blocks * threads * reps;
  *tflops = flops / (ms * 1e-3) / 1e12;
  if (sm_clock_ghz) {
    int khz = 0;
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, device);
    *sm_clock_ghz = khz / 1e6;
  }
  return IGA_OK;
}
