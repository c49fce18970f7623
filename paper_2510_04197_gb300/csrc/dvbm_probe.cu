// dvbm_probe.cu -- throughput probe of the FP64 FMA pipe (libdvbm_probe.so).
//
// Not part of the method: bench.py uses it to measure the FP64 peak that the
// step kernels' FP64 work is reported against (GB300 issues FP64 at a small
// fraction of its FP32 rate, so this pipe, not HBM, can bound the step).
// Each thread runs kChains independent FMA chains, so the pipe, not the FMA
// latency, limits the rate; the grid holds 8 blocks of 256 threads per SM.
#include <cuda_runtime.h>

namespace {
constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_dfma(double* __restrict__ out, int iters, double b, double c) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * kThreads + threadIdx.x] = s;
}
}  // namespace

// Measures FP64 FMA throughput on the current device: best of `reps` timed
// launches after one warm-up launch, CUDA events on a private stream.
// Writes FP64 flops per second (an FMA counts 2) in TFLOP/s and the best
// launch time in ms.  Returns 0, or the CUDA error code.
extern "C" int dvbm_probe_fp64_fma(int reps, double* tflops, double* best_ms) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  const int blocks = 8 * sms, iters = 4096;
  double* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&out, sizeof(double) * blocks * kThreads);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 1e30f;
  if (e == cudaSuccess) {
    k_dfma<<<blocks, kThreads, 0, st>>>(out, iters, 0.999999, 1e-6);
    e = cudaGetLastError();
  }
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    cudaEventRecord(e0, st);
    k_dfma<<<blocks, kThreads, 0, st>>>(out, iters, 0.999999, 1e-6);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms < best) best = ms;
  }
  if (e == cudaSuccess) {
    const double flops = 2.0 * kChains * (double)iters * blocks * kThreads;
    *tflops = flops / (best * 1e-3) / 1e12;
    *best_ms = best;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (out) cudaFree(out);
  return (int)e;
}
