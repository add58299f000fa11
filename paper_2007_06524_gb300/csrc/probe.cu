// Throughput probes: the denominators of the rooflines the benchmark reports.
//
// The paper has no counterpart; these are measurement aids. Both calls are
// synchronous and time their own kernel with CUDA events on the given stream.
//
//  * sq_probe_fma: every thread of a grid filled to the occupancy limit runs
//    eight independent chains a <- a * b + c (fused multiply-add) in FP64 or
//    FP32. Eight chains per thread and a full SM hide the FMA latency, so the
//    rate is the issue rate of the FMA pipe at the current clock.
//  * sq_probe_copy: dst <- src over `bytes` (16-byte vectors, grid-stride),
//    `reps` sweeps inside one launch; the rate counts 2 * bytes * reps (read + write),
//    the convention of a STREAM copy. Buffers much larger than L2 measure
//    HBM, buffers that fit in L2 measure L2 after the first pass.
#include <cuda_runtime.h>

#include "common.cuh"

namespace sq {
namespace {

constexpr int kProbeThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(T *out, int iters, T b, T c) {
  const T seed = (T)(threadIdx.x & 31) * (T)1e-3;
  T a0 = seed, a1 = seed + (T)0.1, a2 = seed + (T)0.2, a3 = seed + (T)0.3;
  T a4 = seed + (T)0.4, a5 = seed + (T)0.5, a6 = seed + (T)0.6, a7 = seed + (T)0.7;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
    a0 = fma(a0, b, c);
    a1 = fma(a1, b, c);
    a2 = fma(a2, b, c);
    a3 = fma(a3, b, c);
    a4 = fma(a4, b, c);
    a5 = fma(a5, b, c);
    a6 = fma(a6, b, c);
    a7 = fma(a7, b, c);
  }
  const T s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
  // never true for the b, c the host passes (the chains converge to c/(1-b)
  // = 1); the test keeps every chain live
  if (s == (T)-1) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_copy_probe(const float4 *__restrict__ src,
                                                              float4 *__restrict__ dst, size_t n, int reps) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int k = 0; k < reps; ++k)
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
}

template <typename T>
int fma_probe(double *tflops, float *ms_out, cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SQ_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SQ_ECUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe<T>, kProbeThreads, 0) != cudaSuccess)
    return SQ_ECUDA;
  if (per_sm < 1) per_sm = 1;
  const int blocks = sms * per_sm;
  // about 30 ms at the expected rates (FP64 ~1.2 TFLOP/s, FP32 ~80 TFLOP/s)
  const int iters = (sizeof(T) == 8) ? (1 << 13) : (1 << 18);
  T *out = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void **>(&out), sizeof(T) * blocks, s) != cudaSuccess) return SQ_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const T b = (T)0.5, c = (T)0.5;
  k_fma_probe<T><<<blocks, kProbeThreads, 0, s>>>(out, iters / 16, b, c);  // warm-up (clocks, first launch)
  cudaEventRecord(e0, s);
  k_fma_probe<T><<<blocks, kProbeThreads, 0, s>>>(out, iters, b, c);
  cudaEventRecord(e1, s);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, s);
  if (err != cudaSuccess || cudaGetLastError() != cudaSuccess) return SQ_ECUDA;
  const double flops = 2.0 * 8.0 * (double)iters * (double)blocks * kProbeThreads;
  if (tflops) *tflops = flops / (ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return SQ_OK;
}

}  // namespace
}  // namespace sq

using namespace sq;

extern "C" int sq_probe_fma(int precision, double *tflops, float *ms, sq_stream_t stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (precision == 0) return fma_probe<double>(tflops, ms, s);
  if (precision == 1) return fma_probe<float>(tflops, ms, s);
  return SQ_EINVAL;
}

extern "C" int sq_probe_copy(const void *src, void *dst, size_t bytes, int reps, double *gbps, sq_stream_t stream) {
  if (!src || !dst || bytes < 16 || (bytes & 15) || reps < 1 || reps > 10000) return SQ_EINVAL;
  if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) != 0) return SQ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SQ_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SQ_ECUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_copy_probe, kProbeThreads, 0) != cudaSuccess)
    return SQ_ECUDA;
  const size_t n = bytes / 16;
  const int blocks = sms * (per_sm > 0 ? per_sm : 1);
  const float4 *a = reinterpret_cast<const float4 *>(src);
  float4 *b = reinterpret_cast<float4 *>(dst);
  k_copy_probe<<<blocks, kProbeThreads, 0, s>>>(a, b, n, 1);  // warm-up (and fills L2 for small buffers)
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  k_copy_probe<<<blocks, kProbeThreads, 0, s>>>(a, b, n, reps);  // one launch, `reps` sweeps
  cudaEventRecord(e1, s);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess || cudaGetLastError() != cudaSuccess) return SQ_ECUDA;
  if (gbps) *gbps = 2.0 * (double)bytes * reps / (ms * 1e-3) / 1e9;
  return SQ_OK;
}
