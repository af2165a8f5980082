// fio_probe.cu -- arithmetic peak probes for the roofline denominators
// (FP32 FMA, FP64 FMA, FP32 sin/cos on the special-function unit).
// Each thread runs 8 independent dependent chains; the grid covers every SM.
#include <cuda_runtime.h>

#include "fio.h"

namespace {

constexpr int kIters = 4096;

template <typename R> __global__ void k_fma(R *sink, R a, R b) {
  R x[8];
#pragma unroll
  for (int i = 0; i < 8; i++) x[i] = (R)(threadIdx.x + i);
  for (int it = 0; it < kIters; it++) {
#pragma unroll
    for (int i = 0; i < 8; i++) x[i] = x[i] * a + b;
  }
  R s = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) s += x[i];
  if (s == (R)1234.5) sink[0] = s;
}

__global__ void k_sfu(float *sink, float a) {
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; i++) x[i] = 0.001f * (threadIdx.x + i);
  for (int it = 0; it < kIters / 4; it++) {
#pragma unroll
    for (int i = 0; i < 8; i++) x[i] = __sinf(x[i]) * a;
  }
  float s = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) s += x[i];
  if (s == 1234.5f) sink[0] = s;
}

}  // namespace

extern "C" int fio_peak_probe(int kind, double *per_second) {
  if (!per_second || kind < 0 || kind > 2) return FIO_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FIO_EDEVICE;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  void *sink = nullptr;
  if (cudaMalloc(&sink, 64) != cudaSuccess) return FIO_ENOMEM;
  const int threads = 256, blocks = sms * 8;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = 1e30f;
  for (int rep = 0; rep < 4; rep++) {
    cudaEventRecord(a);
    if (kind == 0) k_fma<float><<<blocks, threads>>>((float *)sink, 0.999f, 0.001f);
    if (kind == 1) k_fma<double><<<blocks, threads>>>((double *)sink, 0.999, 0.001);
    if (kind == 2) k_sfu<<<blocks, threads>>>((float *)sink, 0.999f);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  if (err != cudaSuccess) return FIO_ECUDA;
  const double ops = (double)blocks * threads * 8.0 * (kind == 2 ? kIters / 4 : kIters);
  *per_second = (kind == 2 ? ops : 2.0 * ops) / (best * 1e-3);
  return FIO_OK;
}
