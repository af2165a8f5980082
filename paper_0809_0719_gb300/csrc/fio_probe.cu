// fio_probe.cu -- arithmetic peak probes for the roofline denominators
// (FP32 FMA, FP64 FMA, FP32 sin/cos on the special-function unit).
// Each thread runs 8 independent dependent chains; the grid covers every SM.
#include <cuda_runtime.h>

#include <algorithm>

#include "fio.h"
#include "fio_tc.cuh"

namespace {

using namespace fio;

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

// Tensor-core MMA rate in the forms the switch uses: one CTA per SM, one thread issues
// `iters` tcgen05.mma of M = 128, N, K = 8 (TF32) or 16 (BF16) -- 32 bytes of K per row
// either way -- accumulating into one tensor-memory accumulator, the operands rotating
// over 16 K-steps (B a zeroed K-major tile in shared memory; A zeroed tensor-memory
// columns, or with ASMEM a zeroed K-major tile in shared memory), then one commit and a
// bounded wait.  The CTA takes all 512 tensor-memory columns.
constexpr int kMmaIters = 4096;
constexpr int kMmaKs = 16;  // K-steps the operands rotate over
template <bool BF16, int N, bool ASMEM, int NACC = 1>
__global__ void __launch_bounds__(128, 1) k_mma_probe(int *status) {
  extern __shared__ __align__(128) unsigned char smp[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_s;
  // [ks][rows / 8 groups][2 core columns][8 rows][4 words]: 32 bytes of K per row and K-step
  float *bsm = (float *)smp;                 // N rows
  float *asm_ = bsm + kMmaKs * N * 8;        // 128 rows (ASMEM)
  for (int i = threadIdx.x; i < kMmaKs * (N + (ASMEM ? 128 : 0)) * 8; i += blockDim.x) bsm[i] = 0.f;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_s);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(dst));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_s;
  const uint32_t acol = 256;  // A columns [256, 256 + 8 kMmaKs) after the (at most 256-column) accumulator
  {
    const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int ks = 0; ks < kMmaKs; ks++) tm_st8(tmem + acol + 8 * ks + ((uint32_t)(32 * warp) << 16), z);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (threadIdx.x == 0) {
    const uint32_t bb = (uint32_t)__cvta_generic_to_shared(bsm), ab = (uint32_t)__cvta_generic_to_shared(asm_);
    const uint32_t idesc = BF16 ? ((1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((128u >> 4) << 24))
                                : tf32_idesc<N>();
    for (int it = 0; it < kMmaIters; it++) {
      const int ks = it % kMmaKs;
      const uint32_t acc = it >= NACC ? 1u : 0u;
      const uint32_t dcol = tmem + (uint32_t)(N * (it % NACC));  // NACC accumulators in turn
      const uint64_t db = tc_desc(bb + ks * N * 32, 128, 256);
      if (ASMEM) {
        const uint64_t da = tc_desc(ab + ks * 128 * 32, 128, 256);
        if (BF16)
          asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                       "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
                       "l"(da), "l"(db), "r"(idesc), "r"(acc));
        else
          asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                       "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
                       "l"(da), "l"(db), "r"(idesc), "r"(acc));
      } else {
        const uint32_t ta = tmem + acol + 8 * ks;
        if (BF16)
          asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                       "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(dcol),
                       "r"(ta), "l"(db), "r"(idesc), "r"(acc));
        else
          asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                       "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(dcol),
                       "r"(ta), "l"(db), "r"(idesc), "r"(acc));
      }
    }
    tc_commit(&mbar);
    if (!tc_wait(&mbar, 0)) atomicExch(status, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

int mma_probe(int kind, double *per_second) {
  int dev = 0, sms = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FIO_EDEVICE;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const bool asmem = kind == 7 || kind == 8;
  const int nn = (kind == 5 || kind == 6) ? 256 : 64;
  // the rotating operands, and at least more than half an SM's shared memory: one CTA per SM
  const int smem = std::max(120 * 1024, kMmaKs * (nn + (asmem ? 128 : 0)) * 32);
  if (optin < smem) return FIO_EDEVICE;
  int *status = nullptr;
  if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) return FIO_ENOMEM;
  cudaMemset(status, 0, sizeof(int));
  const bool bf16 = kind == 4 || kind == 6 || kind == 8;
  const int n = (kind == 5 || kind == 6) ? 256 : 64;
  auto launch = [&]() {
    if (kind == 3) k_mma_probe<false, 64, false><<<sms, 128, smem>>>(status);
    if (kind == 4) k_mma_probe<true, 64, false><<<sms, 128, smem>>>(status);
    if (kind == 5) k_mma_probe<false, 256, false><<<sms, 128, smem>>>(status);
    if (kind == 6) k_mma_probe<true, 256, false><<<sms, 128, smem>>>(status);
    if (kind == 7) k_mma_probe<false, 64, true><<<sms, 128, smem>>>(status);
    if (kind == 8) k_mma_probe<true, 64, true><<<sms, 128, smem>>>(status);
    if (kind == 9) k_mma_probe<false, 64, false, 3><<<sms, 128, smem>>>(status);
    if (kind == 10) k_mma_probe<false, 64, false, 2><<<sms, 128, smem>>>(status);
  };
  cudaFuncSetAttribute(k_mma_probe<false, 64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_mma_probe<true, 64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_mma_probe<false, 256, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_mma_probe<true, 256, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_mma_probe<false, 64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_mma_probe<true, 64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_mma_probe<false, 64, false, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_mma_probe<false, 64, false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = 1e30f;
  for (int rep = 0; rep < 4; rep++) {
    cudaEventRecord(a);
    launch();
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaError_t err = cudaGetLastError();
  int st = 0;
  cudaMemcpy(&st, status, sizeof st, cudaMemcpyDeviceToHost);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(status);
  if (err != cudaSuccess) return FIO_ECUDA;
  if (st) return FIO_ETIMEOUT;
  const double k = bf16 ? 16.0 : 8.0;
  *per_second = 2.0 * 128.0 * n * k * kMmaIters * sms / (best * 1e-3);
  return FIO_OK;
}

}  // namespace

extern "C" int fio_peak_probe(int kind, double *per_second) {
  if (!per_second || kind < 0 || kind > 10) return FIO_EINVAL;
  if (kind >= 3) return mma_probe(kind, per_second);
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
