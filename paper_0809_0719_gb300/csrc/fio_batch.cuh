// fio_batch.cuh -- persistent kernels that run one butterfly step for many
// FP32 plans of one q in a single launch (fio_batch_* in include/fio.h).
//
// A batched launch covers a list of work items, one per plan taking part in the
// step; item i owns the work indices [start[i], start[i+1]) (its units times its
// RHS tiles).  Each CTA walks the index space with stride gridDim.x, copies the
// descriptor of the item it is in to shared memory when the item changes, and
// runs the same per-unit body as the single-plan FP32 kernels (fio_k32.cuh), so
// a plan gives bit-identical results alone or in a batch.  The plans may differ
// in N, phase, number of right-hand sides and truncation; q (which fixes the
// translation matrices T, Sec. 4) and s (which fixes the termination matrix V)
// are shared by the launch.
#pragma once
#include "fio_run.cuh"

namespace fio {

// One plan's share of one batched launch (plain data, copied to the device).
struct BWork {
  Tables tb;
  TablesF tf;
  Phase ph;
  Geom g;
  const float2 *in;  // state read by the step (NULL where the packed user buffer is read)
  float2 *out;       // state written by the step (NULL where the packed user buffer is written)
  long long io_off;  // the plan's element offset in the packed user buffers
  int nrt;           // RHS tiles of kRMax per unit
  int maxsrc, GA;    // initialization only: sources per box, boxes A per pass
  int plan;          // the plan's index in the batch
};
// The user buffers of the current apply, written by a small kernel ahead of each
// graph launch so that the captured graph needs no new pointers: either one packed
// buffer per direction (pin, pout NULL; plan i at element io_off), or one pointer per
// plan (pin[i], pout[i]: fio_apply_batch).
struct BIo {
  const float2 *in;
  float2 *out;
  const float2 *const *pin;
  float2 *const *pout;
};
__device__ __forceinline__ const float2 *io_in(const BIo *io, const BWork &w) {
  return io->pin ? io->pin[w.plan] : io->in + w.io_off;
}
__device__ __forceinline__ float2 *io_out(const BIo *io, const BWork &w) {
  return io->pout ? io->pout[w.plan] : io->out + w.io_off;
}

// Item holding work index w: the largest i with start[i] <= w.
__device__ __forceinline__ int batch_find(const long long *__restrict__ start, int n, long long w) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= w) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Persistent walk over the work indices; body(unit, rhs_tile) sees the item in w_s.
template <typename F>
__device__ __forceinline__ void batch_loop(const BWork *__restrict__ items, const long long *__restrict__ start, int n,
                                           BWork &w_s, F &&body) {
  const long long total = start[n];
  int cur = -1;
  for (long long w = blockIdx.x; w < total; w += gridDim.x) {
    const int i = batch_find(start, n, w);
    __syncthreads();  // the previous unit is done with shared memory
    if (i != cur) {
      const int *src = (const int *)(items + i);
      int *dst = (int *)&w_s;
      for (int k = threadIdx.x; k < (int)(sizeof(BWork) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
      cur = i;
      __syncthreads();
    }
    const long long loc = w - start[i];
    body(loc / w_s.nrt, (int)(loc % w_s.nrt));
  }
}

template <int Q, bool TYPE_P, bool FWD, int RS>
__global__ void __launch_bounds__(TransShape<Q, RS>::threads, TransShape<Q, RS>::min_blocks)
    kb_trans(const BWork *__restrict__ items, const long long *__restrict__ start, int n, TMat<float, Q> tm) {
  __shared__ BWork w_s;
  batch_loop(items, start, n, w_s, [&](long long unit, int ry) {
    k32_trans_body<Q, TYPE_P, FWD, RS>(w_s.tb, w_s.tf, w_s.ph, w_s.g, tm, w_s.in, w_s.out, unit, ry);
  });
}

template <int Q, bool FWD>
__global__ void __launch_bounds__(SwShape<Q>::threads, 2) kb_switch(const BWork *__restrict__ items, const long long *__restrict__ start,
                                                 int n) {
  __shared__ BWork w_s;
  batch_loop(items, start, n, w_s, [&](long long unit, int ry) {
    k32_switch_body<Q, FWD>(w_s.tb, w_s.tf, w_s.ph, w_s.g, w_s.in, w_s.out, unit, ry);
  });
}

template <int Q>
__global__ void __launch_bounds__(InitShape<Q>::threads) kb_init(const BWork *__restrict__ items,
                                                                  const long long *__restrict__ start, int n,
                                                                  const BIo *__restrict__ io) {
  __shared__ BWork w_s;
  batch_loop(items, start, n, w_s, [&](long long unit, int ry) {
    k32_init_body<Q>(w_s.tb, w_s.tf, w_s.ph, w_s.g, w_s.maxsrc, w_s.GA, io_in(io, w_s), w_s.out, unit, ry);
  });
}

template <int Q>
__global__ void __launch_bounds__(256) kb_init_adj(const BWork *__restrict__ items, const long long *__restrict__ start,
                                                   int n, const BIo *__restrict__ io) {
  __shared__ BWork w_s;
  batch_loop(items, start, n, w_s, [&](long long unit, int ry) {
    k32_init_adj_body<Q>(w_s.tb, w_s.tf, w_s.ph, w_s.g, w_s.maxsrc, w_s.in, io_out(io, w_s), unit, ry);
  });
}

template <int Q>
__global__ void __launch_bounds__(32 * (Q > kTermM ? Q : kTermM)) kb_term(const BWork *__restrict__ items,
                                                                         const long long *__restrict__ start, int n,
                                                                         VMat<float, Q> vm, const BIo *__restrict__ io) {
  __shared__ BWork w_s;
  batch_loop(items, start, n, w_s, [&](long long unit, int ry) {
    k32_term_body<Q>(w_s.tb, w_s.tf, w_s.ph, w_s.g, vm, w_s.in, io_out(io, w_s), unit, ry);
  });
}

template <int Q>
__global__ void __launch_bounds__(32 * (Q > kTermM ? Q : kTermM)) kb_term_adj(const BWork *__restrict__ items,
                                                                             const long long *__restrict__ start, int n,
                                                                             VMat<float, Q> vm,
                                                                             const BIo *__restrict__ io) {
  __shared__ BWork w_s;
  batch_loop(items, start, n, w_s, [&](long long unit, int ry) {
    k32_term_adj_body<Q>(w_s.tb, w_s.tf, w_s.ph, w_s.g, vm, io_in(io, w_s), w_s.out, unit, ry);
  });
}

// One batched launch as the host schedules it.
struct BLaunch {
  int kind;                 // KernelKind (K_INIT ... K_INIT_ADJ)
  int q, s;
  const BWork *items;       // device
  const long long *start;   // device, n + 1 entries
  int n;
  long long total;          // start[n]
  int smem;                 // dynamic shared memory bytes (max over the items)
  int grid;                 // CTAs (persistent: a multiple of the SM count, at most total)
  int rs;                   // translations: RHS per subtile (4 or 8)
  const BIo *io;            // device
  const double (*T)[kQMax][kQMax];  // host: T[2][q][q] of a plan of this q
  const double (*V)[kQMax];         // host: V[kMMax][q] of a plan of this s
};

constexpr int kBatchBlockInit = 256;

// Launch L on st, or (blocks_per_sm != NULL) set the kernel's shared-memory limit
// and report its occupancy at L.smem instead.  Returns a cudaError_t.
template <int Q> int batch_launch(const BLaunch &L, cudaStream_t st, int smem_optin, int *blocks_per_sm, int *block) {
  TMat<float, Q> tm;
  for (int a = 0; a < 2; a++)
    for (int i = 0; i < Q; i++)
      for (int j = 0; j < Q; j++) tm.T[a][i][j] = (float)L.T[a][i][j];
  VMat<float, Q> vm;
  for (int m = 0; m < kMMax; m++)
    for (int j = 0; j < Q; j++) vm.V[m][j] = (float)L.V[m][j];
  auto go = [&](auto kernel, int threads, auto... args) -> int {
    if (block) *block = threads;
    if (blocks_per_sm) {
      // the dynamic limit leaves room for the kernel's static shared memory (the item copy)
      cudaFuncAttributes fa;
      cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
      if (e != cudaSuccess) return (int)e;
      const int maxdyn = smem_optin - (int)fa.sharedSizeBytes;
      if (L.smem > maxdyn) return (int)cudaErrorInvalidConfiguration;
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, maxdyn);
      if (e != cudaSuccess) return (int)e;
      return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kernel, threads, L.smem);
    }
    kernel<<<L.grid, threads, L.smem, st>>>(args...);
    return (int)cudaGetLastError();
  };
  constexpr int tterm = 32 * (Q > kTermM ? Q : kTermM);
  switch (L.kind) {
  case K_INIT: return go(kb_init<Q>, InitShape<Q>::threads, L.items, L.start, L.n, L.io);
  case K_TRANS_P:
    return L.rs == 4 ? go(kb_trans<Q, true, true, 4>, TransShape<Q, 4>::threads, L.items, L.start, L.n, tm)
                     : go(kb_trans<Q, true, true, 8>, TransShape<Q, 8>::threads, L.items, L.start, L.n, tm);
  case K_SWITCH: return go(kb_switch<Q, true>, SwShape<Q>::threads, L.items, L.start, L.n);
  case K_TRANS_X:
    return L.rs == 4 ? go(kb_trans<Q, false, true, 4>, TransShape<Q, 4>::threads, L.items, L.start, L.n, tm)
                     : go(kb_trans<Q, false, true, 8>, TransShape<Q, 8>::threads, L.items, L.start, L.n, tm);
  case K_TERM: return go(kb_term<Q>, tterm, L.items, L.start, L.n, vm, L.io);
  case K_TERM_ADJ: return go(kb_term_adj<Q>, tterm, L.items, L.start, L.n, vm, L.io);
  case K_TRANS_P_ADJ:
    return L.rs == 4 ? go(kb_trans<Q, true, false, 4>, TransShape<Q, 4>::threads, L.items, L.start, L.n, tm)
                     : go(kb_trans<Q, true, false, 8>, TransShape<Q, 8>::threads, L.items, L.start, L.n, tm);
  case K_SWITCH_ADJ: return go(kb_switch<Q, false>, SwShape<Q>::threads, L.items, L.start, L.n);
  case K_TRANS_X_ADJ:
    return L.rs == 4 ? go(kb_trans<Q, false, false, 4>, TransShape<Q, 4>::threads, L.items, L.start, L.n, tm)
                     : go(kb_trans<Q, false, false, 8>, TransShape<Q, 8>::threads, L.items, L.start, L.n, tm);
  case K_INIT_ADJ: return go(kb_init_adj<Q>, kBatchBlockInit, L.items, L.start, L.n, L.io);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace fio
