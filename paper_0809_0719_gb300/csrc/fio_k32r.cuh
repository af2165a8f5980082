// fio_k32r.cuh -- register-tiled FP32 translations (eqs. alg2b and alg2c) for 32
// right-hand sides per CTA.
//
// One CTA owns one translation unit (A_p at level l-1, B at level L-l: four input
// pairs, four output pairs, Sec. 4) and 32 RHS; lane r of every warp is RHS r, so a
// phase factor of the unit is read by all lanes of a warp at once (a shared-memory
// broadcast) and a coefficient row of one RHS is read by one lane (the 32 lanes of a
// warp hit distinct banks: the RHS stride of q^2 complex values is 2 banks mod 32).
// Each thread keeps the q x q output block of its (output, RHS) in registers while
// it streams the input rows, so the dimension-wise Lagrange sums (the O(q^3) scheme
// of Sec. 4) run as paired FMAs (FFMA2) on registers, with T^sigma entries as
// compile-time constant-bank operands, and shared memory carries only the inputs
// and, for the x-shape, one intermediate block per input:
//
//  p-shape  out_j = post_j (.) sum_i (T^{i1} (x) T^{i2}) (pre_{j,i} (.) in_i)
//           (recursion in p, eq. alg2b; and the conjugate transpose of the recursion
//           in x).  Warp j = output j.  The 2q rows (i1, t'1) of the assembled 2q x 2q
//           input are streamed: z = row . [T^0 T^1]^T (q results), then the outer
//           product Y += T^{i1}[:, t'1] z^T.  6 q^3 FFMA2 per (output, RHS).
//  x-shape  out_j = sum_i post_{j,i} (.) (T^{j1} (x) T^{j2})^T (pre_i (.) in_i)
//           (recursion in x, eq. alg2c; and the conjugate transpose of the recursion
//           in p).  Input i at a time: pass A forms W_{j1} = T^{j1 T} along dimension 1
//           of pre_i (.) in_i for both j1 (shared by the two j2) in shared memory;
//           pass B: thread (j, r) takes each row t1 of W_{j1}, applies T^{j2 T} and
//           accumulates post_{j,i} (.) that row into its registers.
//
// Inputs are staged by the bulk-copy (TMA) engine: cp.async.bulk of each input
// block (a contiguous run of rc q^2 complex values) into shared memory, completion
// tracked by an mbarrier transaction count; every mbarrier wait is bounded in wall
// time and, on expiry, sets the plan's status word (read by fio_check) and lets the
// kernel run to its end.  Where a run is not 16-byte aligned (odd RHS counts) the
// threads copy with cp.async instead.
#pragma once
#include "fio_tc.cuh"

namespace fio {

constexpr int kRT = 32;  // RHS per CTA (one per lane)

__host__ __device__ constexpr int trans_rp_smem_bytes(int q) {
  // mbarriers | phases 20 q^2 | inputs 4 x 32 q^2 | scratch of the centre family | T transposed
  return 16 + (20 + 4 * kRT) * q * q * 8 + 1024 + (2 * q * q * 4 + 15) / 16 * 16;
}
__host__ __device__ constexpr int trans_rx_smem_bytes(int q) {
  // mbarriers | phases 20 q^2 | ring 2 x 32 q^2 | W 2 x 32 q^2
  return 16 + (20 + 4 * kRT) * q * q * 8;
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
  const uint32_t mb = (uint32_t)__cvta_generic_to_shared(mbar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes) {
  const uint32_t mb = (uint32_t)__cvta_generic_to_shared(mbar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
}
// Bulk copy of `bytes` (a multiple of 16) from global to shared memory (both
// 16-byte aligned), completing on mbar's transaction count.
__device__ __forceinline__ void bulk_g2s(void *smem, const void *gmem, uint32_t bytes, uint64_t *mbar) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  const uint32_t mb = (uint32_t)__cvta_generic_to_shared(mbar);
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sa),
               "l"(gmem), "r"(bytes), "r"(mb)
               : "memory");
}
// Bounded wait for the phase of the given parity (as tc_wait); on expiry it records
// status 2.  It does not give up early on another kernel's or CTA's status: a copy
// into this CTA's shared memory must have landed before the CTA may end.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, uint32_t parity, int *status) {
  const uint32_t mb = (uint32_t)__cvta_generic_to_shared(mbar);
  const unsigned long long t0 = globaltimer_ns();
  for (uint32_t it = 1; it < (1u << 26); it++) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mb), "r"(parity), "r"(kTcSuspendNs)
        : "memory");
    if (done) return true;
    if (globaltimer_ns() - t0 > kTcWaitNs) {
      atomicExch(status, 2);
      return false;
    }
  }
  atomicExch(status, 2);
  return false;
}

// Stage nb input blocks of rc RHS (block b from src[b], nq = rc q^2 complex values
// each) into dst + b * kRT q^2.  bulk: one thread issues nb bulk copies on mbar;
// otherwise every thread takes part in cp.async copies, which this call waits for
// (the caller's barrier then publishes them).
template <int Q>
__device__ __forceinline__ void stage_blocks(float2 *dst, const float2 *const *src, int nb, int rc, bool bulk,
                                             uint64_t *mbar) {
  constexpr int Q2 = Q * Q;
  if (bulk) {
    if (threadIdx.x == 0) {
      mbar_expect_tx(mbar, (uint32_t)(nb * rc * Q2 * 8));
      for (int b = 0; b < nb; b++) bulk_g2s(dst + b * kRT * Q2, src[b], (uint32_t)(rc * Q2 * 8), mbar);
    }
  } else {
    for (int b = 0; b < nb; b++) cp_async_run(dst + b * kRT * Q2, src[b], rc * Q2);
    cp_async_commit();
    cp_async_wait(0);
  }
}
// Wait for a stage_blocks call; ends with a barrier (cp.async path) or the mbarrier.
__device__ __forceinline__ void stage_wait(bool bulk, uint64_t *mbar, uint32_t parity, int *status) {
  if (bulk) mbar_wait_bounded(mbar, parity, status);
  else __syncthreads();
}

// acc + conj-free complex product a b (FFMA/FMUL on the FMA pipe).
__device__ __forceinline__ float2 cmac(float2 a, float2 b, float2 acc) {
  acc.x = __fmaf_rn(a.x, b.x, __fmaf_rn(-a.y, b.y, acc.x));
  acc.y = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, acc.y));
  return acc;
}

// The unit's 20 q^2 phase factors, shared by every RHS (as k32_trans_body sets them up):
//  p-shape: pre[j][i] (16 q^2) at ph_s, post[j] (4 q^2) at ph_s + 16 q^2;
//  x-shape: pre[i] (4 q^2) at ph_s, post[j][i] (16 q^2) at ph_s + 4 q^2.
// tmp: 16 q^2 float2 (the two families that are rearranged), scratch: the family's
// scratch (>= 10 q^2 df for the node family, 4 XDesc + 12 q df for the centre family).
// Ends with a barrier.
template <int Q, bool TYPE_P, bool FWD>
__device__ __forceinline__ void unit_phases(const Tables &tb, const TablesF &tf, const Phase &ph, const UnitIdx &d,
                                            int l, int lb, float2 *ph_s, float2 *tmp, unsigned char *scratch) {
  constexpr int Q2 = Q * Q;
  float2 *pre_s = ph_s;
  float2 *post_s = TYPE_P ? ph_s + 16 * Q2 : ph_s + 4 * Q2;
  if (TYPE_P && FWD) {  // pre[j=sigma][i=c] = ec[sigma][c], post[j=sigma] = conj ep[sigma]
    family_centres<Q>(tb, tf, ph, d, l, lb, pre_s, post_s, scratch);
    for (int idx = threadIdx.x; idx < 4 * Q2; idx += blockDim.x) post_s[idx] = conjf2(post_s[idx]);
  } else if (TYPE_P) {  // pre[j=c][i=sigma] = conj ea[sigma][c], post[j=c] = eq[c]
    family_nodes<Q>(tb, tf, ph, d, l, lb, tmp, post_s, scratch);
    for (int idx = threadIdx.x; idx < 16 * Q2; idx += blockDim.x) {
      const int sg = idx / (4 * Q2), c = (idx / Q2) & 3, t = idx % Q2;
      pre_s[(c * 4 + sg) * Q2 + t] = conjf2(tmp[idx]);
    }
  } else if (FWD) {  // pre[i=c] = conj eq[c], post[j=sigma][i=c] = ea[sigma][c]
    family_nodes<Q>(tb, tf, ph, d, l, lb, post_s, pre_s, scratch);
    for (int idx = threadIdx.x; idx < 4 * Q2; idx += blockDim.x) pre_s[idx] = conjf2(pre_s[idx]);
  } else {  // pre[i=sigma] = ep[sigma], post[j=c][i=sigma] = conj ec[sigma][c]
    family_centres<Q>(tb, tf, ph, d, l, lb, tmp, pre_s, scratch);
    for (int idx = threadIdx.x; idx < 16 * Q2; idx += blockDim.x) {
      const int sg = idx / (4 * Q2), c = (idx / Q2) & 3, u = idx % Q2;
      post_s[(c * 4 + sg) * Q2 + u] = conjf2(tmp[idx]);
    }
  }
  __syncthreads();
}

// Whether every input run of this launch can go through the bulk-copy engine: the
// pair stride nrhs q^2, the RHS offset and the run length must all be whole 16-byte
// multiples of complex64 values (an even number of values, q odd).
__host__ __device__ __forceinline__ bool trans_r_bulk_ok(int nrhs, int q) {
  return ((nrhs * q * q) & 1) == 0;
}

// Write the thread's q x q block (already final) into shared staging [j][r][t], then,
// after a barrier, store the four output blocks with 16-byte stores.
template <int Q, typename Dst>
__device__ __forceinline__ void store_outputs(float2 *stage, float2 (&Y)[Q][Q], int j, int r, int rc, Dst &&dst) {
  constexpr int Q2 = Q * Q;
  if (r < rc) {
#pragma unroll
    for (int t1 = 0; t1 < Q; t1++)
#pragma unroll
      for (int t2 = 0; t2 < Q; t2++) stage[(j * kRT + r) * Q2 + t1 * Q + t2] = Y[t1][t2];
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < 4; b++) store_run(dst(b), stage + b * kRT * Q2, rc * Q2);
}

// The p-shape's sweep over the 2q rows (i1, t'1) of the assembled input: for each row,
// z = row . [T^0 T^1]^T (q values), then Y += T^{i1}[.][t'1] z^T.  The rows of one i1
// run as a runtime loop over t'1 (a small loop body keeps the instruction stream in
// cache); the column T^{i1}[.][t'1] of the outer product comes from a shared copy of T
// stored transposed, tT[i1][t'1][t1] (every lane reads the same word), the entries of
// the row product are compile-time constant-bank operands.  It waits for the two halves
// of the inputs (i1 = 0, 1) as it reaches them.
template <int Q>
__device__ __forceinline__ void rp_sweep(float2 (&Y)[Q][Q], const float2 *pre, const float2 *in_s, int rr,
                                         const TMat<float, Q> &tm, const float *tT, bool bulk, uint64_t *mbar,
                                         int *status) {
  constexpr int Q2 = Q * Q;
#pragma unroll
  for (int t1 = 0; t1 < Q; t1++)
#pragma unroll
    for (int t2 = 0; t2 < Q; t2++) Y[t1][t2] = make_float2(0.f, 0.f);
#pragma unroll
  for (int i1 = 0; i1 < 2; i1++) {
    stage_wait(bulk, &mbar[i1], 0, status);
#pragma unroll 1
    for (int tp1 = 0; tp1 < Q; tp1++) {
      // z[t2] = sum_{i2, t'2} T^{i2}[t2][t'2] (pre (.) in)[i2][t'1][t'2]: the row is streamed
      // one element at a time into q independent accumulators
      float2 z[Q];
#pragma unroll
      for (int t2 = 0; t2 < Q; t2++) z[t2] = make_float2(0.f, 0.f);
#pragma unroll
      for (int i2 = 0; i2 < 2; i2++)
#pragma unroll
        for (int tp2 = 0; tp2 < Q; tp2++) {
          const int i = 2 * i1 + i2;
          const float2 sv = cmul(pre[i * Q2 + tp1 * Q + tp2], in_s[(i * kRT + rr) * Q2 + tp1 * Q + tp2]);
#pragma unroll
          for (int t2 = 0; t2 < Q; t2++) z[t2] = fma2s(tm.T[i2][t2][tp2], sv, z[t2]);
        }
      float tc[Q];
#pragma unroll
      for (int t1 = 0; t1 < Q; t1++) tc[t1] = tT[(i1 * Q + tp1) * Q + t1];
#pragma unroll
      for (int t2 = 0; t2 < Q; t2++)
#pragma unroll
        for (int t1 = 0; t1 < Q; t1++) Y[t1][t2] = fma2s(tc[t1], z[t2], Y[t1][t2]);
    }
  }
}

// ---------------------------------------------------------------------------
// p-shape (TYPE_P): FWD = recursion in p (eq. alg2b), !FWD = conjugate transpose
// of the recursion in x.  128 threads: warp j computes output j for lane r's RHS.
// ---------------------------------------------------------------------------
template <int Q, bool FWD>
__global__ void __launch_bounds__(4 * kRT, 2)
    k32_trans_rp(Tables tb, TablesF tf, Phase ph, Geom g, TMat<float, Q> tm, const float2 *__restrict__ in,
                 float2 *__restrict__ out, int *status) {
  constexpr int Q2 = Q * Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];  // bulk copies need 16-byte alignment
  uint64_t *mbar = (uint64_t *)smem_raw;                  // [2]: inputs of i1 = 0 and i1 = 1
  float2 *ph_s = (float2 *)(smem_raw + 16);               // pre [4 j][4 i][Q2] | post [4 j][Q2]
  float2 *in_s = ph_s + 20 * Q2;                          // [4 i][kRT][Q2]; output staging [4 j][kRT][Q2]
  unsigned char *small = (unsigned char *)(in_s + 4 * kRT * Q2);  // centre-family scratch (1 KB)
  float *tT = (float *)(small + 1024);  // tT[i1][t'1][t1] = T^{i1}[t1][t'1]
  for (int idx = threadIdx.x; idx < 2 * Q * Q; idx += blockDim.x) {
    const int i1 = idx / (Q * Q), tp1 = (idx / Q) % Q, t1 = idx % Q;
    tT[idx] = tm.T[i1][t1][tp1];
  }
  const int l = g.l, lb = g.L - g.l, e = g.e;
  const UnitIdx d = unit_decode(blockIdx.x, l, lb, e);
  const int r0 = blockIdx.y * kRT;
  const int rc = min(kRT, g.nrhs - r0);
  const long long nrq = (long long)g.nrhs * Q2;
  const bool bulk = trans_r_bulk_ok(g.nrhs, Q);
  auto srcp = [&](int i) {
    return in + (FWD ? pair_child_b(d, i, lb, e) : pair_child_a(d, i, l, lb, e)) * nrq + (long long)r0 * Q2;
  };
  auto dstp = [&](int i) {
    return out + (FWD ? pair_child_a(d, i, l, lb, e) : pair_child_b(d, i, lb, e)) * nrq + (long long)r0 * Q2;
  };
  if (threadIdx.x == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const float2 *src[4] = {srcp(0), srcp(1), srcp(2), srcp(3)};
  if (FWD) {  // the centre family needs little scratch: the copies overlap the phases
    stage_blocks<Q>(in_s, src, 2, rc, bulk, &mbar[0]);
    stage_blocks<Q>(in_s + 2 * kRT * Q2, src + 2, 2, rc, bulk, &mbar[1]);
    unit_phases<Q, true, FWD>(tb, tf, ph, d, l, lb, ph_s, nullptr, small);
  } else {  // the node family's scratch lives in the input area: copy afterwards
    unit_phases<Q, true, FWD>(tb, tf, ph, d, l, lb, ph_s, in_s, (unsigned char *)(in_s + 16 * Q2));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    stage_blocks<Q>(in_s, src, 2, rc, bulk, &mbar[0]);
    stage_blocks<Q>(in_s + 2 * kRT * Q2, src + 2, 2, rc, bulk, &mbar[1]);
  }
  const int j = threadIdx.x >> 5, r = threadIdx.x & 31;
  const int rr = min(r, rc - 1);  // lanes past the last RHS recompute it (results not stored)
  const float2 *pre = ph_s + j * 4 * Q2;
  float2 Y[Q][Q];
  rp_sweep<Q>(Y, pre, in_s, rr, tm, tT, bulk, mbar, status);
  const float2 *post = ph_s + 16 * Q2 + j * Q2;
#pragma unroll
  for (int t1 = 0; t1 < Q; t1++)
#pragma unroll
    for (int t2 = 0; t2 < Q; t2++) Y[t1][t2] = cmul(post[t1 * Q + t2], Y[t1][t2]);
  __syncthreads();  // every warp is done with the inputs: their area becomes the output staging
  store_outputs<Q>(in_s, Y, j, r, rc, dstp);
}

// Pass B of the x-shape for one input: acc += post (.) (W row by row times T^{j2}).
// One code path for both j2: the Chebyshev nodes are symmetric (z_{q-1-k} = -z_k), so
// l_k(-y) = l_{q-1-k}(y) and T^0[a][b] = T^1[q-1-a][q-1-b].  For j2 = 0 the thread reads
// its W row and its post factors with the t2 index reversed (rev) and applies T^1; its
// accumulator then holds the output block with t2 reversed, undone when it is stored.
template <int Q>
__device__ __forceinline__ void rx_pass_b(float2 (&acc)[Q][Q], const float2 *wrow, const float2 *post, bool rev,
                                          const TMat<float, Q> &tm) {
  const int o = rev ? Q - 1 : 0, st = rev ? -1 : 1;
#pragma unroll
  for (int t1 = 0; t1 < Q; t1++) {
    float2 v[Q];  // q independent accumulators, the W row streamed one element at a time
#pragma unroll
    for (int t2 = 0; t2 < Q; t2++) v[t2] = make_float2(0.f, 0.f);
#pragma unroll
    for (int tp2 = 0; tp2 < Q; tp2++) {
      const float2 w = wrow[t1 * Q + o + st * tp2];
#pragma unroll
      for (int t2 = 0; t2 < Q; t2++) v[t2] = fma2s(tm.T[1][tp2][t2], w, v[t2]);
    }
#pragma unroll
    for (int t2 = 0; t2 < Q; t2++) acc[t1][t2] = cmac(post[t1 * Q + o + st * t2], v[t2], acc[t1][t2]);
  }
}

// ---------------------------------------------------------------------------
// x-shape (TYPE_X): FWD = recursion in x (eq. alg2c), !FWD = conjugate transpose
// of the recursion in p.  Inputs pass through a two-slot ring (input i in slot
// i & 1), so the copy of input i+2 overlaps the work on input i+1.
// ---------------------------------------------------------------------------
template <int Q, bool FWD>
__global__ void __launch_bounds__(4 * kRT, 2)
    k32_trans_rx(Tables tb, TablesF tf, Phase ph, Geom g, TMat<float, Q> tm, const float2 *__restrict__ in,
                 float2 *__restrict__ out, int *status) {
  constexpr int Q2 = Q * Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];  // bulk copies need 16-byte alignment
  uint64_t *mbar = (uint64_t *)smem_raw;                 // [2]: ring slots
  float2 *ph_s = (float2 *)(smem_raw + 16);              // pre [4 i][Q2] | post [4 j][4 i][Q2]
  float2 *ring = ph_s + 20 * Q2;                         // [2 slot][kRT][Q2]
  float2 *W = ring + 2 * kRT * Q2;                       // [2 j1][kRT][Q2]; ring + W: output staging
  const int l = g.l, lb = g.L - g.l, e = g.e;
  const UnitIdx d = unit_decode(blockIdx.x, l, lb, e);
  const int r0 = blockIdx.y * kRT;
  const int rc = min(kRT, g.nrhs - r0);
  const long long nrq = (long long)g.nrhs * Q2;
  const bool bulk = trans_r_bulk_ok(g.nrhs, Q);
  auto srcp = [&](int i) {
    return in + (FWD ? pair_child_b(d, i, lb, e) : pair_child_a(d, i, l, lb, e)) * nrq + (long long)r0 * Q2;
  };
  auto dstp = [&](int i) {
    return out + (FWD ? pair_child_a(d, i, l, lb, e) : pair_child_b(d, i, lb, e)) * nrq + (long long)r0 * Q2;
  };
  if (threadIdx.x == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  {
    const float2 *s0 = srcp(0), *s1 = srcp(1);
    stage_blocks<Q>(ring, &s0, 1, rc, bulk, &mbar[0]);
    stage_blocks<Q>(ring + kRT * Q2, &s1, 1, rc, bulk, &mbar[1]);
  }
  // phases, with W as the families' scratch
  unit_phases<Q, false, FWD>(tb, tf, ph, d, l, lb, ph_s, W, (unsigned char *)(W + 16 * Q2));
  const float2 *pre_s = ph_s, *post_s = ph_s + 4 * Q2;
  const int j = threadIdx.x >> 5, r = threadIdx.x & 31;
  const int j1 = j >> 1, j2 = j & 1;
  const int rr = min(r, rc - 1);
  float2 acc[Q][Q];
#pragma unroll
  for (int t1 = 0; t1 < Q; t1++)
#pragma unroll
    for (int t2 = 0; t2 < Q; t2++) acc[t1][t2] = make_float2(0.f, 0.f);
#pragma unroll 1
  for (int i = 0; i < 4; i++) {
    const float2 *slot = ring + (i & 1) * kRT * Q2;
    stage_wait(bulk, &mbar[i & 1], (uint32_t)(i >> 1), status);
    // pass A: W[k1][r][t1][t'2] = sum_{t'1} T^{k1}[t'1][t1] (pre_i (.) in_i)[r][t'1][t'2],
    // task (t'2, k1) per warp, RHS per lane
    for (int c = j; c < 2 * Q; c += 4) {
      const int tp2 = c >> 1, k1 = c & 1;
      float2 a[Q];  // W[k1][r][t1][t'2] for every t1, the column streamed one element at a time
#pragma unroll
      for (int t1 = 0; t1 < Q; t1++) a[t1] = make_float2(0.f, 0.f);
      float2 *wcol = W + (k1 * kRT + r) * Q2 + tp2;
      if (k1 == 0) {
#pragma unroll
        for (int tp1 = 0; tp1 < Q; tp1++) {
          const float2 sv = cmul(pre_s[i * Q2 + tp1 * Q + tp2], slot[rr * Q2 + tp1 * Q + tp2]);
#pragma unroll
          for (int t1 = 0; t1 < Q; t1++) a[t1] = fma2s(tm.T[0][tp1][t1], sv, a[t1]);
        }
      } else {
#pragma unroll
        for (int tp1 = 0; tp1 < Q; tp1++) {
          const float2 sv = cmul(pre_s[i * Q2 + tp1 * Q + tp2], slot[rr * Q2 + tp1 * Q + tp2]);
#pragma unroll
          for (int t1 = 0; t1 < Q; t1++) a[t1] = fma2s(tm.T[1][tp1][t1], sv, a[t1]);
        }
      }
#pragma unroll
      for (int t1 = 0; t1 < Q; t1++) wcol[t1 * Q] = a[t1];
    }
    __syncthreads();  // W complete; slot i & 1 no longer read
    if (i + 2 < 4) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      const float2 *sn = srcp(i + 2);
      stage_blocks<Q>(ring + (i & 1) * kRT * Q2, &sn, 1, rc, bulk, &mbar[i & 1]);
    }
    // pass B: acc[t1][t2] += post_{j,i}[t1][t2] sum_{t'2} T^{j2}[t'2][t2] W[j1][r][t1][t'2]
    const float2 *wrow = W + (j1 * kRT + rr) * Q2;
    const float2 *post = post_s + (j * 4 + i) * Q2;
    rx_pass_b<Q>(acc, wrow, post, j2 == 0, tm);
    __syncthreads();  // W read by every warp before the next pass A rewrites it
  }
  // (j2 = 0: acc holds the block with t2 reversed)
  if (r < rc) {
    const int o = j2 == 0 ? Q - 1 : 0, st = j2 == 0 ? -1 : 1;
#pragma unroll
    for (int t1 = 0; t1 < Q; t1++)
#pragma unroll
      for (int t2 = 0; t2 < Q; t2++) ring[(j * kRT + r) * Q2 + t1 * Q + o + st * t2] = acc[t1][t2];
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < 4; b++) store_run(dstp(b), ring + b * kRT * Q2, rc * Q2);
}

}  // namespace fio
