// fio_tc.cuh -- the FP32 form's switch (eq. alg2m) on the 5th-generation tensor
// cores: tcgen05.mma kind::tf32 with the FP32 accumulator in tensor memory, as an
// error-compensated split-TF32 product.  Two kernels: k32_switch_tc (both operands
// staged in shared memory) and k32_switch_tm (the kernel matrix written straight to
// tensor memory by the threads that compute it; the faster one at q = 9).
//
// Per pair (A, B) the switch is the complex product OUT[t][r] = sum_s K[t][s] IN[s][r]
// (q^2 x q^2 kernel, up to 32 RHS).  It is posed as ONE real GEMM D = A B with
//   A[t][2s] = Re K[t][s],  A[t][2s+1] = Im K[t][s]                    (M = q^2 -> 128 rows)
//   B[2s][n] = Re IN[s][n], B[2s][32+n] = Im IN[s][n],
//   B[2s+1][n] = -Im IN[s][n], B[2s+1][32+n] = Re IN[s][n]              (K = 2q^2 -> mult. of 8, N = 64)
// so that D[t][n] = Re OUT[t][n] and D[t][32+n] = Im OUT[t][n].
//
// Precision: B (the coefficients) is split into three TF32 parts (33 bits) and
// A (the kernel) into two (22 bits); D keeps A0B0 + A0B1 + A1B0 + A0B2 + A1B1.
// The dropped terms are ~2^-33 relative.  The two-part kernel is a perturbation of
// K of ~2^-22 that the forward and the adjoint switch share exactly (the adjoint
// uses the conjugate transpose of the same parts), so it stays far below the
// method's error and does not show in the dot test; a two-part B would (~2^-22
// between forward and adjoint).
//
// Warp-specialised pipeline (a tcgen05.mma of this shape occupies the tensor core
// for ~95 cycles and blocks its issuing thread that long): 8 producer warps
// generate both operands in chunks of 16 K-columns into two shared buffers -- A
// from the phases (double-float theta, reduced exactly, then the SFU sine and
// cosine), B from the coefficients staged in shared memory (the next pair's are
// copied asynchronously) -- and signal "full"; one MMA warp waits for a full chunk,
// issues its MMAs and commits them to the chunk's "free" barrier.  Two TMEM
// accumulators alternate between pairs so that the epilogue of a pair overlaps the
// MMAs of the next.  Shared operands use the K-major layout
// without swizzle: 8-row x 16-byte core matrices, consecutive along K
// (LBO = 128 B), 8-row groups SBO bytes apart.  Every mbarrier wait is bounded;
// on expiry the kernel records status 1, stops issuing work, and still waits
// (bounded) for its MMAs before freeing its tensor memory.
#pragma once
#include <type_traits>

#include "fio_k32.cuh"

namespace fio {

constexpr int kTcProducers = 256;               // 8 producer warps
constexpr int kTcThreads = kTcProducers + 32;   // + 1 MMA warp
constexpr int kTcKC = 16;                       // K columns per chunk (2 MMA K-steps)
constexpr int kTcPA = 2, kTcPB = 3;             // TF32 parts of A (kernel) and B (coefficients)
constexpr unsigned long long kTcWaitNs = 2000000000ULL;  // bound of one mbarrier wait (2 s)
constexpr uint32_t kTcSuspendNs = 1000000;               // suspend-time hint of one try_wait (1 ms)

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the 5th-generation tensor core; no swizzle
  return d;
}
// D f32, A and B tf32, both K-major, N = 64, M = 128.
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

// Compile-time loop f(integral_constant<0>) .. f(integral_constant<N-1>), and a dispatch of
// a runtime v in [0, N) to f(integral_constant<v>).
template <int N, int I = 0, typename F> __device__ __forceinline__ void static_for(F &&f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<N, I + 1>(f);
  }
}
template <int N, int I = 0, typename F> __device__ __forceinline__ void static_switch(int v, F &&f) {
  if constexpr (I < N) {
    if (v == I) f(std::integral_constant<int, I>{});
    else static_switch<N, I + 1>(v, f);
  }
}

// Round a finite FP32 value to TF32 (10 stored mantissa bits), to nearest with ties away
// from zero: add half a TF32 unit to the magnitude bits and clear the 13 low bits (a
// carry into the exponent is the correct round-up).  Two integer operations.
__device__ __forceinline__ float tf32_rna(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
// x = p0 + p1 (+ p2) with p0, p1 rounded to TF32; the residual is ~2^-22 |x|.  With three
// parts p2 is the exact remainder in FP32: the tensor core reads its leading TF32 bits
// (truncation), so what it drops is ~2^-32 |x|.
template <int P> __device__ __forceinline__ void tf32_split(float x, float *p) {
  p[0] = tf32_rna(x);
  float r = x - p[0];
  p[1] = tf32_rna(r);
  if (P > 2) p[2] = r - p[1];
}
__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(kTcIdesc), "r"(acc));
}
__device__ __forceinline__ void tc_commit(uint64_t *mbar) {
  const uint32_t mb = (uint32_t)__cvta_generic_to_shared(mbar);
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb) : "memory");
}
// Bounded wait for the completion of the mbarrier phase with the given parity:
// mbarrier.try_wait suspends the thread in hardware until the phase completes or
// the suspend-time hint passes, so the loop neither spins on the issue slots nor
// sleeps past the completion; the bound is wall time.
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool tc_wait(uint64_t *mbar, uint32_t parity, unsigned long long limit_ns = kTcWaitNs) {
  const uint32_t mb = (uint32_t)__cvta_generic_to_shared(mbar);
  const unsigned long long t0 = globaltimer_ns();
  if (limit_ns < kTcSuspendNs) {
    // short limits (tests of the failure path): non-blocking polls, so the limit is exact
    for (uint32_t it = 1; it < (1u << 26); it++) {
      uint32_t done;
      asm volatile(
          "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(mb), "r"(parity)
          : "memory");
      if (done) return true;
      if (globaltimer_ns() - t0 > limit_ns) return false;
    }
    return false;
  }
  for (uint32_t it = 1; it < (1u << 26); it++) {  // the wall-time bound normally ends it first
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mb), "r"(parity), "r"(kTcSuspendNs)
        : "memory");
    if (done) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
  return false;
}
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 16; c++) v[c] = __uint_as_float(r[c]);
}

template <int Q> struct TcShape {
  static constexpr int Q2 = Q * Q;
  static constexpr int KP = ((2 * Q2 + 7) / 8) * 8;                  // padded K (multiple of the MMA K-step)
  static constexpr int NCH = (KP + kTcKC - 1) / kTcKC;                // chunks per pair (the last may be partial)
  static constexpr int A_FLOATS = 128 * kTcKC;                        // one part of one A chunk
  static constexpr int B_FLOATS = 64 * kTcKC;                         // one part of one B chunk
  static constexpr size_t smem_bytes() {
    return (size_t)(2 * kTcPA * A_FLOATS + 2 * kTcPB * B_FLOATS) * 4 + (size_t)2 * kRMax * Q2 * 8 +
           (size_t)Q2 * sizeof(XDesc) + (size_t)(Q2 * Q + Q) * sizeof(df) + 9 * 8 + 16;
  }
};

// Named barrier among the producer warps only.
__device__ __forceinline__ void producers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kTcProducers) : "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
  const uint32_t mb = (uint32_t)__cvta_generic_to_shared(mbar);
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mb) : "memory");
}

template <int Q, bool FWD>
__global__ void __launch_bounds__(kTcThreads, 2) k32_switch_tc(Tables tb, TablesF tf, Phase ph, Geom g,
                                                                const float2 *__restrict__ in,
                                                                float2 *__restrict__ out, int *status) {
  typedef TcShape<Q> S;
  constexpr int Q2 = S::Q2, KP = S::KP, NCH = S::NCH;
  extern __shared__ __align__(16) unsigned char smem_raw[];  // no-swizzle operands need 16-byte alignment
  float *as = (float *)smem_raw;                   // A [part][buffer][16 row groups][kTcKC/4][8][4]
  float *bs = as + 2 * kTcPA * S::A_FLOATS;        // B [part][buffer][8 col groups][kTcKC/4][8][4]
  float2 *instage = (float2 *)(bs + 2 * kTcPB * S::B_FLOATS);  // [2][kRMax][Q2] coefficients
  XDesc *xd = (XDesc *)(instage + 2 * kRMax * Q2);  // [Q2]
  df *gt = (df *)(xd + Q2);                         // [Q2][Q]
  df *rho_s = gt + Q2 * Q;                          // [Q] rho of the p1 nodes of B
  uint64_t *full = (uint64_t *)(rho_s + Q);         // [2] producers -> MMA warp: chunk buffer written
  uint64_t *fre = full + 2;                         // [2] MMA commit -> producers: chunk buffer read
  uint64_t *dfull = fre + 2;                        // [2] MMA commit -> producers: accumulator complete
  uint64_t *dempty = dfull + 2;                     // [2] producers -> MMA warp: accumulator read out
  uint64_t *fin = dempty + 2;                       // [1] final drain of the MMA warp
  uint32_t *tmem_s = (uint32_t *)(fin + 1);
  volatile int *abort_s = (volatile int *)(tmem_s + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int l = g.l, lb = g.L - g.l, e = g.e;
  const int nb2 = 1 << (lb + e);
  const long long nBl = (1LL << lb) * nb2;
  const int r0 = blockIdx.y * kRMax;
  const int rc = min(kRMax, g.nrhs - r0);
  const long long nrq = (long long)g.nrhs * Q2;
  const bool sep = ph.id == 3;

  for (int i = tid; i < 2 * kTcPA * S::A_FLOATS + 2 * kTcPB * S::B_FLOATS; i += blockDim.x) as[i] = 0.f;
  if (tid == 0) {
    for (int b = 0; b < 9; b++) {  // full, fre, dfull, dempty, fin
      const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&full[b]);
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_s = 0;
  }
  if (warp == 0) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(tmem_s);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(dst));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_s;
  // waits: bounded; on expiry record the status, raise the abort flag, report failure
  auto waitp = [&](uint64_t *mb, uint32_t parity) {
    if (*abort_s) return false;
    if (tc_wait(mb, parity)) return true;
    atomicExch(status, 1);
    *abort_s = 1;
    return false;
  };

  if (warp == kTcProducers / 32) {
    // ------------------------------------------------------------ MMA warp
    const uint32_t aA = (uint32_t)__cvta_generic_to_shared(as);
    const uint32_t aB = (uint32_t)__cvta_generic_to_shared(bs);
    uint32_t fullph[2] = {0, 0}, demph[2] = {0, 0};
    int np = 0;  // pairs issued
    for (long long pr = blockIdx.x; pr < g.nunits; pr += gridDim.x, np++) {
      const int dsel = np & 1;
      if (np >= 2 && !waitp(&dempty[dsel], demph[dsel]++ & 1)) break;  // accumulator dsel read out
      const uint32_t dtm = tmem + 64 * dsel;
      bool live = true;
      for (int c = 0; c < NCH && live; c++) {
        const int b = c & 1;
        if (!waitp(&full[b], fullph[b]++ & 1)) { live = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int kcols = min(kTcKC, KP - c * kTcKC);
        if (lane == 0) {
          constexpr uint32_t sbo = (kTcKC / 4) * 128;
          for (int ks = 0; ks < kcols / 8; ks++) {
            uint64_t dA[kTcPA], dB[kTcPB];
#pragma unroll
            for (int q_ = 0; q_ < kTcPA; q_++) dA[q_] = tc_desc(aA + ((2 * q_ + b) * S::A_FLOATS) * 4 + ks * 256, 128, sbo);
#pragma unroll
            for (int q_ = 0; q_ < kTcPB; q_++) dB[q_] = tc_desc(aB + ((2 * q_ + b) * S::B_FLOATS) * 4 + ks * 256, 128, sbo);
            tc_mma(dtm, dA[0], dB[0], (c > 0 || ks > 0) ? 1u : 0u);
            tc_mma(dtm, dA[0], dB[1], 1u);
            tc_mma(dtm, dA[1], dB[0], 1u);
            tc_mma(dtm, dA[0], dB[2], 1u);
            tc_mma(dtm, dA[1], dB[1], 1u);
          }
          tc_commit(&fre[b]);                           // chunk buffer may be rewritten
          if (c == NCH - 1) tc_commit(&dfull[dsel]);    // accumulator complete
        }
        __syncwarp();
      }
      if (!live) break;
    }
    // drain: wait (bounded) until every MMA this warp issued has completed
    if (lane == 0) tc_commit(fin);
    __syncwarp();
    if (!tc_wait(fin, 0)) atomicExch(status, 1);
  } else {
    // ------------------------------------------------------------ producer warps
    uint32_t freeph[2] = {0, 0}, dfph[2] = {0, 0};
    uint32_t issued[2] = {0, 0};  // chunks handed to each buffer
    auto prefetch = [&](long long pr, int slot) {
      if (pr < g.nunits)
        for (int k = tid; k < rc * Q2; k += kTcProducers)
          cp_async8(instage + slot * kRMax * Q2 + k, in + pr * nrq + (long long)r0 * Q2 + k);
      cp_async_commit();
    };
    prefetch(blockIdx.x, 0);
    int np = 0;
    bool live = true;
    for (long long pr = blockIdx.x; pr < g.nunits && live; pr += gridDim.x, np++) {
      const int slot = np & 1, dsel = np & 1;
      const float2 *ins = instage + slot * kRMax * Q2;
      const long long a = pr / nBl, bidx = pr - a * nBl;
      const int a1 = (int)(a >> l), a2 = (int)(a & ((1LL << l) - 1));
      const int b1 = (int)(bidx / nb2), b2 = (int)(bidx - (long long)b1 * nb2);
      if (!sep) {
        for (int t = tid; t < Q2; t += kTcProducers)
          xd[t] = xdesc(tf.ph, xnf(tb, tf, l, a1, t / Q, Q), xnf(tb, tf, l, a2, t % Q, Q));
        if (tid < Q) rho_s[tid] = rhof(tb, tf, lb, b1, tid, Q);
      }
      producers_sync();  // xd ready; the previous pair's chunks are all generated
      prefetch(pr + gridDim.x, slot ^ 1);
      if (!sep)
        for (int idx = tid; idx < Q2 * Q; idx += kTcProducers)
          gt[idx] = g_eval(tf.ph, xd[idx / Q], p2f(tb, tf, lb, b2, idx % Q, Q));
      cp_async_wait(1);
      producers_sync();
      for (int c = 0; c < NCH; c++) {
        const int b = c & 1;
        if (issued[b] > 0 && !waitp(&fre[b], freeph[b]++ & 1)) { live = false; break; }
        const int kcols = min(kTcKC, KP - c * kTcKC);
        float *ca = as + b * S::A_FLOATS;
        float *cb = bs + b * S::B_FLOATS;
        const int kcm = kcols / 4;  // core-matrix columns in this chunk (even)
        // A: a warp owns an 8-row group; each lane computes two entries (core-matrix columns
        // kc and kc+2) as independent chains, and each of the two float2 (Re, Im) stores of a
        // warp covers two whole core matrices (256 contiguous bytes, no bank conflicts)
        for (int gq = warp; gq < (Q2 + 7) / 8; gq += kTcProducers / 32) {
          const int o = 8 * gq + ((lane >> 1) & 7);
          if (o < Q2) {
            float2 v[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
              const int kc = (lane >> 4) + 2 * h, il = 2 * kc + (lane & 1);
              const int i = c * (kTcKC / 2) + il;
              v[h] = make_float2(0.f, 0.f);
              if (kc < kcm && i < Q2) {
                const int t = FWD ? o : i, s_ = FWD ? i : o;  // x-node t, p-node s
                if (sep) {
                  v[h] = expi<float>(theta_xp(ph, xn(tb, l, a1, t / Q, Q), xn(tb, l, a2, t % Q, Q),
                                              pn1(tb, lb, b1, s_ / Q, Q), pn2(tb, lb, b2, s_ % Q, Q)));
                } else {
                  const df th = df_mul(rho_s[s_ / Q], gt[t * Q + s_ % Q]);
                  const float r = (th.h - rintf(th.h)) + th.l;  // exact reduction, |r| <= 1/2
                  __sincosf(6.283185307179586f * r, &v[h].y, &v[h].x);
                }
                if (!FWD) v[h].y = -v[h].y;
              }
            }
#pragma unroll
            for (int h = 0; h < 2; h++) {
              const int kc = (lane >> 4) + 2 * h;
              if (kc < kcm) {
                const int off = ((o >> 3) * (kTcKC / 4) + kc) * 32 + (o & 7) * 4 + 2 * (lane & 1);
                float pr_[kTcPA], pi_[kTcPA];
                tf32_split<kTcPA>(v[h].x, pr_);
                tf32_split<kTcPA>(v[h].y, pi_);
#pragma unroll
                for (int q_ = 0; q_ < kTcPA; q_++)
                  *reinterpret_cast<float2 *>(ca + 2 * q_ * S::A_FLOATS + off) = make_float2(pr_[q_], pi_[q_]);
              }
            }
          }
        }
        // B: a warp writes one whole core matrix per store (lane: row n, K index j)
        for (int unit = warp; unit < 8 * kcm; unit += kTcProducers / 32) {
          const int gn = unit / kcm, kc = unit - gn * kcm;
          const int n = 8 * gn + (lane >> 2), j = lane & 3;
          const int kl = 4 * kc + j, il = kl >> 1, part = kl & 1;
          const int s_ = c * (kTcKC / 2) + il, r = n & 31;
          float x = 0.f;
          if (r < rc && s_ < Q2) {
            const float2 v = ins[r * Q2 + s_];
            x = n < 32 ? (part == 0 ? v.x : -v.y) : (part == 0 ? v.y : v.x);
          }
          const int off = (gn * (kTcKC / 4) + kc) * 32 + (lane >> 2) * 4 + j;
          float pt[kTcPB];
          tf32_split<kTcPB>(x, pt);
#pragma unroll
          for (int q_ = 0; q_ < kTcPB; q_++) cb[2 * q_ * S::B_FLOATS + off] = pt[q_];
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        producers_sync();
        if (tid == 0) mbar_arrive(&full[b]);
        issued[b]++;
      }
      if (!live) break;
      // epilogue of this pair (its accumulator dsel), warps 0-3 = TMEM lanes 0..127
      if (!waitp(&dfull[dsel], dfph[dsel]++ & 1)) { live = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (warp < 4) {
        const int o = 32 * warp + lane;
        const uint32_t trow = tmem + 64 * dsel + ((uint32_t)(32 * warp) << 16);
#pragma unroll 1
        for (int h = 0; h < 2; h++) {
          float re[16], im[16];
          tc_ld16(trow + 16 * h, re);
          tc_ld16(trow + 32 + 16 * h, im);
          if (o < Q2)
            for (int r = 0; r < 16 && 16 * h + r < rc; r++)
              out[pr * nrq + (long long)(r0 + 16 * h + r) * Q2 + o] = make_float2(re[r], im[r]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      producers_sync();
      if (tid == 0) mbar_arrive(&dempty[dsel]);
    }
    cp_async_wait(0);
  }
  // the MMA warp has drained its MMAs (fin) and the producers their loads
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}

// ---------------------------------------------------------------------------
// Second tensor-core switch: the kernel matrix lives in tensor memory.
//
// Same real GEMM as above (A = kernel, M = q^2 rows padded to 128; B = the
// coefficients in the [Re, Im; -Im, Re] form, N = 64; split TF32, 5 or 3 products),
// but A never touches shared memory: the producer thread that owns row t of A
// (TMEM lane t) computes its kernel entries and writes both TF32 parts to tensor
// memory with tcgen05.st, and the MMA reads A from there (the [a-tmem] operand
// form), so only B (2 KB per MMA) is read from shared memory.
//
// K is cut into chunks of kTmCK MMA K-steps.  A chunk occupies one A slot in
// tensor memory (2 parts x kTmKC columns) and one B slot in shared memory (3 or 2
// parts); kTmNB slots of each form a ring, so the producers run up to kTmNB
// chunks ahead of the MMA warp.  Tensor memory (512 columns, one CTA per SM):
// two 64-column accumulators (the epilogue of a pair overlaps the MMAs of the
// next) and the A ring.  Pairs are walked (box A, angular box of B) first and
// radial box of B last; the producers tabulate G(x_t, p2) (q^3 values, homogeneity
// of Phi) once per 2^l pairs that share it, keep rho(p1) of every radial box, and
// prefetch the next pair's coefficients; each kernel entry is then one
// double-float product, the exact reduction mod 1 and the SFU sine/cosine.  Producer warps own TMEM lane quarters (warp % 4); the
// kTmPQ warps of a quarter split a chunk's columns, and warps whose quarter holds
// no row of A (q^2 <= 96 leaves quarter 3 empty) build B.
//
// Hand-offs are mbarriers (all waits bounded, warp-uniform outcome):
//   full[j]   producers -> MMA   (arrive count kTmProducers) chunk in slot j written
//   fre[j]    MMA -> producers   (tcgen05.commit)            slot j read
//   dfull[d]  MMA -> producers   (tcgen05.commit)            accumulator d complete
//   dempty[d] producers -> MMA   (arrive count kTmProducers) accumulator d read out
// On the producer side one warp (kTmWaiter) polls fre / dfull and the other producer warps
// park at named barrier 1 (bar.red.and: every producer gets the same go/abort outcome),
// so only one warp spends issue slots on a hand-off; the producers' own step (tables and
// inputs of the next pair in place) is that barrier alone.
// ---------------------------------------------------------------------------
constexpr int kTmProducers = 512;               // 16 producer warps, 4 per TMEM lane quarter
constexpr int kTmThreads = kTmProducers + 32;   // + 1 MMA warp
constexpr int kTmCK = 7;                        // MMA K-steps per chunk (q = 9: 3 chunks per pair)
constexpr int kTmKC = 8 * kTmCK;                // K columns per chunk (28 complex kernel columns)
constexpr int kTmNB = 3;                        // ring slots (A in TMEM, B in shared memory)
constexpr int kTmDcols = 128;                   // two accumulators of 64 columns
constexpr int kTmAcols = 2 * kTmKC;             // TMEM columns of one A slot (two TF32 parts)
constexpr int kTmSmemFloor = 120 * 1024;        // > half an SM's shared memory: one CTA (512 TMEM columns) per SM
constexpr int kTmNb1Max = 64;                   // radial boxes at the switch level (2^ceil(L/2), N <= 4096)
constexpr int kTmPQ = kTmProducers / 128;        // producer warps per lane quarter
constexpr int kTmWaiter = kTmProducers / 32 - 1; // the producer warp that polls the MMA warp's mbarriers
static_assert(kTmProducers % 128 == 0, "producer warps per lane quarter");

// NP: split-TF32 products per K-step.  5: A = A0 + A1, B = B0 + B1 + B2 (B2 the exact FP32
// remainder), A0 B0 + A0 B1 + A1 B0 + A0 B2 + A1 B1; the dropped terms are ~2^-22 |A||B|
// and the truncation of B2 ~2^-33 |B|.  3: B = B0 + B1 as well, A0 B0 + A0 B1 + A1 B0;
// A1 B1 and the two split residuals each stay below 2^-22 |A||B| (|A1| <= 2^-11 |A|,
// |A - A0 - A1| <= 2^-22 |A|, likewise for B), so a product is off by at most ~3 * 2^-22
// of |A||B|: about the rounding an FP32 sum of the q^2-term row already carries.
// W (wide): the products as two wide MMAs per K-step into one accumulator whose 64-column
// blocks the epilogue sums: A0 x [B0|B1|B2] (N = 192) and A1 x [B0|B1] (N = 128) for NP = 5;
// A0 x [B0|B1] (N = 128) and A1 x B0 (N = 64) for NP = 3.  Two accumulators double-buffer
// the pairs.
template <bool W, int NP = 5> struct TmCfg {
  static_assert(NP == 5 || NP == 3, "split-TF32 products per K-step");
  static constexpr int PB = NP == 5 ? 3 : 2;       // TF32 parts of B
  static constexpr int CK = (W && NP == 5) ? 4 : kTmCK;  // MMA K-steps per chunk
  static constexpr int KC = 8 * CK;                // K columns per chunk
  static constexpr int NB = W ? 2 : kTmNB;         // ring slots
  static constexpr int ACC = W ? 64 * PB : 64;     // columns of one accumulator
  static constexpr int DC = 2 * ACC;               // both accumulators
  static constexpr int AC = 2 * KC;                // one A slot (two TF32 parts)
  static_assert(DC + NB * AC <= 512, "tensor memory budget");
  static_assert((KC / 2) % kTmPQ == 0, "producer warps split a chunk's columns evenly");
};

template <int Q, bool W = false, int NP = 5> struct TmShape {
  typedef TmCfg<W, NP> C;
  static constexpr int Q2 = Q * Q;
  static constexpr int KP = ((2 * Q2 + 7) / 8) * 8;        // padded K
  static constexpr int KS = KP / 8;                        // MMA K-steps per pair
  static constexpr int NCH = (KS + C::CK - 1) / C::CK;     // chunks per pair (the last may be partial)
  static constexpr int B_FLOATS = 64 * C::KC;              // one TF32 part of one B slot
  static constexpr size_t b_bytes = (size_t)C::NB * C::PB * B_FLOATS * 4;
  static constexpr size_t in_bytes = (size_t)2 * kRMax * Q2 * 8;
  static constexpr size_t gt_bytes = (size_t)2 * Q2 * Q * sizeof(df);
  static constexpr size_t rho_bytes = (size_t)kTmNb1Max * Q * sizeof(df);
  static constexpr int nbar = 2 * C::NB + 5;
  static constexpr size_t used = b_bytes + in_bytes + gt_bytes + rho_bytes + nbar * 8 + 16;
  static constexpr size_t smem_bytes() { return used > (size_t)kTmSmemFloor ? used : (size_t)kTmSmemFloor; }
};

// Instruction descriptor of kind::tf32: D f32, A and B tf32 K-major, M = 128, N as given.
template <int N> constexpr uint32_t tf32_idesc() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((128u >> 4) << 24);
}
template <int N> __device__ __forceinline__ void tm_mma_n(uint32_t dtm, uint32_t atm, uint64_t db, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(dtm),
      "r"(atm), "l"(db), "r"(tf32_idesc<N>()), "r"(acc));
}
__device__ __forceinline__ void tm_mma(uint32_t dtm, uint32_t atm, uint64_t db, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(dtm),
      "r"(atm), "l"(db), "r"(kTcIdesc), "r"(acc));
}
__device__ __forceinline__ void tm_st8(uint32_t taddr, const float *v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
               "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
               "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
               "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
               : "memory");
}
__device__ __forceinline__ void tm_st4(uint32_t taddr, const float *v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr), "r"(__float_as_uint(v[0])),
               "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3]))
               : "memory");
}
__device__ __forceinline__ void tm_st2(uint32_t taddr, const float *v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1,%2};" ::"r"(taddr), "r"(__float_as_uint(v[0])),
               "r"(__float_as_uint(v[1]))
               : "memory");
}
// Store NC (a multiple of 2) consecutive columns of this warp's lanes.
template <int NC> __device__ __forceinline__ void tm_st(uint32_t taddr, const float *v) {
  static_assert(NC % 2 == 0, "column count");
#pragma unroll
  for (int c = 0; c + 8 <= NC; c += 8) tm_st8(taddr + c, v + c);
  constexpr int O8 = NC / 8 * 8;
  if constexpr (NC - O8 >= 4) tm_st4(taddr + O8, v + O8);
  constexpr int O4 = NC - O8 >= 4 ? O8 + 4 : O8;
  if constexpr (NC - O4 == 2) tm_st2(taddr + O4, v + O4);
}
__device__ __forceinline__ void tc_ld8(uint32_t taddr, float *v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 8; c++) v[c] = __uint_as_float(r[c]);
}
// tcgen05.ld of 8 columns without the wait (the caller waits once for several loads).
__device__ __forceinline__ void tc_ld8_issue(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tm_arrive(uint64_t *mbar) { mbar_arrive(mbar); }

// handoff_ns: limit of the waits between the producer warps and the MMA warp (0: the
// normal 2 s); a test sets it tiny to make them expire.  The final drain of the issued
// MMAs (fin) always waits with the normal limit.
template <int Q, bool FWD, bool W = false, int NP = 5>
__global__ void __launch_bounds__(kTmThreads, 1) k32_switch_tm(Tables tb, TablesF tf, Phase ph, Geom g,
                                                                const float2 *__restrict__ in,
                                                                float2 *__restrict__ out, int *status,
                                                                unsigned long long handoff_ns) {
  typedef TmShape<Q, W, NP> S;
  typedef TmCfg<W, NP> C;
  constexpr int Q2 = S::Q2, KS = S::KS, NCH = S::NCH, PB = C::PB;
  constexpr int CPW = C::KC / 2 / kTmPQ;  // complex kernel columns per producer warp and chunk
  constexpr int RPW = kRMax / kTmPQ;      // RHS per producer warp in the epilogue
  constexpr int KCC = C::KC / 4;  // core-matrix columns (4 K each) per chunk
  extern __shared__ __align__(16) unsigned char smem_raw[];  // no-swizzle operands need 16-byte alignment
  float *bs = (float *)smem_raw;                                   // B [slot][part][8 row groups][KCC][8][4]
  float2 *instage = (float2 *)(smem_raw + S::b_bytes);             // [2][kRMax][Q2] coefficients
  df *gt = (df *)(smem_raw + S::b_bytes + S::in_bytes);            // [2][Q2][Q] G(x_t, p2_s2)
  df *rho = gt + 2 * Q2 * Q;                                       // [kTmNb1Max][Q] rho of every radial box
  uint64_t *full = (uint64_t *)(rho + kTmNb1Max * Q);
  uint64_t *fre = full + C::NB;
  uint64_t *dfull = fre + C::NB;
  uint64_t *dempty = dfull + 2;
  uint64_t *fin = dempty + 2;
  uint32_t *tmem_s = (uint32_t *)(fin + 1);
  volatile int *abort_s = (volatile int *)(tmem_s + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int l = g.l, lb = g.L - g.l, e = g.e;
  const int nb1 = 1 << lb, nb2 = 1 << (lb + e);
  // Pair order: the pairs of one super-unit (box A, angular box b2) differ only in the
  // radial box b1 and share G(x_t, p2); CTA c takes super-units c, c + gridDim.x, ...
  // and within each all nb1 radial boxes.
  // nb1 and nb2 are powers of two: every index below is a shift or a mask
  const int lb2 = lb + e;  // log2 nb2
  const long long nsu = g.nunits >> lb;
  const int r0 = blockIdx.y * kRMax;
  const int rc = min(kRMax, g.nrhs - r0);
  const long long nrq = (long long)g.nrhs * Q2;
  const bool sep = ph.id == 3;
  auto su_of = [&](long long k) { return (long long)blockIdx.x + (k >> lb) * gridDim.x; };
  auto pair_of = [&](long long k) {  // global pair index of the CTA's k-th pair
    const long long su = su_of(k);
    return ((su >> lb2) << (lb + lb2)) + ((k & (nb1 - 1)) << lb2) + (su & (nb2 - 1));
  };

  if (tid == 0) {
    for (int b = 0; b < S::nbar; b++) {
      const int cnt = (b < C::NB || (b >= 2 * C::NB + 2 && b < 2 * C::NB + 4)) ? kTmProducers : 1;
      const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&full[b]);
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(cnt));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_s = 0;
  }
  if (warp == 0) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(tmem_s);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(dst));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_s;
  // bounded wait with a warp-uniform outcome; on expiry record the status and raise the abort flag
  const unsigned long long hlim = handoff_ns ? handoff_ns : kTcWaitNs;
  auto waitw = [&](uint64_t *mb, uint32_t parity) {
    bool ok = !*abort_s && tc_wait(mb, parity, hlim);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok && lane == 0) {
      atomicExch(status, 1);
      *abort_s = 1;
    }
    return ok;
  };
  // producers only: AND of `ok` over all producer threads at named barrier 1
  auto psync = [&](bool ok) {
    uint32_t r;
    asm volatile(
        "{\n.reg .pred pi, po;\nsetp.ne.u32 pi, %1, 0;\nbar.red.and.pred po, 1, %2, pi;\nselp.u32 %0, 1, 0, po;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)ok), "n"(kTmProducers)
        : "memory");
    return r != 0;
  };
  auto pwait = [&](uint64_t *mb, uint32_t parity) { return psync(warp == kTmWaiter ? waitw(mb, parity) : true); };

  if (warp == kTmProducers / 32) {
    // ------------------------------------------------------------ MMA warp
    const uint32_t aB = (uint32_t)__cvta_generic_to_shared(bs);
    constexpr uint32_t sbo = KCC * 128;
    uint32_t gc = 0;
    bool live = true;
    for (long long k = 0; su_of(k) < nsu && live; k++) {
      const int d = (int)(k & 1);
      if (k >= 2 && !waitw(&dempty[d], (uint32_t)((k >> 1) - 1) & 1)) break;  // read-out of pair k - 2
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t dtm = tmem + C::ACC * d;
      for (int c = 0; c < NCH; c++, gc++) {
        const int j = (int)(gc % C::NB);
        if (!waitw(&full[j], (gc / C::NB) & 1)) { live = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (lane == 0) {
          const int nks = min(C::CK, KS - c * C::CK);
          const uint32_t a0 = tmem + C::DC + j * C::AC;
          for (int ks = 0; ks < nks; ks++) {
            uint64_t dB[PB];
#pragma unroll
            for (int q_ = 0; q_ < PB; q_++)
              dB[q_] = tc_desc(aB + ((j * PB + q_) * S::B_FLOATS) * 4 + ks * 256, 128, sbo);
            const uint32_t ta0 = a0 + 8 * ks, ta1 = a0 + C::KC + 8 * ks;
            const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
            if (W) {  // the B parts lie one after another: one descriptor spans 64 PB rows
              tm_mma_n<64 * PB>(dtm, ta0, dB[0], acc);
              tm_mma_n<64 * (PB - 1)>(dtm, ta1, dB[0], 1u);
            } else {
              tm_mma(dtm, ta0, dB[0], acc);
              tm_mma(dtm, ta0, dB[1], 1u);
              tm_mma(dtm, ta1, dB[0], 1u);
              if (NP == 5) {
                tm_mma(dtm, ta0, dB[PB - 1], 1u);
                tm_mma(dtm, ta1, dB[1], 1u);
              }
            }
          }
          tc_commit(&fre[j]);
          if (c == NCH - 1) tc_commit(&dfull[d]);
        }
        __syncwarp();
      }
    }
    // drain: wait (bounded) until every MMA this warp issued has completed
    if (lane == 0) tc_commit(fin);
    __syncwarp();
    if (!tc_wait(fin, 0) && lane == 0) atomicExch(status, 1);
  } else {
    // ------------------------------------------------------------ producer warps
    const int qd = warp & 3, wh = warp >> 2;      // lane quarter, index among the quarter's warps
    const int o = 32 * qd + lane;                 // TMEM lane = row of A
    const bool arows = 32 * qd < Q2;              // this warp's quarter holds rows of A
    const bool ovalid = o < Q2;
    const int oc = ovalid ? o : Q2 - 1;           // clamped row for branch-free table reads
    // B tasks (one core-matrix column kc of a chunk, all 64 rows): spread over the warps
    // whose lane quarter holds no row of A, else over warps 0..KCC-1
    int bidx = -1, bstride = 1;
    {
      const int nA = min(4, (Q2 + 31) / 32);
      if (nA == 4) {
        bidx = warp;
        bstride = kTmProducers / 32;
      } else {
        const int per = 4 - nA;
        if ((warp & 3) >= nA) bidx = (warp >> 2) * per + (warp & 3) - nA;
        bstride = kTmPQ * per;
      }
    }
    auto prefetch = [&](long long k, int slot) {
      if (su_of(k) < nsu) {
        const float2 *src = in + pair_of(k) * nrq + (long long)r0 * Q2;
        for (int i = tid; i < rc * Q2; i += kTmProducers) cp_async8(instage + slot * kRMax * Q2 + i, src + i);
      }
      cp_async_commit();
    };
    auto tables = [&](long long k, int b) {  // G of the super-unit of pair k into gt[b]
      if (sep) return;
      const long long su = su_of(k);
      const long long a = su >> lb2;
      const int a1 = (int)(a >> l), a2 = (int)(a & ((1LL << l) - 1)), b2 = (int)(su & (nb2 - 1));
      df *gtb = gt + b * Q2 * Q;
      for (int idx = tid; idx < Q2 * Q; idx += kTmProducers) {
        const int t = idx / Q, s2 = idx - t * Q;
        const XDesc xdt = xdesc(tf.ph, xnf(tb, tf, l, a1, t / Q, Q), xnf(tb, tf, l, a2, t % Q, Q));
        gtb[idx] = g_eval(tf.ph, xdt, p2f(tb, tf, lb, b2, s2, Q));
      }
    };
    // phase parities: use k of dfull[d] (accumulators alternate) belongs to pair 2k + d
    auto epilogue = [&](long long k) {
      const int d = (int)(k & 1);
      if (!pwait(&dfull[d], (uint32_t)(k >> 1) & 1)) return false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (arows) {
        static_assert(RPW == 8, "epilogue reads 8 columns per warp");
        const uint32_t trow = tmem + C::ACC * d + RPW * wh + ((uint32_t)(32 * qd) << 16);
        // every block's loads in flight at once, one wait; the wide accumulator's further
        // 64-column blocks are then added in order
        constexpr int NBK = W ? PB : 1;
        uint32_t v[NBK][2][RPW];
#pragma unroll
        for (int blk = 0; blk < NBK; blk++)
#pragma unroll
          for (int h = 0; h < 2; h++) tc_ld8_issue(trow + 64 * blk + 32 * h, v[blk][h]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float re[RPW], im[RPW];
#pragma unroll
        for (int r = 0; r < RPW; r++) {
          re[r] = __uint_as_float(v[0][0][r]);
          im[r] = __uint_as_float(v[0][1][r]);
        }
#pragma unroll
        for (int blk = 1; blk < NBK; blk++)
#pragma unroll
          for (int r = 0; r < RPW; r++) {
            re[r] += __uint_as_float(v[blk][0][r]);
            im[r] += __uint_as_float(v[blk][1][r]);
          }
        if (o < Q2) {
          float2 *dst = out + pair_of(k) * nrq + (long long)(r0 + RPW * wh) * Q2 + o;
#pragma unroll
          for (int r = 0; r < RPW; r++)
            if (RPW * wh + r < rc) dst[(long long)r * Q2] = make_float2(re[r], im[r]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      tm_arrive(&dempty[d]);
      return true;
    };

    if (blockIdx.x < nsu) {
      if (!sep)
        for (int idx = tid; idx < nb1 * Q; idx += kTmProducers) rho[idx] = rhof(tb, tf, lb, idx / Q, idx % Q, Q);
      prefetch(0, 0);
      tables(0, 0);
      cp_async_wait(0);
    }
    uint32_t gc = 0;
    long long k = 0;
    bool live = true;
    for (; su_of(k) < nsu && live; k++) {
      const int b = (int)(k & 1);
      if (!psync(!*abort_s)) break;  // inputs and tables of pair k in place
      prefetch(k + 1, b ^ 1);
      const float2 *ins = instage + b * kRMax * Q2;
      const df *gtb = gt + (int)((k >> lb) & 1) * Q2 * Q;
      const int b1 = (int)(k & (nb1 - 1));
      const df *rhob = rho + b1 * Q;
      int a1 = 0, a2 = 0, b2 = 0;
      if (sep) {
        const long long su = su_of(k), a = su >> lb2;
        a1 = (int)(a >> l);
        a2 = (int)(a & ((1LL << l) - 1));
        b2 = (int)(su & (nb2 - 1));
      }
      // FWD: row o = x-node t, columns s walk (s1, s2); adjoint: row o = p-node s (fixed
      // rho and s2), columns t walk G down a column
      const df rho_row = (!FWD && !sep) ? rhob[oc / Q] : df{0.f, 0.f};
      const df *grow = FWD ? gtb + oc * Q : gtb + oc % Q;
      // The chunks of a pair are unrolled at compile time (c) and each producer warp's
      // columns are dispatched on its index among the quarter's warps (wh), so every column
      // index is a constant: table reads take immediate offsets and the padding columns
      // (i >= q^2) are zeros known at compile time.  Rows o >= q^2 (lanes of the M = 128
      // padding) repeat row q^2 - 1: finite values in rows of D nobody reads.
      static_for<NCH>([&](auto cI) {
        constexpr int c = decltype(cI)::value;
        if (!live) return;
        const int j = (int)(gc % C::NB);
        if (gc >= C::NB && !pwait(&fre[j], (gc / C::NB - 1) & 1)) {
          live = false;
          return;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (arows) {
          const uint32_t ta = tmem + ((uint32_t)(32 * qd) << 16) + C::DC + j * C::AC + 2 * CPW * wh;
          if (!sep) {
            static_switch<kTmPQ>(wh, [&](auto whI) {
              constexpr int i0 = c * (C::KC / 2) + decltype(whI)::value * CPW;  // first column of this warp
              float p0[2 * CPW], p1[2 * CPW];
#pragma unroll
              for (int kk = 0; kk < CPW; kk++) {
                const int i = i0 + kk;
                float2 v = make_float2(0.f, 0.f);
                if (i < Q2) {
                  // FWD: row o = x-node t, column i = (s1, s2); adjoint: row o = p-node s,
                  // column i = x-node t (G read down the column of s2).  theta = R G in
                  // double-float; (p - rint p) is exact, so the reduction mod 1 needs no
                  // renormalisation of (p, lo)
                  const df G = FWD ? grow[i % Q] : grow[i * Q];
                  const df R = FWD ? rhob[i / Q] : rho_row;
                  const float pp = R.h * G.h;
                  const float lo = __fmaf_rn(R.h, G.l, __fmaf_rn(R.l, G.h, __fmaf_rn(R.h, G.h, -pp)));
                  const float r = (pp - rintf(pp)) + lo;
                  __sincosf(6.283185307179586f * r, &v.y, &v.x);
                  if (!FWD) v.y = -v.y;
                }
                p0[2 * kk] = tf32_rna(v.x);
                p0[2 * kk + 1] = tf32_rna(v.y);
                p1[2 * kk] = tf32_rna(v.x - p0[2 * kk]);
                p1[2 * kk + 1] = tf32_rna(v.y - p0[2 * kk + 1]);
              }
              __syncwarp();
              tm_st<2 * CPW>(ta, p0);
              tm_st<2 * CPW>(ta + C::KC, p1);
            });
          } else {  // separable phase: theta from the node coordinates, invalid entries zeroed
            float p0[2 * CPW], p1[2 * CPW];
            const int i0 = c * (C::KC / 2) + wh * CPW;
#pragma unroll
            for (int kk = 0; kk < CPW; kk++) {
              const int i = i0 + kk;
              const bool ok = ovalid && i < Q2;
              const int ic = i < Q2 ? i : Q2 - 1;
              const int t = FWD ? oc : ic, s_ = FWD ? ic : oc;
              float2 v = expi<float>(theta_xp(ph, xn(tb, l, a1, t / Q, Q), xn(tb, l, a2, t % Q, Q),
                                              pn1(tb, lb, b1, s_ / Q, Q), pn2(tb, lb, b2, s_ % Q, Q)));
              v.x = ok ? v.x : 0.f;
              v.y = ok ? (FWD ? v.y : -v.y) : 0.f;
              p0[2 * kk] = tf32_rna(v.x);
              p0[2 * kk + 1] = tf32_rna(v.y);
              p1[2 * kk] = tf32_rna(v.x - p0[2 * kk]);
              p1[2 * kk + 1] = tf32_rna(v.y - p0[2 * kk + 1]);
            }
            __syncwarp();
            tm_st<2 * CPW>(ta, p0);
            tm_st<2 * CPW>(ta + C::KC, p1);
          }
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        // B: lane r builds rows r and 32 + r of core-matrix column kc from X[r][s0], X[r][s0+1]
        // (s0 = the chunk's first complex column + 2 kc): [Re, -Im] and [Im, Re], three TF32 parts
        if (bidx >= 0) {
          float *cb = bs + j * PB * S::B_FLOATS;
          for (int kc = bidx; kc < KCC; kc += bstride) {
            const int s0 = c * (C::KC / 2) + 2 * kc;
            const int rr = lane < rc ? lane : 0;
            float2 x0 = ins[rr * Q2 + min(s0, Q2 - 1)], x1 = ins[rr * Q2 + min(s0 + 1, Q2 - 1)];
            if (!(lane < rc && s0 < Q2)) x0 = make_float2(0.f, 0.f);  // rows beyond rc were not loaded
            if (!(lane < rc && s0 + 1 < Q2)) x1 = make_float2(0.f, 0.f);
            float ar[PB], ai[PB], br[PB], bi[PB];
            tf32_split<PB>(x0.x, ar);
            tf32_split<PB>(x0.y, ai);
            tf32_split<PB>(x1.x, br);
            tf32_split<PB>(x1.y, bi);
            float *top = cb + ((lane >> 3) * KCC + kc) * 32 + (lane & 7) * 4;
            float *bot = top + 4 * KCC * 32;
#pragma unroll
            for (int q_ = 0; q_ < PB; q_++) {
              *reinterpret_cast<float4 *>(top + q_ * S::B_FLOATS) = make_float4(ar[q_], -ai[q_], br[q_], -bi[q_]);
              *reinterpret_cast<float4 *>(bot + q_ * S::B_FLOATS) = make_float4(ai[q_], ar[q_], bi[q_], br[q_]);
            }
          }
        }
        // B went through the generic proxy: make it visible to the tensor core's async proxy
        if (bidx >= 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        tm_arrive(&full[j]);
        gc++;
      });
      if (!live) break;
      if (k > 0 && !epilogue(k - 1)) break;
      if (su_of(k + 1) < nsu) {
        if (((k + 1) & (nb1 - 1)) == 0) tables(k + 1, (int)(((k + 1) >> lb) & 1));
        cp_async_wait(0);
      }
    }
    if (live && k > 0 && psync(!*abort_s)) epilogue(k - 1);
    cp_async_wait(0);
  }
  // the MMA warp has drained its MMAs (fin) and the producers their loads
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

}  // namespace fio
