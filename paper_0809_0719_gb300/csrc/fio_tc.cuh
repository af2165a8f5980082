// fio_tc.cuh -- the FP32 form's switch (eq. alg2m) on the 5th-generation tensor
// cores: tcgen05.mma kind::tf32 with operands in shared memory and the FP32
// accumulator in tensor memory, as an error-compensated 3xTF32 product.
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
#include "fio_k32.cuh"

namespace fio {

constexpr int kTcProducers = 256;               // 8 producer warps
constexpr int kTcThreads = kTcProducers + 32;   // + 1 MMA warp
constexpr int kTcKC = 16;                       // K columns per chunk (2 MMA K-steps)
constexpr int kTcPA = 2, kTcPB = 3;             // TF32 parts of A (kernel) and B (coefficients)
constexpr long long kTcSpin = 1LL << 24;        // bounded mbarrier polling (>= ~2 s with the back-off)

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the 5th-generation tensor core; no swizzle
  return d;
}
// D f32, A and B tf32, both K-major, N = 64, M = 128.
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// x = p0 + p1 (+ p2) with each part in TF32; the residual is ~2^-22 |x| (~2^-33 |x|).
template <int P> __device__ __forceinline__ void tf32_split(float x, float *p) {
  p[0] = tf32_rna(x);
  float r = x - p[0];
  p[1] = tf32_rna(r);
  if (P > 2) p[2] = tf32_rna(r - p[1]);
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
// Bounded wait for the completion of the mbarrier phase with the given parity.
__device__ __forceinline__ bool tc_wait(uint64_t *mbar, uint32_t parity) {
  const uint32_t mb = (uint32_t)__cvta_generic_to_shared(mbar);
  uint32_t done = 0;
  for (long long it = 0; it < kTcSpin; it++) {
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done)
                 : "r"(mb), "r"(parity)
                 : "memory");
    if (done) return true;
    if (it > 2) __nanosleep(128);  // yield the issue slots to the warps doing work
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

}  // namespace fio
