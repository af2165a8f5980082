// fio_k32.cuh -- kernels of the FP32 form (coefficients, interpolation and
// accumulation in FP32; phases in double-float on the FMA pipe, fio_df.cuh).
//
// Differences from the FP64-form kernels in fio_kernels.cuh:
//  * one CTA owns a translation unit for up to 32 right-hand sides, so its
//    20 q^2 phase factors are computed once and shared by all of them;
//  * the CTA has 32 q threads and works on 8-RHS subtiles, which makes each
//    pass of the dimension-wise Lagrange sums exactly one or two task rounds;
//  * outputs are staged in shared memory and written as contiguous runs;
//  * the switch evaluates G(x_t, p2_s) once per (t, s2) (q^3 per pair) and
//    forms the q^4 kernel entries as rho(p1_s) G (homogeneity of Phi, Sec. 1).
#pragma once
#include "fio_df.cuh"
#include "fio_kernels.cuh"

namespace fio {

// Translation CTA shape for an RHS subtile of RS right-hand sides: 4 RS q threads
// (rounded up to whole warps), shared memory: phases 20 q^2 | staging 2 x 4 RS q^2 |
// intermediate max(8 RS, 26) q^2 complex.
// The intermediate area also serves as the phase scratch (26 q^2 complex at most).
__host__ __device__ constexpr int trans32_zsize(int rs) { return 8 * rs > 26 ? 8 * rs : 26; }
__host__ __device__ constexpr int trans32_smem_bytes(int q, int rs) {
  return (20 + 8 * rs + trans32_zsize(rs)) * q * q * 8;
}
template <int Q, int RS> struct TransShape {
  static constexpr int threads = (4 * RS * Q + 31) / 32 * 32;
  static constexpr int smem = trans32_smem_bytes(Q, RS);
  static constexpr int min_blocks = RS >= 8 ? 2 : RS >= 4 ? 4 : 5;
};
constexpr int kRMax = 32;   // RHS per CTA (grid.y covers the rest)

// df tables of an FP32-form plan (same indexing as the FP64 tables in Tables).
struct TablesF {
  const XNodeF *xnode;
  const P1NodeF *p1node;
  const P2NodeF *p2node;
  const XNodeF *xgrid;
  const SrcF *src;
  PhaseF ph;
};

__device__ __forceinline__ const XNodeF &xnf(const Tables &tb, const TablesF &tf, int l, int box, int j, int q) {
  return tf.xnode[tb.xoff[l] + box * (q + 1) + j];
}
__device__ __forceinline__ df rhof(const Tables &tb, const TablesF &tf, int j, int box, int t, int q) {
  return tf.p1node[tb.p1off[j] + box * (q + 1) + t].rho;
}
__device__ __forceinline__ const P2NodeF &p2f(const Tables &tb, const TablesF &tf, int j, int box, int t, int q) {
  return tf.p2node[tb.p2off[j] + box * (q + 1) + t];
}

// Phase family "centres": x at the centres of the four children A_sigma of A_p
// (level l), p on the node grids of B (level lb) and of its children B_c (lb+1).
//   ec[sigma][c][u] = e(x0(A_sigma), p^{B_c}_u)   (16 q^2)
//   ep[sigma][t]    = e(x0(A_sigma), p^B_t)       (4 q^2)
// scratch: >= 4 XDesc + 12 q df.
template <int Q>
__device__ void family_centres(const Tables &tb, const TablesF &tf, const Phase &ph, const UnitIdx &d, int l, int lb,
                               float2 *ec, float2 *ep, unsigned char *scratch) {
  constexpr int Q2 = Q * Q;
  XDesc *xd = (XDesc *)scratch;
  df *gc = (df *)(xd + 4);  // [4 sigma][2 c2][Q]
  df *gp = gc + 8 * Q;      // [4 sigma][Q]
  if (ph.id == 3) {  // separable test phase: direct FP64 evaluation
    for (int idx = threadIdx.x; idx < 20 * Q2; idx += blockDim.x) {
      const int sg = idx < 16 * Q2 ? idx / (4 * Q2) : (idx - 16 * Q2) / Q2;
      const int a1 = 2 * d.ap1 + (sg >> 1), a2 = 2 * d.ap2 + (sg & 1);
      const XNode &x1 = xn(tb, l, a1, Q, Q), &x2 = xn(tb, l, a2, Q, Q);
      if (idx < 16 * Q2) {
        const int c = (idx / Q2) & 3, u = idx % Q2;
        ec[idx] = expi<float>(theta_xp(ph, x1, x2, pn1(tb, lb + 1, 2 * d.b1 + (c >> 1), u / Q, Q),
                                       pn2(tb, lb + 1, 2 * d.b2 + (c & 1), u % Q, Q)));
      } else {
        const int t = (idx - 16 * Q2) % Q2;
        ep[idx - 16 * Q2] = expi<float>(theta_xp(ph, x1, x2, pn1(tb, lb, d.b1, t / Q, Q), pn2(tb, lb, d.b2, t % Q, Q)));
      }
    }
    __syncthreads();
    return;
  }
  if (threadIdx.x < 4) {
    const int sg = threadIdx.x;
    xd[sg] = xdesc(tf.ph, xnf(tb, tf, l, 2 * d.ap1 + (sg >> 1), Q, Q), xnf(tb, tf, l, 2 * d.ap2 + (sg & 1), Q, Q));
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 12 * Q; idx += blockDim.x) {
    if (idx < 8 * Q) {
      const int sg = idx / (2 * Q), c2 = (idx / Q) & 1, u2 = idx % Q;
      gc[idx] = g_eval(tf.ph, xd[sg], p2f(tb, tf, lb + 1, 2 * d.b2 + c2, u2, Q));
    } else {
      const int k = idx - 8 * Q, sg = k / Q, t2 = k % Q;
      gp[k] = g_eval(tf.ph, xd[sg], p2f(tb, tf, lb, d.b2, t2, Q));
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 20 * Q2; idx += blockDim.x) {
    if (idx < 16 * Q2) {
      const int sg = idx / (4 * Q2), c = (idx / Q2) & 3, u = idx % Q2;
      const df rho = rhof(tb, tf, lb + 1, 2 * d.b1 + (c >> 1), u / Q, Q);
      ec[idx] = expi_df(df_mul(rho, gc[(sg * 2 + (c & 1)) * Q + u % Q]));
    } else {
      const int k = idx - 16 * Q2, sg = k / Q2, t = k % Q2;
      ep[k] = expi_df(df_mul(rhof(tb, tf, lb, d.b1, t / Q, Q), gp[sg * Q + t % Q]));
    }
  }
  __syncthreads();
}

// Phase family "nodes": x on the node grids of A_sigma (level l) and A_p (l-1),
// p at the centres of the children B_c (level lb+1).
//   ea[sigma][c][t] = e(x^{A_sigma}_t, p0(B_c))   (16 q^2)
//   eq[c][t']       = e(x^{A_p}_t', p0(B_c))       (4 q^2)
// scratch: >= 10 q^2 df.
template <int Q>
__device__ void family_nodes(const Tables &tb, const TablesF &tf, const Phase &ph, const UnitIdx &d, int l, int lb,
                             float2 *ea, float2 *eq, unsigned char *scratch) {
  constexpr int Q2 = Q * Q;
  df *g = (df *)scratch;  // [5][Q2][2 c2]: 4 sigma, then A_p
  if (ph.id == 3) {
    for (int idx = threadIdx.x; idx < 20 * Q2; idx += blockDim.x) {
      if (idx < 16 * Q2) {
        const int sg = idx / (4 * Q2), c = (idx / Q2) & 3, t = idx % Q2;
        const int a1 = 2 * d.ap1 + (sg >> 1), a2 = 2 * d.ap2 + (sg & 1);
        ea[idx] = expi<float>(theta_xp(ph, xn(tb, l, a1, t / Q, Q), xn(tb, l, a2, t % Q, Q),
                                       pn1(tb, lb + 1, 2 * d.b1 + (c >> 1), Q, Q), pn2(tb, lb + 1, 2 * d.b2 + (c & 1), Q, Q)));
      } else {
        const int k = idx - 16 * Q2, c = k / Q2, t = k % Q2;
        eq[k] = expi<float>(theta_xp(ph, xn(tb, l - 1, d.ap1, t / Q, Q), xn(tb, l - 1, d.ap2, t % Q, Q),
                                     pn1(tb, lb + 1, 2 * d.b1 + (c >> 1), Q, Q), pn2(tb, lb + 1, 2 * d.b2 + (c & 1), Q, Q)));
      }
    }
    __syncthreads();
    return;
  }
  for (int idx = threadIdx.x; idx < 5 * Q2; idx += blockDim.x) {
    const int w = idx / Q2, t = idx % Q2;
    const XDesc x = w < 4 ? xdesc(tf.ph, xnf(tb, tf, l, 2 * d.ap1 + (w >> 1), t / Q, Q),
                                  xnf(tb, tf, l, 2 * d.ap2 + (w & 1), t % Q, Q))
                          : xdesc(tf.ph, xnf(tb, tf, l - 1, d.ap1, t / Q, Q), xnf(tb, tf, l - 1, d.ap2, t % Q, Q));
    g[2 * idx] = g_eval(tf.ph, x, p2f(tb, tf, lb + 1, 2 * d.b2, Q, Q));
    g[2 * idx + 1] = g_eval(tf.ph, x, p2f(tb, tf, lb + 1, 2 * d.b2 + 1, Q, Q));
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 20 * Q2; idx += blockDim.x) {
    if (idx < 16 * Q2) {
      const int sg = idx / (4 * Q2), c = (idx / Q2) & 3, t = idx % Q2;
      const df rho = rhof(tb, tf, lb + 1, 2 * d.b1 + (c >> 1), Q, Q);
      ea[idx] = expi_df(df_mul(rho, g[(sg * Q2 + t) * 2 + (c & 1)]));
    } else {
      const int k = idx - 16 * Q2, c = k / Q2, t = k % Q2;
      const df rho = rhof(tb, tf, lb + 1, 2 * d.b1 + (c >> 1), Q, Q);
      eq[k] = expi_df(df_mul(rho, g[(4 * Q2 + t) * 2 + (c & 1)]));
    }
  }
  __syncthreads();
}

__device__ __forceinline__ float2 conjf2(float2 v) { return make_float2(v.x, -v.y); }
// acc + s v for a real s and a complex v as one paired FMA (FFMA2: both components in
// one instruction, each rounded as __fmaf_rn).
__device__ __forceinline__ float2 fma2s(float s, float2 v, float2 acc) { return __ffma2_rn(make_float2(s, s), v, acc); }

// Asynchronous 8-byte global->shared copies (LDGSTS), waited on by group.
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// Copy n float2 from global to shared (both 8-byte aligned) asynchronously, 16 bytes
// at a time when the global side allows it (the shared side is 16-byte aligned).
// (tid, nthr: this thread's index among the nthr threads sharing the copy.)
__device__ __forceinline__ void cp_async_run(float2 *dst, const float2 *src, int n, int tid, int nthr) {
  if ((((uintptr_t)src) & 15) == 0) {
    const int n2 = n >> 1;
    for (int k = tid; k < n2; k += nthr) cp_async16(dst + 2 * k, src + 2 * k);
    if ((n & 1) && tid == 0) cp_async8(dst + n - 1, src + n - 1);
  } else {
    for (int k = tid; k < n; k += nthr) cp_async8(dst + k, src + k);
  }
}
__device__ __forceinline__ void cp_async_run(float2 *dst, const float2 *src, int n) {
  cp_async_run(dst, src, n, threadIdx.x, blockDim.x);
}
// Store n float2 from shared (16-byte aligned) to global, 16 bytes at a time when aligned.
__device__ __forceinline__ void store_run(float2 *dst, const float2 *src, int n, int tid, int nthr) {
  if ((((uintptr_t)dst) & 15) == 0) {
    const int n2 = n >> 1;
    for (int k = tid; k < n2; k += nthr) reinterpret_cast<float4 *>(dst)[k] = reinterpret_cast<const float4 *>(src)[k];
    if ((n & 1) && tid == 0) dst[n - 1] = src[n - 1];
  } else {
    for (int k = tid; k < n; k += nthr) dst[k] = src[k];
  }
}
__device__ __forceinline__ void store_run(float2 *dst, const float2 *src, int n) {
  store_run(dst, src, n, threadIdx.x, blockDim.x);
}
// Bulk copy (TMA engine) of `bytes` (a multiple of 16) from shared to global memory, both
// 16-byte aligned, as part of the calling thread's current bulk group; commit, and wait
// until the thread's groups have read their shared-memory source (read) or completed.
__device__ __forceinline__ void bulk_s2g(void *gmem, const void *smem, uint32_t bytes) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gmem), "r"(sa), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait(int pending) {
  if (pending) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
  else asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// ---------------------------------------------------------------------------
// FP32 translation of both shapes (one CTA per unit, up to 32 RHS, 32 Q threads).
// TYPE_P: out_j = post_j (.) sum_i (T^{i1} (x) T^{i2}) (pre_{j,i} (.) in_i)
//         FWD: recursion in p (eq. alg2b); !FWD: conjugate transpose of the recursion in x.
// TYPE_X: out_j = sum_i post_{j,i} (.) (T^{j1} (x) T^{j2})^T (pre_i (.) in_i)
//         FWD: recursion in x (eq. alg2c); !FWD: conjugate transpose of the recursion in p.
// The inputs of RS-RHS subtile k+1 are copied asynchronously while subtile k is
// computed (two staging buffers); the first copies overlap the phase setup.
// Shared memory (float2): phases 20 Q^2 | staging 2 x 4 RS Q^2 | intermediate 8 RS Q^2.
// ---------------------------------------------------------------------------
template <int Q, bool TYPE_P, bool FWD, int RS>
__device__ __forceinline__ void k32_trans_body(const Tables &tb, const TablesF &tf, const Phase &ph, const Geom &g, const TMat<float, Q> &tm,
                                               const float2 *__restrict__ in, float2 *__restrict__ out, long long bx_, int by_) {
  constexpr int Q2 = Q * Q;
  constexpr int SUB = 4 * RS * Q2;  // one staging buffer
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *ph_s = (float2 *)smem_raw;  // TYPE_P: pre [4 j][4 i], post [4 j]; TYPE_X: pre [4 i], post [4 j][4 i]
  float2 *io_s = ph_s + 20 * Q2;      // [2][4][RS][Q2]
  float2 *z_s = io_s + 2 * SUB;       // [4][2][RS][Q2]
  float2 *pre_s = ph_s;
  float2 *post_s = TYPE_P ? ph_s + 16 * Q2 : ph_s + 4 * Q2;
  const int l = g.l, lb = g.L - g.l, e = g.e;
  const UnitIdx d = unit_decode(bx_, l, lb, e);
  const int r0 = by_ * kRMax;
  const int rc = min(kRMax, g.nrhs - r0);
  const int nsub = (rc + RS - 1) / RS;
  const long long nrq = (long long)g.nrhs * Q2;
  // inputs come from the children of B (forward) or of A (conjugate transposes)
  auto in_pair = [&](int i) { return FWD ? pair_child_b(d, i, lb, e) : pair_child_a(d, i, l, lb, e); };
  auto out_pair = [&](int j) { return FWD ? pair_child_a(d, j, l, lb, e) : pair_child_b(d, j, lb, e); };
  auto issue = [&](int k) {
    if (k < nsub) {
      const int rs0 = k * RS, rs = min(RS, rc - rs0);
      float2 *buf = io_s + (k & 1) * SUB;
#pragma unroll
      for (int i = 0; i < 4; i++)
        cp_async_run(buf + i * RS * Q2, in + in_pair(i) * nrq + (long long)(r0 + rs0) * Q2, rs * Q2);
    }
    cp_async_commit();
  };
  issue(0);
  issue(1);

  // phase factors of the unit, shared by all right-hand sides (scratch: z_s)
  if (TYPE_P && FWD) {  // pre[j=sigma][i=c] = ec[sigma][c], post[j=sigma] = conj ep[sigma]
    family_centres<Q>(tb, tf, ph, d, l, lb, pre_s, post_s, (unsigned char *)z_s);
    for (int idx = threadIdx.x; idx < 4 * Q2; idx += blockDim.x) post_s[idx] = conjf2(post_s[idx]);
  } else if (TYPE_P) {  // pre[j=c][i=sigma] = conj ea[sigma][c], post[j=c] = eq[c]
    float2 *ea = z_s;
    family_nodes<Q>(tb, tf, ph, d, l, lb, ea, post_s, (unsigned char *)(z_s + 16 * Q2));
    for (int idx = threadIdx.x; idx < 16 * Q2; idx += blockDim.x) {
      const int sg = idx / (4 * Q2), c = (idx / Q2) & 3, t = idx % Q2;
      pre_s[(c * 4 + sg) * Q2 + t] = conjf2(ea[idx]);
    }
  } else if (FWD) {  // pre[i=c] = conj eq[c], post[j=sigma][i=c] = ea[sigma][c]
    family_nodes<Q>(tb, tf, ph, d, l, lb, post_s, pre_s, (unsigned char *)z_s);
    for (int idx = threadIdx.x; idx < 4 * Q2; idx += blockDim.x) pre_s[idx] = conjf2(pre_s[idx]);
  } else {  // pre[i=sigma] = ep[sigma], post[j=c][i=sigma] = conj ec[sigma][c]
    float2 *ec = z_s;
    family_centres<Q>(tb, tf, ph, d, l, lb, ec, pre_s, (unsigned char *)(z_s + 16 * Q2));
    for (int idx = threadIdx.x; idx < 16 * Q2; idx += blockDim.x) {
      const int sg = idx / (4 * Q2), c = (idx / Q2) & 3, u = idx % Q2;
      post_s[(c * 4 + sg) * Q2 + u] = conjf2(ec[idx]);
    }
  }

  for (int k = 0; k < nsub; k++) {
    const int rs0 = k * RS, rs = min(RS, rc - rs0);
    float2 *io = io_s + (k & 1) * SUB;
    cp_async_wait(k + 1 < nsub);
    __syncthreads();
    if (TYPE_P) {
      // Z_{j,i1}[t'1][t2] = sum_{i2,t'2} T^{i2}[t2][t'2] (pre (.) in)_{(i1,i2)}[t'1][t'2]
      for (int task = threadIdx.x; task < 8 * RS * Q; task += blockDim.x) {
        const int tp1 = task % Q, r = (task / Q) % RS, i1 = (task / (Q * RS)) & 1, j = task / (2 * Q * RS);
        if (r >= rs) continue;
        float2 sv[2][Q];
#pragma unroll
        for (int i2 = 0; i2 < 2; i2++)
#pragma unroll
          for (int tp2 = 0; tp2 < Q; tp2++) {
            const int i = i1 * 2 + i2;
            sv[i2][tp2] = cmul(pre_s[(j * 4 + i) * Q2 + tp1 * Q + tp2], io[(i * RS + r) * Q2 + tp1 * Q + tp2]);
          }
        float2 *zrow = z_s + ((j * 2 + i1) * RS + r) * Q2 + tp1 * Q;
#pragma unroll
        for (int t2 = 0; t2 < Q; t2++) {
          float2 acc = make_float2(0.f, 0.f);
#pragma unroll
          for (int i2 = 0; i2 < 2; i2++)
#pragma unroll
            for (int tp2 = 0; tp2 < Q; tp2++) acc = fma2s(tm.T[i2][t2][tp2], sv[i2][tp2], acc);
          zrow[t2] = acc;
        }
      }
      __syncthreads();
      // Y_j[t1][t2] = sum_{i1,t'1} T^{i1}[t1][t'1] Z_{j,i1}[t'1][t2];  out_j = post_j (.) Y_j  -> io
      for (int task = threadIdx.x; task < 4 * RS * Q; task += blockDim.x) {
        const int t2 = task % Q, r = (task / Q) % RS, j = task / (Q * RS);
        if (r >= rs) continue;
        float2 zc[2][Q];
#pragma unroll
        for (int i1 = 0; i1 < 2; i1++)
#pragma unroll
          for (int tp1 = 0; tp1 < Q; tp1++) zc[i1][tp1] = z_s[((j * 2 + i1) * RS + r) * Q2 + tp1 * Q + t2];
#pragma unroll
        for (int t1 = 0; t1 < Q; t1++) {
          float2 acc = make_float2(0.f, 0.f);
#pragma unroll
          for (int i1 = 0; i1 < 2; i1++)
#pragma unroll
            for (int tp1 = 0; tp1 < Q; tp1++) acc = fma2s(tm.T[i1][t1][tp1], zc[i1][tp1], acc);
          io[(j * RS + r) * Q2 + t1 * Q + t2] = cmul(post_s[j * Q2 + t1 * Q + t2], acc);
        }
      }
    } else {
      // W_{i,j1}[t1][t'2] = sum_{t'1} T^{j1}[t'1][t1] (pre_i (.) in_i)[t'1][t'2], both j1 per task
      for (int task = threadIdx.x; task < 4 * RS * Q; task += blockDim.x) {
        const int tp2 = task % Q, r = (task / Q) % RS, i = task / (Q * RS);
        if (r >= rs) continue;
        float2 col[Q];
#pragma unroll
        for (int tp1 = 0; tp1 < Q; tp1++)
          col[tp1] = cmul(pre_s[i * Q2 + tp1 * Q + tp2], io[(i * RS + r) * Q2 + tp1 * Q + tp2]);
#pragma unroll
        for (int j1 = 0; j1 < 2; j1++) {
          float2 *wb = z_s + ((i * 2 + j1) * RS + r) * Q2 + tp2;
#pragma unroll
          for (int t1 = 0; t1 < Q; t1++) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int tp1 = 0; tp1 < Q; tp1++) acc = fma2s(tm.T[j1][tp1][t1], col[tp1], acc);
            wb[t1 * Q] = acc;
          }
        }
      }
      __syncthreads();
      // out_j[t1][t2] = sum_i post_{j,i}[t1][t2] sum_{t'2} T^{j2}[t'2][t2] W_{i,j1}[t1][t'2]  -> io.
      // A task is (j1, r, t1, half): both j2 and two of the four i; the lane pair
      // (half = 0, 1) exchanges partial sums so that half h finishes j2 = h.
      constexpr int NT = 4 * RS * Q, NTW = (NT + 31) / 32 * 32;  // whole warps take part in the shuffles
      for (int tw = threadIdx.x; tw < NTW; tw += blockDim.x) {
        const int task = tw < NT ? tw : NT - 2 + (tw & 1);
        const int half = task & 1, t1 = (task >> 1) % Q, r = (task >> 1) / Q % RS, j1 = (task >> 1) / (Q * RS);
        const bool live = tw < NT && r < rs;
        float ax[2][Q], ay[2][Q];
#pragma unroll
        for (int j2 = 0; j2 < 2; j2++)
#pragma unroll
          for (int t2 = 0; t2 < Q; t2++) ax[j2][t2] = ay[j2][t2] = 0.f;
        if (live) {
#pragma unroll 1
          for (int ii = 0; ii < 2; ii++) {
            const int i = 2 * half + ii;
            float2 row[Q];
#pragma unroll
            for (int tp2 = 0; tp2 < Q; tp2++) row[tp2] = z_s[((i * 2 + j1) * RS + r) * Q2 + t1 * Q + tp2];
#pragma unroll
            for (int j2 = 0; j2 < 2; j2++) {
              const float2 *pp = post_s + ((2 * j1 + j2) * 4 + i) * Q2 + t1 * Q;
#pragma unroll
              for (int t2 = 0; t2 < Q; t2++) {
                float2 v = make_float2(0.f, 0.f);
#pragma unroll
                for (int tp2 = 0; tp2 < Q; tp2++) v = fma2s(tm.T[j2][tp2][t2], row[tp2], v);
                const float vx = v.x, vy = v.y;
                const float2 p = pp[t2];
                ax[j2][t2] = __fmaf_rn(p.x, vx, __fmaf_rn(-p.y, vy, ax[j2][t2]));
                ay[j2][t2] = __fmaf_rn(p.x, vy, __fmaf_rn(p.y, vx, ay[j2][t2]));
              }
            }
          }
        }
        float2 *dst = io + ((2 * j1 + half) * RS + r) * Q2 + t1 * Q;  // staged inputs were last read in the W pass
#pragma unroll
        for (int t2 = 0; t2 < Q; t2++) {
          const float sx = half ? ax[0][t2] : ax[1][t2], sy = half ? ay[0][t2] : ay[1][t2];
          const float mx = half ? ax[1][t2] : ax[0][t2], my = half ? ay[1][t2] : ay[0][t2];
          const float ox = __shfl_xor_sync(0xffffffffu, sx, 1), oy = __shfl_xor_sync(0xffffffffu, sy, 1);
          if (live) dst[t2] = make_float2(mx + ox, my + oy);
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; j++) store_run(out + out_pair(j) * nrq + (long long)(r0 + rs0) * Q2, io + j * RS * Q2, rs * Q2);
    __syncthreads();
    issue(k + 2);
  }
}
template <int Q, bool TYPE_P, bool FWD, int RS>
__global__ void __launch_bounds__(TransShape<Q, RS>::threads, TransShape<Q, RS>::min_blocks)
    k32_trans(Tables tb, TablesF tf, Phase ph, Geom g, TMat<float, Q> tm, const float2 *__restrict__ in,
              float2 *__restrict__ out) {
  k32_trans_body<Q, TYPE_P, FWD, RS>(tb, tf, ph, g, tm, in, out, blockIdx.x, blockIdx.y);
}

// e^{2 pi i theta(x, p)} for the FP32 form: x by its two 1D node entries (FP64 and df
// copies), p by its polar node entries.  Homogeneous phases go through df
// arithmetic; the separable test phase through FP64.
__device__ __forceinline__ float2 e32(const Phase &ph, const TablesF &tf, const XNode &x1, const XNode &x2,
                                      const XNodeF &f1, const XNodeF &f2, const P1Node &u, const P2Node &v,
                                      const df &rho, const P2NodeF &vf) {
  if (ph.id == 3) return expi<float>(theta_xp(ph, x1, x2, u, v));
  return expi_df(df_mul(rho, g_eval(tf.ph, xdesc(tf.ph, f1, f2), vf)));
}
// e^{2 pi i Phi(x, k)} at a lattice source.
__device__ __forceinline__ float2 e32k(const Phase &ph, const TablesF &tf, const XNode &x1, const XNode &x2,
                                       const XNodeF &f1, const XNodeF &f2, const Src &k, const SrcF &kf) {
  if (ph.id == 3) return expi<float>(theta_xk(ph, x1, x2, k));
  return expi_df(theta_k(tf.ph, xdesc(tf.ph, f1, f2), kf.k1, kf.k2));
}

// Shape of the FP32 switch CTA: a contraction task owns 4 output rows x 4 RHS,
// 8 RHS groups cover 32 RHS, so ceil(q^2/4) * 8 tasks (rounded up to whole warps).
template <int Q> struct SwShape {
  static constexpr int Q2 = Q * Q;
  static constexpr int NOG = (Q2 + 3) / 4;
  static constexpr int threads = ((NOG * 8 + 31) / 32) * 32;
};
// Dynamic shared memory of k32_switch for q: input/output block, kernel matrix (real
// and imaginary parts, q^2 x q^2 rounded up to 4 columns), rho.
__host__ __device__ constexpr int sw32_smem_bytes(int q) {
  return kRMax * q * q * 8 + 2 * q * q * ((q * q + 3) / 4 * 4) * 4 + q * (int)sizeof(df);
}

// e^{2 pi i theta} from a df theta through the special-function unit: exact
// reduction of hi, then __sincosf of 2 pi r, |2 pi r| <= pi (absolute error below
// 1e-6 per factor; used for the q^4 factors of the switch).
__device__ __forceinline__ float2 expi_df_sfu(df th) {
  const float r = (th.h - rintf(th.h)) + th.l;
  float sn, cs;
  __sincosf(6.28318530717958647692f * r, &sn, &cs);
  return make_float2(cs, sn);
}

// out[r][o] = sum_i K[o][i] in[r][i] for o < q^2, r < rc.  The kernel sits in shared
// memory transposed and split into real and imaginary float arrays kre/kim[i][OP]
// (OP = q^2 rounded up to a multiple of 4, zero rows beyond q^2); the inputs keep
// their HBM layout in_s[r][i] (complex).  A task owns rows o = 4 og + a (a < 4) and
// RHS r = rg + nrg c (c < 4); accumulators hold row pairs (o, o+1), so a complex MAC
// over two rows is four paired FMAs (FFMA2) with the input broadcast, and the lanes
// of a warp read 4 distinct kernel row pairs and 8 distinct input rows (distinct
// banks) per step.  With few RHS the inner sum is split into KS contiguous ranges
// over consecutive lanes, combined with shuffles.
template <int Q> struct SwLayout {
  static constexpr int Q2 = Q * Q;
  static constexpr int OP = (Q2 + 3) / 4 * 4;
};
template <int Q, int KS, int RB>
__device__ __forceinline__ void sw_contract(const float *kre, const float *kim, const float2 *in_s, int rc, int task,
                                            float2 (&ax)[2][RB], float2 (&ay)[2][RB], int &og, int &rg, int &nrg,
                                            bool &live) {
  constexpr int Q2 = Q * Q, OP = SwLayout<Q>::OP;
  constexpr int NOG = SwShape<Q>::NOG;
  constexpr int CH = (Q2 + KS - 1) / KS;
  nrg = (rc + RB - 1) / RB;
  live = task < NOG * nrg * KS;
  const int ks = task % KS, grp = task / KS;
  rg = grp % nrg;
  og = min(grp / nrg, NOG - 1);
#pragma unroll
  for (int h = 0; h < 2; h++)
#pragma unroll
    for (int c_ = 0; c_ < RB; c_++) ax[h][c_] = ay[h][c_] = make_float2(0.f, 0.f);
  int rr[RB];
#pragma unroll
  for (int c_ = 0; c_ < RB; c_++) rr[c_] = min(rg + nrg * c_, rc - 1);
  if (live) {
    const int i1 = min(Q2, (ks + 1) * CH);
    const float *kr = kre + og * 4, *ki = kim + og * 4;
#pragma unroll 3
    for (int i = ks * CH; i < i1; i++) {
      const float2 r01 = *reinterpret_cast<const float2 *>(kr + i * OP);
      const float2 r23 = *reinterpret_cast<const float2 *>(kr + i * OP + 2);
      const float2 m01 = *reinterpret_cast<const float2 *>(ki + i * OP);
      const float2 m23 = *reinterpret_cast<const float2 *>(ki + i * OP + 2);
      float2 iv[RB];
#pragma unroll
      for (int c_ = 0; c_ < RB; c_++) iv[c_] = in_s[rr[c_] * Q2 + i];
#pragma unroll
      for (int c_ = 0; c_ < RB; c_++) {
        const float2 X = make_float2(iv[c_].x, iv[c_].x), Y = make_float2(iv[c_].y, iv[c_].y);
        const float2 NY = make_float2(-iv[c_].y, -iv[c_].y);
        ax[0][c_] = __ffma2_rn(r01, X, ax[0][c_]);
        ax[0][c_] = __ffma2_rn(m01, NY, ax[0][c_]);
        ay[0][c_] = __ffma2_rn(r01, Y, ay[0][c_]);
        ay[0][c_] = __ffma2_rn(m01, X, ay[0][c_]);
        ax[1][c_] = __ffma2_rn(r23, X, ax[1][c_]);
        ax[1][c_] = __ffma2_rn(m23, NY, ax[1][c_]);
        ay[1][c_] = __ffma2_rn(r23, Y, ay[1][c_]);
        ay[1][c_] = __ffma2_rn(m23, X, ay[1][c_]);
      }
    }
  }
#pragma unroll
  for (int m = 1; m < KS; m <<= 1)
#pragma unroll
    for (int h = 0; h < 2; h++)
#pragma unroll
      for (int c_ = 0; c_ < RB; c_++) {
        ax[h][c_].x += __shfl_xor_sync(0xffffffffu, ax[h][c_].x, m);
        ax[h][c_].y += __shfl_xor_sync(0xffffffffu, ax[h][c_].y, m);
        ay[h][c_].x += __shfl_xor_sync(0xffffffffu, ay[h][c_].x, m);
        ay[h][c_].y += __shfl_xor_sync(0xffffffffu, ay[h][c_].y, m);
      }
  live = live && ks == 0;
}

// Pair index -> (A, B) box coordinates at the switch level.
struct SwPair {
  int a1, a2, b1, b2;
};
__device__ __forceinline__ SwPair sw_decode(const Geom &g, long long pr) {
  const int l = g.l, lb = g.L - g.l;
  const int nb2 = 1 << (lb + g.e);
  const long long nBl = (1LL << lb) * nb2;
  const long long a = pr / nBl, b = pr - a * nBl;
  SwPair d;
  d.a1 = (int)(a >> l);
  d.a2 = (int)(a & ((1LL << l) - 1));
  d.b1 = (int)(b / nb2);
  d.b2 = (int)(b - (long long)d.b1 * nb2);
  return d;
}

// The kernel matrix of pair d into kre/kim[i][o] (transposed; rows o < q^2, the
// pad rows are left alone), by nthr threads (this one is tid); sync() orders rho_s
// before its use.
template <int Q, bool FWD, typename Sync>
__device__ __forceinline__ void sw_fill(const Tables &tb, const TablesF &tf, const Phase &ph, const Geom &g,
                                        const SwPair &d, float *kre, float *kim, df *rho_s, int tid, int nthr,
                                        Sync &&sync) {
  constexpr int Q2 = Q * Q, OP = SwLayout<Q>::OP;
  const int l = g.l, lb = g.L - g.l;
  if (ph.id == 3) {
    for (int idx = tid; idx < Q2 * Q2; idx += nthr) {
      const int i = idx / Q2, o = idx % Q2;
      const int t = FWD ? o : i, s = FWD ? i : o;
      float2 v = expi<float>(theta_xp(ph, xn(tb, l, d.a1, t / Q, Q), xn(tb, l, d.a2, t % Q, Q),
                                      pn1(tb, lb, d.b1, s / Q, Q), pn2(tb, lb, d.b2, s % Q, Q)));
      kre[i * OP + o] = v.x;
      kim[i * OP + o] = FWD ? v.y : -v.y;
    }
    return;
  }
  for (int t = tid; t < Q; t += nthr) rho_s[t] = rhof(tb, tf, lb, d.b1, t, Q);
  sync();
  // theta(x_t, p_s) = rho(s1) G(x_t, p2_{s2}): one G per (t, s2), q products each
  for (int task = tid; task < Q2 * Q; task += nthr) {
    const int t = FWD ? task % Q2 : task / Q, s2 = FWD ? task / Q2 : task % Q;
    const XDesc xdt = xdesc(tf.ph, xnf(tb, tf, l, d.a1, t / Q, Q), xnf(tb, tf, l, d.a2, t % Q, Q));
    const df G = g_eval(tf.ph, xdt, p2f(tb, tf, lb, d.b2, s2, Q));
#pragma unroll
    for (int s1 = 0; s1 < Q; s1++) {
      const float2 v = expi_df_sfu(df_mul(rho_s[s1], G));
      const int s = s1 * Q + s2;
      const int at = FWD ? s * OP + t : t * OP + s;  // K[o = t][i = s] or K[o = s][i = t] = conj
      kre[at] = v.x;
      kim[at] = FWD ? v.y : -v.y;
    }
  }
}
// Zero the pad rows o >= q^2 of a kernel buffer.
template <int Q> __device__ __forceinline__ void sw_zero_pad(float *kre, float *kim, int tid, int nthr) {
  constexpr int Q2 = Q * Q, OP = SwLayout<Q>::OP;
  for (int idx = tid; idx < Q2 * (OP - Q2); idx += nthr) {
    const int i = idx / (OP - Q2), o = Q2 + idx % (OP - Q2);
    kre[i * OP + o] = 0.f;
    kim[i * OP + o] = 0.f;
  }
}
// Contraction by nthr threads (this one is task) into registers, then -- after
// sync(), when no thread reads in_s any more -- the results into in_s as [r][o].
template <int Q, int RB, typename Sync>
__device__ __forceinline__ void sw_contract_store(const float *kre, const float *kim, float2 *in_s, int rc, int task,
                                                     int nthr, Sync &&sync) {
  constexpr int Q2 = Q * Q;
  constexpr int NOG = SwShape<Q>::NOG;
  const int nrg0 = (rc + RB - 1) / RB;
  float2 ax[2][RB], ay[2][RB];
  int og, rg, nrg;
  bool live;
  if (NOG * nrg0 * 8 <= nthr) sw_contract<Q, 8, RB>(kre, kim, in_s, rc, task, ax, ay, og, rg, nrg, live);
  else if (NOG * nrg0 * 4 <= nthr) sw_contract<Q, 4, RB>(kre, kim, in_s, rc, task, ax, ay, og, rg, nrg, live);
  else if (NOG * nrg0 * 2 <= nthr) sw_contract<Q, 2, RB>(kre, kim, in_s, rc, task, ax, ay, og, rg, nrg, live);
  else sw_contract<Q, 1, RB>(kre, kim, in_s, rc, task, ax, ay, og, rg, nrg, live);
  sync();
  if (live) {
#pragma unroll
    for (int h = 0; h < 2; h++)
#pragma unroll
      for (int c_ = 0; c_ < RB; c_++) {
        const int o = og * 4 + 2 * h, r = rg + nrg * c_;
        if (r < rc) {
          if (o < Q2) in_s[r * Q2 + o] = make_float2(ax[h][c_].x, ay[h][c_].x);
          if (o + 1 < Q2) in_s[r * Q2 + o + 1] = make_float2(ax[h][c_].y, ay[h][c_].y);
        }
      }
  }
}


// ---------------------------------------------------------------------------
// FP32 switch (eq. alg2m): one CTA per pair (A, B) at level lm and up to 32 RHS.
//   FWD : out[t] = sum_s e(x^A_t, p^B_s) in[s];   !FWD: out[s] = sum_t conj e(x^A_t, p^B_s) in[t].
// theta(x_t, p_s) = rho(s1) G(x_t, p2_{s2}): q^3 evaluations of G, q^4 products.
// The input block arrives by cp.async while the kernel matrix is generated.
// ---------------------------------------------------------------------------
template <int Q, bool FWD, int RB = 4>
__device__ __forceinline__ void k32_switch_body(const Tables &tb, const TablesF &tf, const Phase &ph, const Geom &g,
                                                const float2 *__restrict__ in, float2 *__restrict__ out, long long bx_, int by_) {
  constexpr int Q2 = Q * Q, OP = SwLayout<Q>::OP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *in_s = (float2 *)smem_raw;          // [kRMax][Q2]: inputs, then outputs (16-byte aligned)
  float *kre = (float *)(in_s + kRMax * Q2);  // [Q2 in i][OP out o]
  float *kim = kre + Q2 * OP;                 // [Q2 in i][OP out o]
  df *rho_s = (df *)(kim + Q2 * OP);          // [Q]
  const long long pr = bx_;
  const int r0 = by_ * kRMax;
  const int rc = min(kRMax, g.nrhs - r0);
  const long long nrq = (long long)g.nrhs * Q2;
  cp_async_run(in_s, in + pr * nrq + (long long)r0 * Q2, rc * Q2);
  cp_async_commit();
  sw_zero_pad<Q>(kre, kim, threadIdx.x, blockDim.x);
  sw_fill<Q, FWD>(tb, tf, ph, g, sw_decode(g, pr), kre, kim, rho_s, threadIdx.x, blockDim.x, []() { __syncthreads(); });
  cp_async_wait(0);
  __syncthreads();
  sw_contract_store<Q, RB>(kre, kim, in_s, rc, threadIdx.x, blockDim.x, []() { __syncthreads(); });
  __syncthreads();
  store_run(out + pr * nrq + (long long)r0 * Q2, in_s, rc * Q2);
}
template <int Q, bool FWD, int RB>
__global__ void __launch_bounds__(SwShape<Q>::threads, RB == 4 ? 3 : 2)
    k32_switch(Tables tb, TablesF tf, Phase ph, Geom g, const float2 *__restrict__ in, float2 *__restrict__ out) {
  k32_switch_body<Q, FWD, RB>(tb, tf, ph, g, in, out, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// Warp-specialised persistent FP32 switch: producer warps build the kernel matrix
// of the CTA's next work item (and start its input copy) while consumer warps
// contract the current one.  Two kernel/input buffers; hardware named barriers
// hand them over (FULL_b: producers -> consumers, EMPTY_b: consumers -> producers).
// Work item w = pair * nry + RHS tile; CTA c takes w = c, c + gridDim.x, ...
// ---------------------------------------------------------------------------
template <int Q> struct SwWs {
  static constexpr int Q2 = Q * Q, OP = SwLayout<Q>::OP;
  static constexpr int cons = SwShape<Q>::threads;   // consumer threads
  static constexpr int prod = SwShape<Q>::threads;   // producer threads
  static constexpr int threads = cons + prod;
  static constexpr int kfloats = 2 * Q2 * OP;        // one kernel buffer (re, im)
  static constexpr int ifloat2 = kRMax * Q2;         // one input/output buffer
  static constexpr int smem = 2 * (kfloats * 4 + ifloat2 * 8) + 2 * Q * 8;
};
enum { kBarFull0 = 1, kBarEmpty0 = 3, kBarProd = 5, kBarCons = 6 };
__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void named_arrive(int id, int n) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

template <int Q, bool FWD>
__global__ void __launch_bounds__(SwWs<Q>::threads, 1) k32_switch_ws(Tables tb, TablesF tf, Phase ph, Geom g,
                                                                    const float2 *__restrict__ in,
                                                                    float2 *__restrict__ out, long long nwork) {
  using W = SwWs<Q>;
  constexpr int Q2 = Q * Q, OP = W::OP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *ibuf = (float2 *)smem_raw;                     // [2][kRMax][Q2]
  float *kbuf = (float *)(ibuf + 2 * W::ifloat2);        // [2][re, im][Q2][OP]
  df *rho = (df *)(kbuf + 2 * W::kfloats);               // [2][Q]
  const int nry = (g.nrhs + kRMax - 1) / kRMax;
  const long long nrq = (long long)g.nrhs * Q2;
  const long long nstage = blockIdx.x < nwork ? (nwork - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  if (threadIdx.x < W::prod) {
    const int tid = threadIdx.x;
    for (long long s = 0; s < nstage; s++) {
      const int b = (int)(s & 1);
      const long long w = blockIdx.x + s * gridDim.x;
      const long long pr = w / nry;
      const int r0 = (int)(w % nry) * kRMax, rc = min(kRMax, g.nrhs - r0);
      float *kre = kbuf + b * W::kfloats, *kim = kre + Q2 * OP;
      if (s >= 2) named_sync(kBarEmpty0 + b, W::threads);
      else sw_zero_pad<Q>(kre, kim, tid, W::prod);
      cp_async_run(ibuf + b * W::ifloat2, in + pr * nrq + (long long)r0 * Q2, rc * Q2, tid, W::prod);
      cp_async_commit();
      sw_fill<Q, FWD>(tb, tf, ph, g, sw_decode(g, pr), kre, kim, rho + b * Q, tid, W::prod,
                      []() { named_sync(kBarProd, W::prod); });
      cp_async_wait(0);
      named_arrive(kBarFull0 + b, W::threads);
    }
  } else {
    const int task = threadIdx.x - W::prod;
    for (long long s = 0; s < nstage; s++) {
      const int b = (int)(s & 1);
      const long long w = blockIdx.x + s * gridDim.x;
      const long long pr = w / nry;
      const int r0 = (int)(w % nry) * kRMax, rc = min(kRMax, g.nrhs - r0);
      const float *kre = kbuf + b * W::kfloats, *kim = kre + Q2 * OP;
      float2 *io = ibuf + b * W::ifloat2;
      named_sync(kBarFull0 + b, W::threads);
      sw_contract_store<Q, 4>(kre, kim, io, rc, task, W::cons, []() { named_sync(kBarCons, W::cons); });
      named_sync(kBarCons, W::cons);
      store_run(out + pr * nrq + (long long)r0 * Q2, io, rc * Q2, task, W::cons);
      if (s + 2 < nstage) named_arrive(kBarEmpty0 + b, W::threads);
    }
  }
}

// ---------------------------------------------------------------------------
// FP32 initialization (eq. alg2a), as k_init with df phases; one CTA per box B and
// up to 32 RHS; the phases of GA boxes A are staged at a time, then each thread
// accumulates one (RHS, t1) row for every A of the chunk.  With use_stage (shared room
// for one kRMax q^2 output block after the tables) and a full 32-RHS tile, each block
// (A, B) goes through shared memory and leaves as one contiguous run: a bulk copy by the
// TMA engine where the run is 16-byte aligned (an even RHS count), else 16-byte stores.
// Otherwise each thread stores its row directly (9 values at a 72-byte stride per lane).
// ---------------------------------------------------------------------------
template <int Q>
__device__ __forceinline__ void k32_init_body(const Tables &tb, const TablesF &tf, const Phase &ph, const Geom &g, int maxsrc, int GA,
                                              const float2 *__restrict__ f, float2 *__restrict__ st, long long bx_, int by_,
                                              bool use_stage = false) {
  constexpr int Q2 = Q * Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int l0 = g.l, lb = g.L - g.l, e = g.e;
  const int box = bx_;
  const int nb2 = 1 << (lb + e);
  const int b1 = box / nb2, b2 = box % nb2;
  const int r0 = by_ * kRMax;
  const int rt = min(kRMax, g.nrhs - r0);
  const int j0 = tb.box_off[box], ns = tb.box_off[box + 1] - j0;
  const long long NN = 1LL << (2 * g.L);
  float2 *fv = (float2 *)smem_raw;     // [maxsrc][kRMax]
  float2 *pk = fv + maxsrc * kRMax;    // [GA][maxsrc]
  float2 *post = pk + GA * maxsrc;     // [GA][Q2]
  float *w = (float *)(post + GA * Q2);  // [maxsrc][2Q]
  XDesc *xds = (XDesc *)(w + maxsrc * 2 * Q);  // [GA]: x-side data of the centre x0(A) of each A
  df *gtab = (df *)(xds + GA);                 // [GA][Q]: G(x0(A), p2 node t2 of B)
  float2 *stage = (float2 *)(((uintptr_t)(gtab + GA * Q) + 15) & ~(uintptr_t)15);  // [kRMax][Q2]
  const bool staged = use_stage && rt == kRMax && (int)blockDim.x == kRMax * Q;
  const bool bulk = staged && ((g.nrhs * Q2) & 1) == 0;
  for (int idx = threadIdx.x; idx < ns * rt; idx += blockDim.x) {
    const int j = idx / rt, r = idx % rt;
    fv[j * kRMax + r] = f[(long long)(r0 + r) * NN + tb.src_f[j0 + j]];
  }
  for (int idx = threadIdx.x; idx < ns * 2 * Q; idx += blockDim.x) w[idx] = (float)tb.src_w[(long long)j0 * 2 * Q + idx];
  const int nA1 = 1 << l0, nA = nA1 * nA1;
  const long long nB = (1LL << lb) * nb2;
  const long long nrq = (long long)g.nrhs * Q2;
  for (int A0 = 0; A0 < nA; A0 += GA) {
    const int ga_n = min(GA, nA - A0);
    __syncthreads();
    if (ph.id == 3) {  // separable phase: theta straight from the node coordinates
      for (int idx = threadIdx.x; idx < ga_n * (ns + Q2); idx += blockDim.x) {
        const int ga = idx / (ns + Q2), k = idx % (ns + Q2);
        const int A = A0 + ga, a1 = A >> l0, a2 = A & (nA1 - 1);
        const XNode &x1 = xn(tb, l0, a1, Q, Q), &x2 = xn(tb, l0, a2, Q, Q);
        const XNodeF &f1 = xnf(tb, tf, l0, a1, Q, Q), &f2 = xnf(tb, tf, l0, a2, Q, Q);
        if (k < ns) {
          pk[ga * maxsrc + k] = e32k(ph, tf, x1, x2, f1, f2, tb.src[j0 + k], tf.src[j0 + k]);
        } else {
          const int t = k - ns;
          post[ga * Q2 + t] = conjf2(e32(ph, tf, x1, x2, f1, f2, pn1(tb, lb, b1, t / Q, Q), pn2(tb, lb, b2, t % Q, Q),
                                         rhof(tb, tf, lb, b1, t / Q, Q), p2f(tb, tf, lb, b2, t % Q, Q)));
        }
      }
    } else {
      // homogeneous phase: the x-side data of each x0(A) once, then the source phases
      // theta(x0(A), k) and G(x0(A), p2_t2) (q per A), then the q^2 post factors
      // e^{-2 pi i rho(p1_t1) G(x0(A), p2_t2)} as products
      for (int ga = threadIdx.x; ga < ga_n; ga += blockDim.x) {
        const int A = A0 + ga, a1 = A >> l0, a2 = A & (nA1 - 1);
        xds[ga] = xdesc(tf.ph, xnf(tb, tf, l0, a1, Q, Q), xnf(tb, tf, l0, a2, Q, Q));
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < ga_n * (ns + Q); idx += blockDim.x) {
        const int ga = idx / (ns + Q), k = idx % (ns + Q);
        if (k < ns) {
          const SrcF &kf = tf.src[j0 + k];
          pk[ga * maxsrc + k] = expi_df(theta_k(tf.ph, xds[ga], kf.k1, kf.k2));
        } else {
          gtab[ga * Q + k - ns] = g_eval(tf.ph, xds[ga], p2f(tb, tf, lb, b2, k - ns, Q));
        }
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < ga_n * Q2; idx += blockDim.x) {
        const int ga = idx / Q2, t = idx % Q2;
        post[ga * Q2 + t] = conjf2(expi_df(df_mul(rhof(tb, tf, lb, b1, t / Q, Q), gtab[ga * Q + t % Q])));
      }
    }
    __syncthreads();
    // thread (r, t1) sums the row t1 of boxes A of the chunk (no barrier inside); with
    // fewer than kRMax RHS the threads split into groups that take different A
    const int per = rt * Q, ngrp = blockDim.x / per;
    const int r = (threadIdx.x % per) / Q, t1 = threadIdx.x % Q;
    if (staged) {  // every thread is one (r, t1) row; all take every A of the chunk in turn
      for (int ga = 0; ga < ga_n; ga++) {
        float2 acc[Q];
#pragma unroll
        for (int t2 = 0; t2 < Q; t2++) acc[t2] = make_float2(0.f, 0.f);
        for (int j = 0; j < ns; j++) {
          const float2 v = cmul(pk[ga * maxsrc + j], fv[j * kRMax + r]);
          const float w1 = w[j * 2 * Q + t1];
          const float2 h = __fmul2_rn(make_float2(w1, w1), v);
#pragma unroll
          for (int t2 = 0; t2 < Q; t2++) acc[t2] = fma2s(w[j * 2 * Q + Q + t2], h, acc[t2]);
        }
        if (bulk && threadIdx.x == 0) bulk_wait_read0();  // the previous block's copy has read the stage
        __syncthreads();
#pragma unroll
        for (int t2 = 0; t2 < Q; t2++) stage[r * Q2 + t1 * Q + t2] = cmul(post[ga * Q2 + t1 * Q + t2], acc[t2]);
        if (bulk) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        float2 *dst = st + ((long long)(A0 + ga) * nB + box) * nrq + (long long)r0 * Q2;
        if (bulk) {
          if (threadIdx.x == 0) {
            bulk_s2g(dst, stage, (uint32_t)(kRMax * Q2 * 8));
            bulk_commit();
          }
        } else {
          store_run(dst, stage, kRMax * Q2);
        }
      }
    } else if (threadIdx.x < ngrp * per) {
      for (int ga = threadIdx.x / per; ga < ga_n; ga += ngrp) {
        float2 acc[Q];
#pragma unroll
        for (int t2 = 0; t2 < Q; t2++) acc[t2] = make_float2(0.f, 0.f);
        for (int j = 0; j < ns; j++) {
          const float2 v = cmul(pk[ga * maxsrc + j], fv[j * kRMax + r]);
          const float w1 = w[j * 2 * Q + t1];
          const float2 h = __fmul2_rn(make_float2(w1, w1), v);
#pragma unroll
          for (int t2 = 0; t2 < Q; t2++) acc[t2] = fma2s(w[j * 2 * Q + Q + t2], h, acc[t2]);
        }
        const int A = A0 + ga;
        float2 *dst = st + ((long long)A * nB + box) * nrq + (long long)(r0 + r) * Q2 + t1 * Q;
#pragma unroll
        for (int t2 = 0; t2 < Q; t2++) dst[t2] = cmul(post[ga * Q2 + t1 * Q + t2], acc[t2]);
      }
    }
  }
  if (bulk && threadIdx.x == 0) bulk_wait0();  // the bulk copies are done before the CTA ends
}
// Initialization CTA: one thread per (RHS, t1) row, kRMax q threads.
template <int Q> struct InitShape {
  static constexpr int threads = kRMax * Q;
};
constexpr int kInitChunk = 16;  // boxes A whose phases are staged together
template <int Q>
__global__ void __launch_bounds__(InitShape<Q>::threads) k32_init(Tables tb, TablesF tf, Phase ph, Geom g, int maxsrc,
                                                                   int GA, const float2 *__restrict__ f,
                                                                   float2 *__restrict__ st, int use_stage) {
  k32_init_body<Q>(tb, tf, ph, g, maxsrc, GA, f, st, blockIdx.x, blockIdx.y, use_stage != 0);
}

// FP32 conjugate transpose of the initialization (see k_init_adj).
template <int Q>
__device__ __forceinline__ void k32_init_adj_body(const Tables &tb, const TablesF &tf, const Phase &ph, const Geom &g, int maxsrc,
                                                  const float2 *__restrict__ st, float2 *__restrict__ fbar, long long bx_, int by_) {
  constexpr int Q2 = Q * Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int l0 = g.l, lb = g.L - g.l, e = g.e;
  const int box = bx_;
  const int nb2 = 1 << (lb + e);
  const int b1 = box / nb2, b2 = box % nb2;
  const int r0 = by_ * kRMax;
  const int rt = min(kRMax, g.nrhs - r0);
  const int j0 = tb.box_off[box], ns = tb.box_off[box + 1] - j0;
  const long long NN = 1LL << (2 * g.L);
  float2 *acc = (float2 *)smem_raw;   // [maxsrc][kRMax]
  float2 *pk = acc + maxsrc * kRMax;  // [maxsrc]
  float2 *pt = pk + maxsrc;           // [Q2]
  float2 *v = pt + Q2;                // [kRMax][Q2]
  float *w = (float *)(v + kRMax * Q2);  // [maxsrc][2Q]
  for (int idx = threadIdx.x; idx < ns * rt; idx += blockDim.x) acc[(idx / rt) * kRMax + idx % rt] = make_float2(0.f, 0.f);
  for (int idx = threadIdx.x; idx < ns * 2 * Q; idx += blockDim.x) w[idx] = (float)tb.src_w[(long long)j0 * 2 * Q + idx];
  const int nA1 = 1 << l0, nA = nA1 * nA1;
  const long long nB = (1LL << lb) * nb2;
  const long long nrq = (long long)g.nrhs * Q2;
  for (int A = 0; A < nA; A++) {
    const int a1 = A >> l0, a2 = A & (nA1 - 1);
    const XNode &x1 = xn(tb, l0, a1, Q, Q), &x2 = xn(tb, l0, a2, Q, Q);
    const XNodeF &f1 = xnf(tb, tf, l0, a1, Q, Q), &f2 = xnf(tb, tf, l0, a2, Q, Q);
    __syncthreads();
    for (int idx = threadIdx.x; idx < ns + Q2; idx += blockDim.x) {
      if (idx < ns) {
        pk[idx] = conjf2(e32k(ph, tf, x1, x2, f1, f2, tb.src[j0 + idx], tf.src[j0 + idx]));
      } else {
        const int t = idx - ns;
        pt[t] = e32(ph, tf, x1, x2, f1, f2, pn1(tb, lb, b1, t / Q, Q), pn2(tb, lb, b2, t % Q, Q),
                    rhof(tb, tf, lb, b1, t / Q, Q), p2f(tb, tf, lb, b2, t % Q, Q));
      }
    }
    __syncthreads();
    const float2 *src = st + ((long long)A * nB + box) * nrq + (long long)r0 * Q2;
    for (int idx = threadIdx.x; idx < rt * Q2; idx += blockDim.x) v[idx] = cmul(pt[idx % Q2], src[idx]);
    __syncthreads();
    for (int task = threadIdx.x; task < ns * rt; task += blockDim.x) {
      const int j = task / rt, r = task % rt;
      const float *w1 = w + j * 2 * Q, *w2 = w1 + Q;
      float px = 0.f, py = 0.f;
#pragma unroll
      for (int t1 = 0; t1 < Q; t1++) {
        float qx = 0.f, qy = 0.f;
#pragma unroll
        for (int t2 = 0; t2 < Q; t2++) {
          const float2 vv = v[r * Q2 + t1 * Q + t2];
          qx = __fmaf_rn(w2[t2], vv.x, qx);
          qy = __fmaf_rn(w2[t2], vv.y, qy);
        }
        px = __fmaf_rn(w1[t1], qx, px);
        py = __fmaf_rn(w1[t1], qy, py);
      }
      const float2 p = cmul(pk[j], make_float2(px, py));
      float2 a_ = acc[j * kRMax + r];
      acc[j * kRMax + r] = make_float2(a_.x + p.x, a_.y + p.y);
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < ns * rt; idx += blockDim.x) {
    const int j = idx / rt, r = idx % rt;
    fbar[(long long)(r0 + r) * NN + tb.src_f[j0 + j]] = acc[j * kRMax + r];
  }
}
template <int Q>
__global__ void __launch_bounds__(256) k32_init_adj(Tables tb, TablesF tf, Phase ph, Geom g, int maxsrc,
                                                     const float2 *__restrict__ st, float2 *__restrict__ fbar) {
  k32_init_adj_body<Q>(tb, tf, ph, g, maxsrc, st, fbar, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// FP32 termination (eq. alg2d): one CTA per box A at level l1 = L - s and up to
// 32 RHS; the boxes B at level s are summed in a fixed order.  Each thread owns
// the accumulators u[r][m1][0..M) of one (r, m1) in registers for the whole sum.
// Per B: y[r][m1][t2] = sum_t1 V[m1][t1] pre_B[t] d[r][t] (thread per (r, t2)),
// then u[r][m1][m2] += post_B[m] sum_t2 V[m2][t2] y[r][m1][t2] (thread per (r, m1)).
// The coefficients of B+1 are copied asynchronously during B.  Needs M = 2^s <= 8.
// blockDim = 32 max(Q, M).
// ---------------------------------------------------------------------------
constexpr int kTermM = 8;
template <int Q>
__device__ __forceinline__ void k32_term_body(const Tables &tb, const TablesF &tf, const Phase &ph, const Geom &g,
                                              const VMat<float, Q> &vm, const float2 *__restrict__ st, float2 *__restrict__ u, long long bx_, int by_) {
  constexpr int Q2 = Q * Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int l = g.l, lb = g.L - g.l, e = g.e;
  const int M = 1 << g.s, M2 = M * M;
  const int A = bx_, nA1 = 1 << l;
  const int a1 = A >> l, a2 = A & (nA1 - 1);
  const int r0 = by_ * kRMax;
  const int rt = min(kRMax, g.nrhs - r0);
  const int nb2 = 1 << (lb + e);
  const int nB = (1 << lb) * nb2;
  const long long NN = 1LL << (2 * g.L);
  const long long nrq = (long long)g.nrhs * Q2;
  float2 *dbuf = (float2 *)smem_raw;         // [2][kRMax][Q2]
  float2 *y = dbuf + 2 * kRMax * Q2;         // [kRMax][kTermM][Q]
  float2 *phb = y + kRMax * kTermM * Q;      // [2][Q2 + M2]: pre then post
  XDesc *xd = (XDesc *)(phb + 2 * (Q2 + kTermM * kTermM));  // [Q2 + M2]
  const bool sep = ph.id == 3;
  if (!sep)
    for (int idx = threadIdx.x; idx < Q2 + M2; idx += blockDim.x) {
      if (idx < Q2) {
        xd[idx] = xdesc(tf.ph, xnf(tb, tf, l, a1, idx / Q, Q), xnf(tb, tf, l, a2, idx % Q, Q));
      } else {
        const int m = idx - Q2;
        xd[idx] = xdesc(tf.ph, tf.xgrid[a1 * M + m / M], tf.xgrid[a2 * M + m % M]);
      }
    }
  // Boxes B are walked angular index first (b2 outer, b1 inner): G(x, p0_2(B)) of the
  // homogeneous phase theta = rho(p0_1) G(x, p0_2) is then evaluated once per b2 and kept
  // in a register of the thread that owns the node (q^2 + M^2 <= 185 < blockDim nodes, one
  // per thread); step k takes B = (k mod nb1) nb2 + k / nb1 and buffer k & 1.
  const int nb1 = 1 << lb;
  auto box_of = [&](int k) { return (k & (nb1 - 1)) * nb2 + (k >> lb); };
  auto issue = [&](int k) {
    if (k < nB) {
      const float2 *src = st + ((long long)A * nB + box_of(k)) * nrq + (long long)r0 * Q2;
      float2 *dst = dbuf + (k & 1) * kRMax * Q2;
      for (int idx = threadIdx.x; idx < rt * Q2; idx += blockDim.x) cp_async8(dst + idx, src + idx);
    }
    cp_async_commit();
  };
  issue(0);
  issue(1);
  df gown = {0.f, 0.f};  // G(x_idx, p0_2) of the current b2, idx = threadIdx.x
  const int rr = threadIdx.x / M, m1o = threadIdx.x % M;  // accumulator owner (r, m1)
  const bool owner = threadIdx.x < rt * M;
  float ux[kTermM], uy[kTermM];
#pragma unroll
  for (int m2 = 0; m2 < kTermM; m2++) ux[m2] = uy[m2] = 0.f;
  __syncthreads();
  for (int B_ = 0; B_ < nB; B_++) {  // step B_ of the walk
    const int b1 = B_ & (nb1 - 1), b2 = B_ >> lb;
    float2 *pre = phb + (B_ & 1) * (Q2 + kTermM * kTermM);
    float2 *post = pre + Q2;
    const int idx = threadIdx.x;
    if (idx < Q2 + M2) {
      float2 v;
      if (sep) {
        const XNode &x1 = idx < Q2 ? xn(tb, l, a1, idx / Q, Q) : tb.xgrid[a1 * M + (idx - Q2) / M];
        const XNode &x2 = idx < Q2 ? xn(tb, l, a2, idx % Q, Q) : tb.xgrid[a2 * M + (idx - Q2) % M];
        v = expi<float>(theta_xp(ph, x1, x2, pn1(tb, lb, b1, Q, Q), pn2(tb, lb, b2, Q, Q)));
      } else {
        if (b1 == 0) gown = g_eval(tf.ph, xd[idx], p2f(tb, tf, lb, b2, Q, Q));
        v = expi_df(df_mul(rhof(tb, tf, lb, b1, Q, Q), gown));
      }
      if (idx < Q2) pre[idx] = conjf2(v);
      else post[idx - Q2] = v;
    }
    cp_async_wait(B_ + 1 < nB);
    __syncthreads();
    const float2 *dv = dbuf + (B_ & 1) * kRMax * Q2;
    for (int task = threadIdx.x; task < rt * Q; task += blockDim.x) {
      const int t2 = task % Q, r = task / Q;
      float2 ym[kTermM];
#pragma unroll
      for (int m = 0; m < kTermM; m++) ym[m] = make_float2(0.f, 0.f);
#pragma unroll
      for (int t1 = 0; t1 < Q; t1++) {
        const float2 c = cmul(pre[t1 * Q + t2], dv[r * Q2 + t1 * Q + t2]);
#pragma unroll
        for (int m = 0; m < kTermM; m++) ym[m] = fma2s(vm.V[m][t1], c, ym[m]);
      }
#pragma unroll
      for (int m = 0; m < kTermM; m++)
        if (m < M) y[(r * kTermM + m) * Q + t2] = ym[m];
    }
    __syncthreads();
    issue(B_ + 2);
    if (owner) {
      float2 yr[Q];
#pragma unroll
      for (int t2 = 0; t2 < Q; t2++) yr[t2] = y[(rr * kTermM + m1o) * Q + t2];
#pragma unroll
      for (int m2 = 0; m2 < kTermM; m2++) {
        if (m2 < M) {
          float2 wv = make_float2(0.f, 0.f);
#pragma unroll
          for (int t2 = 0; t2 < Q; t2++) wv = fma2s(vm.V[m2][t2], yr[t2], wv);
          const float wx = wv.x, wy = wv.y;
          const float2 p = post[m1o * M + m2];
          ux[m2] = __fmaf_rn(p.x, wx, __fmaf_rn(-p.y, wy, ux[m2]));
          uy[m2] = __fmaf_rn(p.x, wy, __fmaf_rn(p.y, wx, uy[m2]));
        }
      }
    }
  }
  if (owner) {
    const long long i1 = (long long)a1 * M + m1o;
#pragma unroll
    for (int m2 = 0; m2 < kTermM; m2++) {  // compile-time index: the accumulators stay in registers
      if (m2 < M) {
        const long long i2 = (long long)a2 * M + m2;
        u[(long long)(r0 + rr) * NN + (i1 << g.L) + i2] = make_float2(ux[m2], uy[m2]);
      }
    }
  }
}
template <int Q>
__global__ void __launch_bounds__(32 * (Q > kTermM ? Q : kTermM)) k32_term(Tables tb, TablesF tf, Phase ph, Geom g,
                                                                          VMat<float, Q> vm,
                                                                          const float2 *__restrict__ st,
                                                                          float2 *__restrict__ u) {
  k32_term_body<Q>(tb, tf, ph, g, vm, st, u, blockIdx.x, blockIdx.y);
}

// FP32 conjugate transpose of the termination: for each B at level s (fixed order),
//   d^{AB}[r][t] = post_B[t] sum_{m1,m2} V[m1][t1] V[m2][t2] pre_B[m] g[r][m],
// pre_B[m] = e^{-2 pi i theta(x_m, p0(B))}, post_B[t] = e^{2 pi i theta(x^A_t, p0(B))}.
template <int Q>
__device__ __forceinline__ void k32_term_adj_body(const Tables &tb, const TablesF &tf, const Phase &ph, const Geom &g,
                                                  const VMat<float, Q> &vm, const float2 *__restrict__ gin,
                                                  float2 *__restrict__ st, long long bx_, int by_) {
  constexpr int Q2 = Q * Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int l = g.l, lb = g.L - g.l, e = g.e;
  const int M = 1 << g.s, M2 = M * M;
  const int A = bx_, nA1 = 1 << l;
  const int a1 = A >> l, a2 = A & (nA1 - 1);
  const int r0 = by_ * kRMax;
  const int rt = min(kRMax, g.nrhs - r0);
  const int nb2 = 1 << (lb + e);
  const int nB = (1 << lb) * nb2;
  const long long NN = 1LL << (2 * g.L);
  const long long nrq = (long long)g.nrhs * Q2;
  float2 *gv = (float2 *)smem_raw;            // [kRMax][M2]
  float2 *y = gv + kRMax * kTermM * kTermM;   // [kRMax][Q][kTermM]
  float2 *pre = y + kRMax * Q * kTermM;       // [M2]
  float2 *post = pre + kTermM * kTermM;       // [Q2]
  XDesc *xd = (XDesc *)(post + Q2);           // [Q2 + M2]
  const bool sep = ph.id == 3;
  for (int idx = threadIdx.x; idx < rt * M2; idx += blockDim.x) {
    const int m = idx % M2, r = idx / M2;
    const long long i1 = (long long)a1 * M + m / M, i2 = (long long)a2 * M + m % M;
    gv[idx] = gin[(long long)(r0 + r) * NN + (i1 << g.L) + i2];
  }
  if (!sep)
    for (int idx = threadIdx.x; idx < Q2 + M2; idx += blockDim.x) {
      if (idx < Q2) {
        xd[idx] = xdesc(tf.ph, xnf(tb, tf, l, a1, idx / Q, Q), xnf(tb, tf, l, a2, idx % Q, Q));
      } else {
        const int m = idx - Q2;
        xd[idx] = xdesc(tf.ph, tf.xgrid[a1 * M + m / M], tf.xgrid[a2 * M + m % M]);
      }
    }
  // boxes B walked angular index first, G of the homogeneous phase evaluated once per b2
  // by the thread that owns the node (as in k32_term_body)
  const int nb1 = 1 << lb;
  df gown = {0.f, 0.f};
  for (int B_ = 0; B_ < nB; B_++) {
    const int b1 = B_ & (nb1 - 1), b2 = B_ >> lb;
    const int B = b1 * nb2 + b2;
    __syncthreads();  // gv/xd are ready; the previous B is done reading pre/post
    const int idx = threadIdx.x;
    if (idx < Q2 + M2) {
      float2 v;
      if (sep) {
        const XNode &x1 = idx < Q2 ? xn(tb, l, a1, idx / Q, Q) : tb.xgrid[a1 * M + (idx - Q2) / M];
        const XNode &x2 = idx < Q2 ? xn(tb, l, a2, idx % Q, Q) : tb.xgrid[a2 * M + (idx - Q2) % M];
        v = expi<float>(theta_xp(ph, x1, x2, pn1(tb, lb, b1, Q, Q), pn2(tb, lb, b2, Q, Q)));
      } else {
        if (b1 == 0) gown = g_eval(tf.ph, xd[idx], p2f(tb, tf, lb, b2, Q, Q));
        v = expi_df(df_mul(rhof(tb, tf, lb, b1, Q, Q), gown));
      }
      if (idx < Q2) post[idx] = v;
      else pre[idx - Q2] = conjf2(v);
    }
    __syncthreads();
    // y[r][t1][m2] = sum_m1 V[m1][t1] pre[m] g[r][m]   (thread per (r, m2))
    for (int task = threadIdx.x; task < rt * M; task += blockDim.x) {
      const int m2 = task % M, r = task / M;
      float2 yv[Q];
#pragma unroll
      for (int t1 = 0; t1 < Q; t1++) yv[t1] = make_float2(0.f, 0.f);
      for (int m1 = 0; m1 < M; m1++) {
        const float2 c = cmul(pre[m1 * M + m2], gv[r * M2 + m1 * M + m2]);
#pragma unroll
        for (int t1 = 0; t1 < Q; t1++) yv[t1] = fma2s(vm.V[m1][t1], c, yv[t1]);
      }
#pragma unroll
      for (int t1 = 0; t1 < Q; t1++) y[(r * Q + t1) * kTermM + m2] = yv[t1];
    }
    __syncthreads();
    // d[r][t1][t2] = post[t] sum_m2 V[m2][t2] y[r][t1][m2]   (thread per (r, t1))
    float2 *dst = st + ((long long)A * nB + B) * nrq + (long long)r0 * Q2;
    for (int task = threadIdx.x; task < rt * Q; task += blockDim.x) {
      const int t1 = task % Q, r = task / Q;
      float2 yr[kTermM];
#pragma unroll
      for (int m2 = 0; m2 < kTermM; m2++) yr[m2] = m2 < M ? y[(r * Q + t1) * kTermM + m2] : make_float2(0.f, 0.f);
#pragma unroll
      for (int t2 = 0; t2 < Q; t2++) {
        float2 av = make_float2(0.f, 0.f);
#pragma unroll
        for (int m2 = 0; m2 < kTermM; m2++) av = fma2s(vm.V[m2][t2], yr[m2], av);
        dst[r * Q2 + t1 * Q + t2] = cmul(post[t1 * Q + t2], av);
      }
    }
  }
}
template <int Q>
__global__ void __launch_bounds__(32 * (Q > kTermM ? Q : kTermM)) k32_term_adj(Tables tb, TablesF tf, Phase ph,
                                                                              Geom g, VMat<float, Q> vm,
                                                                              const float2 *__restrict__ gin,
                                                                              float2 *__restrict__ st) {
  k32_term_adj_body<Q>(tb, tf, ph, g, vm, gin, st, blockIdx.x, blockIdx.y);
}

}  // namespace fio
