// fio_kernels.cuh -- the butterfly steps as sm_103a kernels, templated on the
// working precision R (double: FIO_F64, float: FIO_F32) and on q.
//
// State layout of one level: pairs (A, B), A = (a1, a2) at T_X level l,
// B = (b1, b2) at T_P level L - l with b1 < 2^(L-l), b2 < 2^(L-l+e).
//   pair index = (a1 * 2^l + a2) * nB + b1 * 2^(L-l+e) + b2,   nB = 2^(L-l) 2^(L-l+e)
//   element    = (pair * nrhs + r) * q^2 + t1 * q + t2         (complex R)
// A translation "unit" at level l is (A_p at level l-1, B at level L-l): its
// four pairs (A_p, B_c) at level l-1 and its four pairs (A_sigma, B) at level l.
// Every CTA stages the unit's coefficient blocks and its phase factors (shared by
// all right-hand sides, Sec. 4 "vectorized" form) in shared memory, then applies
// the Lagrange translation one dimension at a time (Sec. 4, O(q^3) per pair).
#pragma once
#include "fio_common.cuh"

namespace fio {

// T[sigma][j][j'] = L_j((2 sigma - 1)/4 + z_j'/2): parent Lagrange polynomial j at
// node j' of child sigma (L^B_t(p^{Bc}_t') of eq. alg2b, L^{Ap}_t'(x^A_t) of eq. alg2c).
template <typename R, int Q> struct TMat {
  R T[2][Q][Q];
};
// V[m][j] = L_j(m / 2^s - 1/2): Lagrange polynomial j at the grid point m of a
// termination box (L^A_t(x) of eq. alg2d).
template <typename R, int Q> struct VMat {
  R V[kMMax][Q];
};

struct UnitIdx {
  int ap1, ap2, b1, b2;
  long long ap_idx, b_idx;
};

// Unit u at level l: u = ap_idx * nBl + b_idx.
__device__ __forceinline__ UnitIdx unit_decode(long long u, int l, int lb, int e) {
  UnitIdx d;
  const long long nb2 = 1LL << (lb + e);
  const long long nBl = (1LL << lb) * nb2;
  d.ap_idx = u / nBl;
  d.b_idx = u - d.ap_idx * nBl;
  d.ap1 = (int)(d.ap_idx >> (l - 1));
  d.ap2 = (int)(d.ap_idx & ((1LL << (l - 1)) - 1));
  d.b1 = (int)(d.b_idx / nb2);
  d.b2 = (int)(d.b_idx - (long long)d.b1 * nb2);
  return d;
}
// Pair (A_sigma, B) at level l, sigma = 2 s1 + s2.
__device__ __forceinline__ long long pair_child_a(const UnitIdx &d, int sg, int l, int lb, int e) {
  const long long a1 = 2 * d.ap1 + (sg >> 1), a2 = 2 * d.ap2 + (sg & 1);
  const long long nBl = (1LL << lb) << (lb + e);
  return ((a1 << l) + a2) * nBl + d.b_idx;
}
// Pair (A_p, B_c) at level l-1, c = 2 c1 + c2.
__device__ __forceinline__ long long pair_child_b(const UnitIdx &d, int c, int lb, int e) {
  const long long nb2c = 1LL << (lb + 1 + e);
  const long long nBp = (1LL << (lb + 1)) * nb2c;
  return d.ap_idx * nBp + (2LL * d.b1 + (c >> 1)) * nb2c + 2LL * d.b2 + (c & 1);
}

// ---------------------------------------------------------------------------
// Translation of type P:  out_j = post_j (.) sum_i (T^{i1} (x) T^{i2}) (pre_{j,i} (.) in_i)
// FWD : recursion in p (eq. alg2b), level l-1 -> l.  i = child c of B, j = child sigma of A.
//       pre_{sigma,c}(t') = e^{2 pi i theta(x0(A_sigma), p^{Bc}_t')},
//       post_sigma(t)     = e^{-2 pi i theta(x0(A_sigma), p^B_t)}.
// !FWD: conjugate transpose of the recursion in x, level l -> l-1.  i = sigma, j = c.
//       pre_{c,sigma}(t) = e^{-2 pi i theta(x^{A_sigma}_t, p0(B_c))},
//       post_c(t')       = e^{2 pi i theta(x^{A_p}_t', p0(B_c))}.
// ---------------------------------------------------------------------------
template <typename R, int Q, bool FWD>
__global__ void __launch_bounds__(kThreads) k_trans_p(Tables tb, Phase ph, Geom g, TMat<R, Q> tm,
                                                       const typename C2<R>::T *__restrict__ in,
                                                       typename C2<R>::T *__restrict__ out) {
  typedef typename C2<R>::T CT;
  constexpr int Q2 = Q * Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int U = g.U, RT = g.rt, l = g.l, lb = g.L - g.l, e = g.e;
  const long long u0 = (long long)blockIdx.x * U;
  const int r0 = blockIdx.y * RT;
  const int rt = min(RT, g.nrhs - r0);
  CT *in_s = (CT *)smem_raw;          // [U][4 i][RT][Q2]
  CT *z_s = in_s + U * 4 * RT * Q2;   // [U][4 j][2 i1][RT][Q][Q]
  CT *pre_s = z_s + U * 8 * RT * Q2;  // [U][4 j][4 i][Q2]
  CT *post_s = pre_s + U * 16 * Q2;   // [U][4 j][Q2]
  const long long nrq = (long long)g.nrhs * Q2;

  for (int idx = threadIdx.x; idx < U * 20 * Q2; idx += blockDim.x) {
    const int uu = idx / (20 * Q2);
    int rem = idx - uu * 20 * Q2;
    if (u0 + uu >= g.nunits) continue;
    const UnitIdx d = unit_decode(u0 + uu, l, lb, e);
    if (rem < 16 * Q2) {
      const int j = rem / (4 * Q2), i = (rem / Q2) & 3, t = rem % Q2;
      if (FWD) {  // x0(A_sigma=j) at level l; p^{B_c=i}_t at level lb+1
        const int a1 = 2 * d.ap1 + (j >> 1), a2 = 2 * d.ap2 + (j & 1);
        const int c1 = 2 * d.b1 + (i >> 1), c2 = 2 * d.b2 + (i & 1);
        const double th = theta_xp(ph, xn(tb, l, a1, Q, Q), xn(tb, l, a2, Q, Q), pn1(tb, lb + 1, c1, t / Q, Q),
                                   pn2(tb, lb + 1, c2, t % Q, Q));
        pre_s[((uu * 4 + j) * 4 + i) * Q2 + t] = expi<R>(th);
      } else {  // x^{A_sigma=i}_t at level l; p0(B_c=j) at level lb+1
        const int a1 = 2 * d.ap1 + (i >> 1), a2 = 2 * d.ap2 + (i & 1);
        const int c1 = 2 * d.b1 + (j >> 1), c2 = 2 * d.b2 + (j & 1);
        const double th = theta_xp(ph, xn(tb, l, a1, t / Q, Q), xn(tb, l, a2, t % Q, Q), pn1(tb, lb + 1, c1, Q, Q),
                                   pn2(tb, lb + 1, c2, Q, Q));
        CT v = expi<R>(th);
        v.y = -v.y;
        pre_s[((uu * 4 + j) * 4 + i) * Q2 + t] = v;
      }
    } else {
      rem -= 16 * Q2;
      const int j = rem / Q2, t = rem % Q2;
      if (FWD) {  // conj e(x0(A_sigma=j), p^B_t), B at level lb
        const int a1 = 2 * d.ap1 + (j >> 1), a2 = 2 * d.ap2 + (j & 1);
        CT v = expi<R>(theta_xp(ph, xn(tb, l, a1, Q, Q), xn(tb, l, a2, Q, Q), pn1(tb, lb, d.b1, t / Q, Q),
                                pn2(tb, lb, d.b2, t % Q, Q)));
        v.y = -v.y;
        post_s[(uu * 4 + j) * Q2 + t] = v;
      } else {  // e(x^{A_p}_t', p0(B_c=j)), A_p at level l-1
        const int c1 = 2 * d.b1 + (j >> 1), c2 = 2 * d.b2 + (j & 1);
        post_s[(uu * 4 + j) * Q2 + t] =
            expi<R>(theta_xp(ph, xn(tb, l - 1, d.ap1, t / Q, Q), xn(tb, l - 1, d.ap2, t % Q, Q),
                             pn1(tb, lb + 1, c1, Q, Q), pn2(tb, lb + 1, c2, Q, Q)));
      }
    }
  }
  for (int idx = threadIdx.x; idx < U * 4 * rt * Q2; idx += blockDim.x) {
    const int uu = idx / (4 * rt * Q2);
    int rem = idx - uu * 4 * rt * Q2;
    const int i = rem / (rt * Q2);
    rem -= i * rt * Q2;
    const int r = rem / Q2, t = rem % Q2;
    if (u0 + uu >= g.nunits) continue;
    const UnitIdx d = unit_decode(u0 + uu, l, lb, e);
    const long long pr = FWD ? pair_child_b(d, i, lb, e) : pair_child_a(d, i, l, lb, e);
    in_s[((uu * 4 + i) * RT + r) * Q2 + t] = in[pr * nrq + (long long)(r0 + r) * Q2 + t];
  }
  __syncthreads();

  // Z_{j,i1}[t'1][t2] = sum_{i2,t'2} T^{i2}[t2][t'2] (pre (.) in)_{(i1,i2)}[t'1][t'2]
  for (int task = threadIdx.x; task < U * 8 * rt * Q; task += blockDim.x) {
    const int tp1 = task % Q;
    const int r = (task / Q) % rt;
    const int i1 = (task / (Q * rt)) & 1;
    const int j = (task / (2 * Q * rt)) & 3;
    const int uu = task / (8 * Q * rt);
    if (u0 + uu >= g.nunits) continue;
    CT s[2][Q];
#pragma unroll
    for (int i2 = 0; i2 < 2; i2++) {
      const int i = i1 * 2 + i2;
#pragma unroll
      for (int tp2 = 0; tp2 < Q; tp2++)
        s[i2][tp2] = cmul(pre_s[((uu * 4 + j) * 4 + i) * Q2 + tp1 * Q + tp2], in_s[((uu * 4 + i) * RT + r) * Q2 + tp1 * Q + tp2]);
    }
    CT *zrow = z_s + (((uu * 4 + j) * 2 + i1) * RT + r) * Q2 + tp1 * Q;
#pragma unroll
    for (int t2 = 0; t2 < Q; t2++) {
      R ax = 0, ay = 0;
#pragma unroll
      for (int i2 = 0; i2 < 2; i2++)
#pragma unroll
        for (int tp2 = 0; tp2 < Q; tp2++) {
          ax += tm.T[i2][t2][tp2] * s[i2][tp2].x;
          ay += tm.T[i2][t2][tp2] * s[i2][tp2].y;
        }
      zrow[t2] = cmk<R>(ax, ay);
    }
  }
  __syncthreads();

  // Y_j[t1][t2] = sum_{i1,t'1} T^{i1}[t1][t'1] Z_{j,i1}[t'1][t2];  out_j = post_j (.) Y_j
  for (int task = threadIdx.x; task < U * 4 * rt * Q; task += blockDim.x) {
    const int t2 = task % Q;
    const int r = (task / Q) % rt;
    const int j = (task / (Q * rt)) & 3;
    const int uu = task / (4 * Q * rt);
    if (u0 + uu >= g.nunits) continue;
    CT zc[2][Q];
#pragma unroll
    for (int i1 = 0; i1 < 2; i1++)
#pragma unroll
      for (int tp1 = 0; tp1 < Q; tp1++) zc[i1][tp1] = z_s[(((uu * 4 + j) * 2 + i1) * RT + r) * Q2 + tp1 * Q + t2];
    const UnitIdx d = unit_decode(u0 + uu, l, lb, e);
    const long long pr = FWD ? pair_child_a(d, j, l, lb, e) : pair_child_b(d, j, lb, e);
    CT *dst = out + pr * nrq + (long long)(r0 + r) * Q2 + t2;
#pragma unroll
    for (int t1 = 0; t1 < Q; t1++) {
      R ax = 0, ay = 0;
#pragma unroll
      for (int i1 = 0; i1 < 2; i1++)
#pragma unroll
        for (int tp1 = 0; tp1 < Q; tp1++) {
          ax += tm.T[i1][t1][tp1] * zc[i1][tp1].x;
          ay += tm.T[i1][t1][tp1] * zc[i1][tp1].y;
        }
      dst[t1 * Q] = cmul(post_s[(uu * 4 + j) * Q2 + t1 * Q + t2], cmk<R>(ax, ay));
    }
  }
}

// ---------------------------------------------------------------------------
// Translation of type X:  out_j = sum_i post_{j,i} (.) (T^{j1} (x) T^{j2})^T (pre_i (.) in_i)
// FWD : recursion in x (eq. alg2c), level l-1 -> l.  i = child c of B, j = child sigma of A.
//       pre_c(t')         = e^{-2 pi i theta(x^{A_p}_t', p0(B_c))},
//       post_{sigma,c}(t) = e^{2 pi i theta(x^{A_sigma}_t, p0(B_c))}.
// !FWD: conjugate transpose of the recursion in p, level l -> l-1.  i = sigma, j = c.
//       pre_sigma(t)      = e^{2 pi i theta(x0(A_sigma), p^B_t)},
//       post_{c,sigma}(u) = e^{-2 pi i theta(x0(A_sigma), p^{Bc}_u)}.
// ---------------------------------------------------------------------------
template <typename R, int Q, bool FWD>
__global__ void __launch_bounds__(kThreads) k_trans_x(Tables tb, Phase ph, Geom g, TMat<R, Q> tm,
                                                       const typename C2<R>::T *__restrict__ in,
                                                       typename C2<R>::T *__restrict__ out) {
  typedef typename C2<R>::T CT;
  constexpr int Q2 = Q * Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int U = g.U, RT = g.rt, l = g.l, lb = g.L - g.l, e = g.e;
  const long long u0 = (long long)blockIdx.x * U;
  const int r0 = blockIdx.y * RT;
  const int rt = min(RT, g.nrhs - r0);
  CT *s_s = (CT *)smem_raw;          // [U][4 i][RT][Q2]     pre_i (.) in_i
  CT *w_s = s_s + U * 4 * RT * Q2;   // [U][4 i][2 j1][RT][Q][Q]
  CT *pre_s = w_s + U * 8 * RT * Q2; // [U][4 i][Q2]
  CT *post_s = pre_s + U * 4 * Q2;   // [U][4 j][4 i][Q2]
  const long long nrq = (long long)g.nrhs * Q2;

  for (int idx = threadIdx.x; idx < U * 20 * Q2; idx += blockDim.x) {
    const int uu = idx / (20 * Q2);
    int rem = idx - uu * 20 * Q2;
    if (u0 + uu >= g.nunits) continue;
    const UnitIdx d = unit_decode(u0 + uu, l, lb, e);
    if (rem < 4 * Q2) {
      const int i = rem / Q2, t = rem % Q2;
      if (FWD) {  // conj e(x^{A_p}_t, p0(B_c=i))
        const int c1 = 2 * d.b1 + (i >> 1), c2 = 2 * d.b2 + (i & 1);
        CT v = expi<R>(theta_xp(ph, xn(tb, l - 1, d.ap1, t / Q, Q), xn(tb, l - 1, d.ap2, t % Q, Q),
                                pn1(tb, lb + 1, c1, Q, Q), pn2(tb, lb + 1, c2, Q, Q)));
        v.y = -v.y;
        pre_s[(uu * 4 + i) * Q2 + t] = v;
      } else {  // e(x0(A_sigma=i), p^B_t)
        const int a1 = 2 * d.ap1 + (i >> 1), a2 = 2 * d.ap2 + (i & 1);
        pre_s[(uu * 4 + i) * Q2 + t] = expi<R>(theta_xp(ph, xn(tb, l, a1, Q, Q), xn(tb, l, a2, Q, Q),
                                                        pn1(tb, lb, d.b1, t / Q, Q), pn2(tb, lb, d.b2, t % Q, Q)));
      }
    } else {
      rem -= 4 * Q2;
      const int j = rem / (4 * Q2), i = (rem / Q2) & 3, t = rem % Q2;
      if (FWD) {  // e(x^{A_sigma=j}_t, p0(B_c=i))
        const int a1 = 2 * d.ap1 + (j >> 1), a2 = 2 * d.ap2 + (j & 1);
        const int c1 = 2 * d.b1 + (i >> 1), c2 = 2 * d.b2 + (i & 1);
        post_s[((uu * 4 + j) * 4 + i) * Q2 + t] = expi<R>(theta_xp(
            ph, xn(tb, l, a1, t / Q, Q), xn(tb, l, a2, t % Q, Q), pn1(tb, lb + 1, c1, Q, Q), pn2(tb, lb + 1, c2, Q, Q)));
      } else {  // conj e(x0(A_sigma=i), p^{B_c=j}_u)
        const int a1 = 2 * d.ap1 + (i >> 1), a2 = 2 * d.ap2 + (i & 1);
        const int c1 = 2 * d.b1 + (j >> 1), c2 = 2 * d.b2 + (j & 1);
        CT v = expi<R>(theta_xp(ph, xn(tb, l, a1, Q, Q), xn(tb, l, a2, Q, Q), pn1(tb, lb + 1, c1, t / Q, Q),
                                pn2(tb, lb + 1, c2, t % Q, Q)));
        v.y = -v.y;
        post_s[((uu * 4 + j) * 4 + i) * Q2 + t] = v;
      }
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < U * 4 * rt * Q2; idx += blockDim.x) {
    const int uu = idx / (4 * rt * Q2);
    int rem = idx - uu * 4 * rt * Q2;
    const int i = rem / (rt * Q2);
    rem -= i * rt * Q2;
    const int r = rem / Q2, t = rem % Q2;
    if (u0 + uu >= g.nunits) continue;
    const UnitIdx d = unit_decode(u0 + uu, l, lb, e);
    const long long pr = FWD ? pair_child_b(d, i, lb, e) : pair_child_a(d, i, l, lb, e);
    s_s[((uu * 4 + i) * RT + r) * Q2 + t] =
        cmul(pre_s[(uu * 4 + i) * Q2 + t], in[pr * nrq + (long long)(r0 + r) * Q2 + t]);
  }
  __syncthreads();

  // W_{i,j1}[t1][t'2] = sum_{t'1} T^{j1}[t'1][t1] S_i[t'1][t'2]
  for (int task = threadIdx.x; task < U * 8 * rt * Q; task += blockDim.x) {
    const int tp2 = task % Q;
    const int r = (task / Q) % rt;
    const int j1 = (task / (Q * rt)) & 1;
    const int i = (task / (2 * Q * rt)) & 3;
    const int uu = task / (8 * Q * rt);
    if (u0 + uu >= g.nunits) continue;
    CT col[Q];
#pragma unroll
    for (int tp1 = 0; tp1 < Q; tp1++) col[tp1] = s_s[((uu * 4 + i) * RT + r) * Q2 + tp1 * Q + tp2];
    CT *wb = w_s + (((uu * 4 + i) * 2 + j1) * RT + r) * Q2 + tp2;
#pragma unroll
    for (int t1 = 0; t1 < Q; t1++) {
      R ax = 0, ay = 0;
#pragma unroll
      for (int tp1 = 0; tp1 < Q; tp1++) {
        ax += tm.T[j1][tp1][t1] * col[tp1].x;
        ay += tm.T[j1][tp1][t1] * col[tp1].y;
      }
      wb[t1 * Q] = cmk<R>(ax, ay);
    }
  }
  __syncthreads();

  // out_j[t1][t2] = sum_i post_{j,i}[t1][t2] sum_{t'2} T^{j2}[t'2][t2] W_{i,j1}[t1][t'2]
  for (int task = threadIdx.x; task < U * 4 * rt * Q; task += blockDim.x) {
    const int t1 = task % Q;
    const int r = (task / Q) % rt;
    const int j = (task / (Q * rt)) & 3;
    const int uu = task / (4 * Q * rt);
    if (u0 + uu >= g.nunits) continue;
    const int j1 = j >> 1, j2 = j & 1;
    R ax[Q], ay[Q];
#pragma unroll
    for (int t2 = 0; t2 < Q; t2++) ax[t2] = ay[t2] = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
      CT row[Q];
#pragma unroll
      for (int tp2 = 0; tp2 < Q; tp2++) row[tp2] = w_s[(((uu * 4 + i) * 2 + j1) * RT + r) * Q2 + t1 * Q + tp2];
#pragma unroll
      for (int t2 = 0; t2 < Q; t2++) {
        R vx = 0, vy = 0;
#pragma unroll
        for (int tp2 = 0; tp2 < Q; tp2++) {
          vx += tm.T[j2][tp2][t2] * row[tp2].x;
          vy += tm.T[j2][tp2][t2] * row[tp2].y;
        }
        const CT p = post_s[((uu * 4 + j) * 4 + i) * Q2 + t1 * Q + t2];
        ax[t2] += p.x * vx - p.y * vy;
        ay[t2] += p.x * vy + p.y * vx;
      }
    }
    const UnitIdx d = unit_decode(u0 + uu, l, lb, e);
    const long long pr = FWD ? pair_child_a(d, j, l, lb, e) : pair_child_b(d, j, lb, e);
    CT *dst = out + pr * nrq + (long long)(r0 + r) * Q2 + t1 * Q;
#pragma unroll
    for (int t2 = 0; t2 < Q; t2++) dst[t2] = cmk<R>(ax[t2], ay[t2]);
  }
}

// ---------------------------------------------------------------------------
// Switch at level lm (eq. alg2m), per pair (A, B):
//   FWD : out[t] = sum_s e^{2 pi i theta(x^A_t, p^B_s)} in[s]
//   !FWD: out[s] = sum_t e^{-2 pi i theta(x^A_t, p^B_s)} in[t]   (conjugate transpose)
// The q^2 x q^2 kernel is generated in shared memory in row chunks of TC rows.
// ---------------------------------------------------------------------------
template <typename R, int Q, bool FWD>
__global__ void __launch_bounds__(kThreads) k_switch(Tables tb, Phase ph, Geom g, int TC,
                                                      const typename C2<R>::T *__restrict__ in,
                                                      typename C2<R>::T *__restrict__ out) {
  typedef typename C2<R>::T CT;
  constexpr int Q2 = Q * Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int U = g.U, RT = g.rt, l = g.l, lb = g.L - g.l, e = g.e;
  const long long p0 = (long long)blockIdx.x * U;
  const int r0 = blockIdx.y * RT;
  const int rt = min(RT, g.nrhs - r0);
  const int nb2 = 1 << (lb + e);
  const long long nBl = (1LL << lb) * nb2;
  CT *in_s = (CT *)smem_raw;     // [U][RT][Q2]
  CT *k_s = in_s + U * RT * Q2;  // [U][TC][Q2]
  const long long nrq = (long long)g.nrhs * Q2;
  for (int idx = threadIdx.x; idx < U * rt * Q2; idx += blockDim.x) {
    const int uu = idx / (rt * Q2), r = (idx / Q2) % rt, t = idx % Q2;
    if (p0 + uu >= g.nunits) continue;
    in_s[(uu * RT + r) * Q2 + t] = in[(p0 + uu) * nrq + (long long)(r0 + r) * Q2 + t];
  }
  for (int o0 = 0; o0 < Q2; o0 += TC) {
    const int tc = min(TC, Q2 - o0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < U * tc * Q2; idx += blockDim.x) {
      const int uu = idx / (tc * Q2), oo = (idx / Q2) % tc, ii = idx % Q2;
      const long long pr = p0 + uu;
      if (pr >= g.nunits) continue;
      const long long a = pr / nBl, b = pr - a * nBl;
      const int a1 = (int)(a >> l), a2 = (int)(a & ((1LL << l) - 1));
      const int b1 = (int)(b / nb2), b2 = (int)(b - (long long)b1 * nb2);
      const int t = FWD ? o0 + oo : ii;  // x-node index
      const int s = FWD ? ii : o0 + oo;  // p-node index
      CT v = expi<R>(theta_xp(ph, xn(tb, l, a1, t / Q, Q), xn(tb, l, a2, t % Q, Q), pn1(tb, lb, b1, s / Q, Q),
                              pn2(tb, lb, b2, s % Q, Q)));
      if (!FWD) v.y = -v.y;
      k_s[(uu * TC + oo) * Q2 + ii] = v;
    }
    __syncthreads();
    for (int task = threadIdx.x; task < U * tc * rt; task += blockDim.x) {
      const int r = task % rt, oo = (task / rt) % tc, uu = task / (rt * tc);
      if (p0 + uu >= g.nunits) continue;
      const CT *kr = k_s + (uu * TC + oo) * Q2;
      const CT *ir = in_s + (uu * RT + r) * Q2;
      R ax = 0, ay = 0;
#pragma unroll 9
      for (int ii = 0; ii < Q2; ii++) {
        const CT kv = kr[ii], iv = ir[ii];
        ax += kv.x * iv.x - kv.y * iv.y;
        ay += kv.x * iv.y + kv.y * iv.x;
      }
      out[(p0 + uu) * nrq + (long long)(r0 + r) * Q2 + o0 + oo] = cmk<R>(ax, ay);
    }
  }
}

// ---------------------------------------------------------------------------
// Initialization (eq. alg2a), pairs (A at level l0, B at level L - l0):
//   delta^{AB}_t = e^{-2 pi i theta(x0(A), p^B_t)} sum_{k in B} L^B_t(p(k)) e^{2 pi i Phi(x0(A), k)} f(k)
// One CTA per box B (its sources staged once) and RHS tile; GA boxes A at a time.
// ---------------------------------------------------------------------------
template <typename R, int Q>
__global__ void __launch_bounds__(kThreads) k_init(Tables tb, Phase ph, Geom g, int maxsrc, int GA,
                                                    const typename C2<R>::T *__restrict__ f,
                                                    typename C2<R>::T *__restrict__ st) {
  typedef typename C2<R>::T CT;
  constexpr int Q2 = Q * Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int RT = g.rt, l0 = g.l, lb = g.L - g.l, e = g.e;
  const int box = blockIdx.x;
  const int nb2 = 1 << (lb + e);
  const int b1 = box / nb2, b2 = box % nb2;
  const int r0 = blockIdx.y * RT;
  const int rt = min(RT, g.nrhs - r0);
  const int j0 = tb.box_off[box], ns = tb.box_off[box + 1] - j0;
  const long long NN = 1LL << (2 * g.L);
  CT *fv = (CT *)smem_raw;                 // [maxsrc][RT]
  CT *pk = fv + maxsrc * RT;               // [GA][maxsrc]
  CT *post = pk + GA * maxsrc;             // [GA][Q2]
  R *w = (R *)(post + GA * Q2);            // [maxsrc][2Q]
  for (int idx = threadIdx.x; idx < ns * rt; idx += blockDim.x) {
    const int j = idx / rt, r = idx % rt;
    fv[j * RT + r] = f[(long long)(r0 + r) * NN + tb.src_f[j0 + j]];
  }
  for (int idx = threadIdx.x; idx < ns * 2 * Q; idx += blockDim.x) w[idx] = (R)tb.src_w[(long long)j0 * 2 * Q + idx];
  const int nA1 = 1 << l0, nA = nA1 * nA1;
  const long long nB = (1LL << lb) * nb2;
  const long long nrq = (long long)g.nrhs * Q2;
  for (int A0 = 0; A0 < nA; A0 += GA) {
    const int ga_n = min(GA, nA - A0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < ga_n * (ns + Q2); idx += blockDim.x) {
      const int ga = idx / (ns + Q2), k = idx % (ns + Q2);
      const int A = A0 + ga, a1 = A >> l0, a2 = A & (nA1 - 1);
      const XNode &x1 = xn(tb, l0, a1, Q, Q), &x2 = xn(tb, l0, a2, Q, Q);
      if (k < ns) {
        pk[ga * maxsrc + k] = expi<R>(theta_xk(ph, x1, x2, tb.src[j0 + k]));
      } else {
        const int t = k - ns;
        CT v = expi<R>(theta_xp(ph, x1, x2, pn1(tb, lb, b1, t / Q, Q), pn2(tb, lb, b2, t % Q, Q)));
        v.y = -v.y;
        post[ga * Q2 + t] = v;
      }
    }
    __syncthreads();
    for (int task = threadIdx.x; task < ga_n * rt * Q; task += blockDim.x) {
      const int t1 = task % Q, r = (task / Q) % rt, ga = task / (Q * rt);
      R ax[Q], ay[Q];
#pragma unroll
      for (int t2 = 0; t2 < Q; t2++) ax[t2] = ay[t2] = 0;
      for (int j = 0; j < ns; j++) {
        const CT v = cmul(pk[ga * maxsrc + j], fv[j * RT + r]);
        const R w1 = w[j * 2 * Q + t1];
        const R vx = w1 * v.x, vy = w1 * v.y;
#pragma unroll
        for (int t2 = 0; t2 < Q; t2++) {
          const R w2 = w[j * 2 * Q + Q + t2];
          ax[t2] += w2 * vx;
          ay[t2] += w2 * vy;
        }
      }
      const int A = A0 + ga;
      CT *dst = st + ((long long)A * nB + box) * nrq + (long long)(r0 + r) * Q2 + t1 * Q;
#pragma unroll
      for (int t2 = 0; t2 < Q; t2++) dst[t2] = cmul(post[ga * Q2 + t1 * Q + t2], cmk<R>(ax[t2], ay[t2]));
    }
  }
}

// Conjugate transpose of the initialization:
//   fbar(k) = sum_{A at l0} e^{-2 pi i Phi(x0(A), k)} sum_t L^B_t(p(k)) e^{2 pi i theta(x0(A), p^B_t)} d^{AB}_t
template <typename R, int Q>
__global__ void __launch_bounds__(kThreads) k_init_adj(Tables tb, Phase ph, Geom g, int maxsrc,
                                                        const typename C2<R>::T *__restrict__ st,
                                                        typename C2<R>::T *__restrict__ fbar) {
  typedef typename C2<R>::T CT;
  constexpr int Q2 = Q * Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int RT = g.rt, l0 = g.l, lb = g.L - g.l, e = g.e;
  const int box = blockIdx.x;
  const int nb2 = 1 << (lb + e);
  const int b1 = box / nb2, b2 = box % nb2;
  const int r0 = blockIdx.y * RT;
  const int rt = min(RT, g.nrhs - r0);
  const int j0 = tb.box_off[box], ns = tb.box_off[box + 1] - j0;
  const long long NN = 1LL << (2 * g.L);
  CT *acc = (CT *)smem_raw;      // [maxsrc][RT]
  CT *pk = acc + maxsrc * RT;    // [maxsrc]
  CT *pt = pk + maxsrc;          // [Q2]
  CT *v = pt + Q2;               // [RT][Q2]
  R *w = (R *)(v + RT * Q2);     // [maxsrc][2Q]
  for (int idx = threadIdx.x; idx < ns * rt; idx += blockDim.x) acc[(idx / rt) * RT + idx % rt] = cmk<R>(0, 0);
  for (int idx = threadIdx.x; idx < ns * 2 * Q; idx += blockDim.x) w[idx] = (R)tb.src_w[(long long)j0 * 2 * Q + idx];
  const int nA1 = 1 << l0, nA = nA1 * nA1;
  const long long nB = (1LL << lb) * nb2;
  const long long nrq = (long long)g.nrhs * Q2;
  for (int A = 0; A < nA; A++) {
    const int a1 = A >> l0, a2 = A & (nA1 - 1);
    const XNode &x1 = xn(tb, l0, a1, Q, Q), &x2 = xn(tb, l0, a2, Q, Q);
    __syncthreads();
    for (int idx = threadIdx.x; idx < ns + Q2; idx += blockDim.x) {
      if (idx < ns) {
        CT p = expi<R>(theta_xk(ph, x1, x2, tb.src[j0 + idx]));
        p.y = -p.y;
        pk[idx] = p;
      } else {
        const int t = idx - ns;
        pt[t] = expi<R>(theta_xp(ph, x1, x2, pn1(tb, lb, b1, t / Q, Q), pn2(tb, lb, b2, t % Q, Q)));
      }
    }
    __syncthreads();
    const CT *src = st + ((long long)A * nB + box) * nrq + (long long)r0 * Q2;
    for (int idx = threadIdx.x; idx < rt * Q2; idx += blockDim.x) v[idx] = cmul(pt[idx % Q2], src[idx]);
    __syncthreads();
    for (int task = threadIdx.x; task < ns * rt; task += blockDim.x) {
      const int j = task / rt, r = task % rt;
      const R *w1 = w + j * 2 * Q, *w2 = w1 + Q;
      R px = 0, py = 0;
#pragma unroll
      for (int t1 = 0; t1 < Q; t1++) {
        R qx = 0, qy = 0;
#pragma unroll
        for (int t2 = 0; t2 < Q; t2++) {
          const CT vv = v[r * Q2 + t1 * Q + t2];
          qx += w2[t2] * vv.x;
          qy += w2[t2] * vv.y;
        }
        px += w1[t1] * qx;
        py += w1[t1] * qy;
      }
      const CT p = cmul(pk[j], cmk<R>(px, py));
      CT a = acc[j * RT + r];
      a.x += p.x;
      a.y += p.y;
      acc[j * RT + r] = a;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < ns * rt; idx += blockDim.x) {
    const int j = idx / rt, r = idx % rt;
    fbar[(long long)(r0 + r) * NN + tb.src_f[j0 + j]] = acc[j * RT + r];
  }
}

// ---------------------------------------------------------------------------
// Termination (eq. alg2d), A at level l1 = L - s, summed over the boxes B at level s:
//   u(x) = sum_B e^{2 pi i theta(x, p0(B))} sum_t L^A_t(x) e^{-2 pi i theta(x^A_t, p0(B))} delta^{AB}_t
// One CTA per box A and RHS tile; the sum over B runs in a fixed order.
// ---------------------------------------------------------------------------
template <typename R, int Q>
__global__ void __launch_bounds__(kThreads) k_term(Tables tb, Phase ph, Geom g, VMat<R, Q> vm,
                                                    const typename C2<R>::T *__restrict__ st,
                                                    typename C2<R>::T *__restrict__ u) {
  typedef typename C2<R>::T CT;
  constexpr int Q2 = Q * Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int RT = g.rt, l = g.l, lb = g.L - g.l, e = g.e;
  const int M = 1 << g.s, M2 = M * M;
  const int A = blockIdx.x, nA1 = 1 << l;
  const int a1 = A >> l, a2 = A & (nA1 - 1);
  const int r0 = blockIdx.y * RT;
  const int rt = min(RT, g.nrhs - r0);
  const int nb2 = 1 << (lb + e);
  const int nB = (1 << lb) * nb2;
  const long long NN = 1LL << (2 * g.L);
  CT *acc = (CT *)smem_raw;   // [RT][M2]
  CT *pre = acc + RT * M2;    // [Q2]
  CT *post = pre + Q2;        // [M2]
  CT *sv = post + M2;         // [RT][Q2]
  CT *y = sv + RT * Q2;       // [RT][M][Q]
  for (int idx = threadIdx.x; idx < rt * M2; idx += blockDim.x) acc[idx] = cmk<R>(0, 0);
  const long long nrq = (long long)g.nrhs * Q2;
  for (int B = 0; B < nB; B++) {
    const int b1 = B / nb2, b2 = B % nb2;
    const P1Node &c1 = pn1(tb, lb, b1, Q, Q);
    const P2Node &c2 = pn2(tb, lb, b2, Q, Q);
    __syncthreads();
    for (int idx = threadIdx.x; idx < Q2 + M2; idx += blockDim.x) {
      if (idx < Q2) {
        CT v = expi<R>(theta_xp(ph, xn(tb, l, a1, idx / Q, Q), xn(tb, l, a2, idx % Q, Q), c1, c2));
        v.y = -v.y;
        pre[idx] = v;
      } else {
        const int m = idx - Q2;
        post[m] = expi<R>(theta_xp(ph, tb.xgrid[a1 * M + m / M], tb.xgrid[a2 * M + m % M], c1, c2));
      }
    }
    __syncthreads();
    const CT *src = st + ((long long)A * nB + B) * nrq + (long long)r0 * Q2;
    for (int idx = threadIdx.x; idx < rt * Q2; idx += blockDim.x) sv[idx] = cmul(pre[idx % Q2], src[idx]);
    __syncthreads();
    // y[r][m1][t2] = sum_t1 V[m1][t1] sv[r][t1][t2]
    for (int task = threadIdx.x; task < rt * M * Q; task += blockDim.x) {
      const int t2 = task % Q, m1 = (task / Q) % M, r = task / (Q * M);
      R ax = 0, ay = 0;
#pragma unroll
      for (int t1 = 0; t1 < Q; t1++) {
        const CT s = sv[r * Q2 + t1 * Q + t2];
        ax += vm.V[m1][t1] * s.x;
        ay += vm.V[m1][t1] * s.y;
      }
      y[(r * M + m1) * Q + t2] = cmk<R>(ax, ay);
    }
    __syncthreads();
    for (int task = threadIdx.x; task < rt * M2; task += blockDim.x) {
      const int m = task % M2, r = task / M2, m1 = m / M, m2 = m % M;
      R ax = 0, ay = 0;
#pragma unroll
      for (int t2 = 0; t2 < Q; t2++) {
        const CT s = y[(r * M + m1) * Q + t2];
        ax += vm.V[m2][t2] * s.x;
        ay += vm.V[m2][t2] * s.y;
      }
      const CT p = cmul(post[m], cmk<R>(ax, ay));
      CT a = acc[task];
      a.x += p.x;
      a.y += p.y;
      acc[task] = a;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < rt * M2; idx += blockDim.x) {
    const int m = idx % M2, r = idx / M2;
    const long long i1 = (long long)a1 * M + m / M, i2 = (long long)a2 * M + m % M;
    u[(long long)(r0 + r) * NN + (i1 << g.L) + i2] = acc[idx];
  }
}

// Conjugate transpose of the termination:
//   d^{AB}_t = e^{2 pi i theta(x^A_t, p0(B))} sum_{x in A} L^A_t(x) e^{-2 pi i theta(x, p0(B))} g(x)
template <typename R, int Q>
__global__ void __launch_bounds__(kThreads) k_term_adj(Tables tb, Phase ph, Geom g, VMat<R, Q> vm,
                                                        const typename C2<R>::T *__restrict__ gin,
                                                        typename C2<R>::T *__restrict__ st) {
  typedef typename C2<R>::T CT;
  constexpr int Q2 = Q * Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int RT = g.rt, l = g.l, lb = g.L - g.l, e = g.e;
  const int M = 1 << g.s, M2 = M * M;
  const int A = blockIdx.x, nA1 = 1 << l;
  const int a1 = A >> l, a2 = A & (nA1 - 1);
  const int r0 = blockIdx.y * RT;
  const int rt = min(RT, g.nrhs - r0);
  const int nb2 = 1 << (lb + e);
  const int nB = (1 << lb) * nb2;
  const long long NN = 1LL << (2 * g.L);
  CT *gv = (CT *)smem_raw;    // [RT][M2]
  CT *pre = gv + RT * M2;     // [M2]
  CT *post = pre + M2;        // [Q2]
  CT *gm = post + Q2;         // [RT][M2]
  CT *y = gm + RT * M2;       // [RT][Q][M]
  for (int idx = threadIdx.x; idx < rt * M2; idx += blockDim.x) {
    const int m = idx % M2, r = idx / M2;
    const long long i1 = (long long)a1 * M + m / M, i2 = (long long)a2 * M + m % M;
    gv[idx] = gin[(long long)(r0 + r) * NN + (i1 << g.L) + i2];
  }
  const long long nrq = (long long)g.nrhs * Q2;
  for (int B = 0; B < nB; B++) {
    const int b1 = B / nb2, b2 = B % nb2;
    const P1Node &c1 = pn1(tb, lb, b1, Q, Q);
    const P2Node &c2 = pn2(tb, lb, b2, Q, Q);
    __syncthreads();
    for (int idx = threadIdx.x; idx < Q2 + M2; idx += blockDim.x) {
      if (idx < M2) {
        CT v = expi<R>(theta_xp(ph, tb.xgrid[a1 * M + idx / M], tb.xgrid[a2 * M + idx % M], c1, c2));
        v.y = -v.y;
        pre[idx] = v;
      } else {
        const int t = idx - M2;
        post[t] = expi<R>(theta_xp(ph, xn(tb, l, a1, t / Q, Q), xn(tb, l, a2, t % Q, Q), c1, c2));
      }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < rt * M2; idx += blockDim.x) gm[idx] = cmul(pre[idx % M2], gv[idx]);
    __syncthreads();
    // y[r][t1][m2] = sum_m1 V[m1][t1] gm[r][m1][m2]
    for (int task = threadIdx.x; task < rt * Q * M; task += blockDim.x) {
      const int m2 = task % M, t1 = (task / M) % Q, r = task / (M * Q);
      R ax = 0, ay = 0;
      for (int m1 = 0; m1 < M; m1++) {
        const CT s = gm[r * M2 + m1 * M + m2];
        ax += vm.V[m1][t1] * s.x;
        ay += vm.V[m1][t1] * s.y;
      }
      y[(r * Q + t1) * M + m2] = cmk<R>(ax, ay);
    }
    __syncthreads();
    CT *dst = st + ((long long)A * nB + B) * nrq + (long long)r0 * Q2;
    for (int task = threadIdx.x; task < rt * Q2; task += blockDim.x) {
      const int t = task % Q2, r = task / Q2, t1 = t / Q, t2 = t % Q;
      R ax = 0, ay = 0;
      for (int m2 = 0; m2 < M; m2++) {
        const CT s = y[(r * Q + t1) * M + m2];
        ax += vm.V[m2][t2] * s.x;
        ay += vm.V[m2][t2] * s.y;
      }
      dst[task] = cmul(post[t], cmk<R>(ax, ay));
    }
  }
}

}  // namespace fio
