// fio3.cu -- the three-dimensional butterfly (Sec. 5, eq. ex3, Table 3) in FP64:
// the initialization, both recursions, the switch and the termination in 3D, and
// their exact conjugate transposes (include/fio3.h states the readings).
//
// State of one level: pairs (A, B), A = (a1, a2, a3) at T_X level l, B = (b1, b2, b3)
// at T_P level L-l (b1 < 2^(L-l), b2, b3 < 2^(L-l+e)); pair = a nB + b with
// a = (a1 2^l + a2) 2^l + a3, b = (b1 n2 + b2) n2 + b3, n2 = 2^(L-l+e);
// element (pair nrhs + r) q^3 + t, t = (t1 q + t2) q + t3.
//
// Every step applies the Lagrange interpolation of the q^3 tensor-product grid one
// dimension at a time (O(q^4) per pair instead of a dense q^3 x q^3 matrix).  The
// translation kernel is one template over the four shapes of the recursions:
//     out_o = P_o (.) sum_i Q_{o,i} (.) T_{o,i} (R_{o,i} (.) in_i)
// with elementwise phase factors P, Q, R (most of them 1) and T_{o,i} the 3D
// translation matrix of one child, transposed or not.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "fio.h"
#include "fio3.h"

namespace fio {
void set_last_error(const char *msg);
}

namespace f3 {

constexpr int kQ3Max = 7;
constexpr int kMaxLev = 16;

// Per-axis node tables (FP64).  x nodes of T_X level l: box a, j < q node, j = q centre.
struct XN3 {
  double x, s;  // x, sin 2 pi x
};
// p1 nodes of T_P level j: rho = (sqrt3/2) N p1.  p2, p3 nodes of angular level j:
struct PA3 {
  double s2, c2, c3, s3;  // sin pi p2, cos pi p2 (p2 axis); cos 2 pi p3, sin 2 pi p3 (p3 axis)
};

struct Tab3 {
  const XN3 *xn;     // per level l at xoff[l]: 2^l boxes x (q+1)
  const double *rho; // per radial level j at roff[j]: 2^j boxes x (q+1)
  const PA3 *pa;     // per angular level j at aoff[j]: 2^j boxes x (q+1) (both angular axes)
  const int *box_off;   // initialization boxes (level L-s): CSR of the sources
  const int *src_f;     // flat index of each sorted source
  const double *src_w;  // 3q Lagrange weights per sorted source (p1, p2, p3 axes)
  int xoff[kMaxLev], roff[kMaxLev], aoff[kMaxLev];
};

struct Ph3 {
  int id;  // 0 linear, 2 sphere
  double a, m, ib, lam;
};

struct G3 {
  int L, e, q, s, l, nrhs, N;
  Ph3 ph;
};

template <int Q> struct Mats {
  double T[2][Q][Q];  // T[sigma][j][j'] = L_j((2 sigma - 1)/4 + z_j'/2)
  double V[8][Q];     // V[m][j] = L_j(m / 2^s - 1/2)
};

__device__ __forceinline__ double2 expi64(double th) {
  const double r = th - rint(th);
  double sn, cs;
  sincospi(2.0 * r, &sn, &cs);
  return make_double2(cs, sn);
}
__device__ __forceinline__ double2 cm(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cj(double2 a) { return make_double2(a.x, -a.y); }

// A point x of T_X given per axis by its node entries, and c(x) of the sphere phase.
struct XP {
  double x1, x2, x3, c;
};
__device__ __forceinline__ XP xpoint(const Ph3 &ph, const XN3 &u, const XN3 &v, const XN3 &w) {
  XP p;
  p.x1 = u.x;
  p.x2 = v.x;
  p.x3 = w.x;
  p.c = ph.id == 2 ? (ph.a + ph.m * u.s * v.s * w.s) * ph.ib : 0.0;
  return p;
}
// theta(x, p) = Phi(x, kappa(p)), p given by rho (radial entry) and the two angular entries.
__device__ __forceinline__ double theta3(const Ph3 &ph, const XP &x, double rho, const PA3 &a2, const PA3 &a3) {
  const double k1 = rho * a2.s2 * a3.c3, k2 = rho * a2.s2 * a3.s3, k3 = rho * a2.c2;
  const double lin = x.x1 * k1 + x.x2 * k2 + x.x3 * k3;
  if (ph.id == 0) return lin;
  return ph.lam * lin + x.c * rho;
}
// Phi(x, k) at a lattice frequency.
__device__ __forceinline__ double phik3(const Ph3 &ph, const XP &x, double k1, double k2, double k3) {
  const double lin = x.x1 * k1 + x.x2 * k2 + x.x3 * k3;
  if (ph.id == 0) return lin;
  return ph.lam * lin + x.c * sqrt(k1 * k1 + k2 * k2 + k3 * k3);
}

// Box decoding and table entries.
struct Box3 {
  int c0, c1, c2;
};
__device__ __forceinline__ Box3 adec(long long a, int l) {
  const long long n = 1LL << l;
  return {(int)(a / (n * n)), (int)((a / n) % n), (int)(a % n)};
}
__device__ __forceinline__ Box3 bdec(long long b, int lb, int e) {
  const long long n2 = 1LL << (lb + e);
  return {(int)(b / (n2 * n2)), (int)((b / n2) % n2), (int)(b % n2)};
}
__device__ __forceinline__ long long aenc(Box3 a, int l) {
  const long long n = 1LL << l;
  return ((long long)a.c0 * n + a.c1) * n + a.c2;
}
__device__ __forceinline__ long long benc(Box3 b, int lb, int e) {
  const long long n2 = 1LL << (lb + e);
  return ((long long)b.c0 * n2 + b.c1) * n2 + b.c2;
}
__device__ __forceinline__ long long nbox_b(int lb, int e) { return (1LL << lb) << (2 * (lb + e)); }
__device__ __forceinline__ Box3 child(Box3 b, int c) {
  return {2 * b.c0 + (c >> 2), 2 * b.c1 + ((c >> 1) & 1), 2 * b.c2 + (c & 1)};
}

// x point of box A (level l) at node t = (t1, t2, t3) (j = q: centre along that axis).
__device__ __forceinline__ XP xat(const Tab3 &tb, const Ph3 &ph, int l, Box3 a, int t1, int t2, int t3, int q) {
  const XN3 *base = tb.xn + tb.xoff[l];
  return xpoint(ph, base[a.c0 * (q + 1) + t1], base[a.c1 * (q + 1) + t2], base[a.c2 * (q + 1) + t3]);
}
// theta(x, p^B_u) with B at T_P level lb, node u = (u1, u2, u3) (q: centre).
__device__ __forceinline__ double thp(const Tab3 &tb, const G3 &g, const XP &x, int lb, Box3 b, int u1, int u2,
                                      int u3) {
  const int q = g.q;
  const double rho = tb.rho[tb.roff[lb] + b.c0 * (q + 1) + u1];
  const PA3 *pa = tb.pa + tb.aoff[lb + g.e];
  return theta3(g.ph, x, rho, pa[b.c1 * (q + 1) + u2], pa[b.c2 * (q + 1) + u3]);
}

}  // namespace f3

namespace f3 {

constexpr int kThr = 128;  // threads per CTA of every 3D kernel
constexpr int kSrcChunk = 128;

// Flat lattice index -> (k1, k2, k3).
__device__ __forceinline__ void kof(long long idx, int N, double &k1, double &k2, double &k3) {
  const long long NN = (long long)N * N;
  k1 = (double)(idx / NN) - N / 2;
  k2 = (double)((idx / N) % N) - N / 2;
  k3 = (double)(idx % N) - N / 2;
}

// ---------------------------------------------------------------------------
// Initialization (3D form of eq. alg2a), A at level l0 = s, B at level L - s:
//   delta^{AB}_t = conj e(x0(A), p^B_t) sum_{k in B} L^B_t(p(k)) e(x0(A), k) f(k).
// One CTA per (box B, RHS); the boxes A in turn; sources in chunks.
// ---------------------------------------------------------------------------
template <int Q>
__global__ void __launch_bounds__(kThr) k3_init(Tab3 tb, G3 g, const double2 *__restrict__ f, double2 *__restrict__ st) {
  constexpr int Q3 = Q * Q * Q, PT = (Q3 + kThr - 1) / kThr;
  __shared__ double2 v_s[kSrcChunk];
  __shared__ double w_s[kSrcChunk][3 * Q];
  const int l = g.l, lb = g.L - l, e = g.e;
  const long long b = blockIdx.x, nB = nbox_b(lb, e);
  const int r = blockIdx.y;
  const Box3 bb = bdec(b, lb, e);
  const int j0 = tb.box_off[b], ns = tb.box_off[b + 1] - j0;
  const long long NNN = (long long)g.N * g.N * g.N;
  const long long nA = 1LL << (3 * l);
  for (long long A = 0; A < nA; A++) {
    const Box3 ab = adec(A, l);
    const XP x0 = xat(tb, g.ph, l, ab, Q, Q, Q, Q);
    double2 acc[PT];
#pragma unroll
    for (int c = 0; c < PT; c++) acc[c] = make_double2(0.0, 0.0);
    for (int c0 = 0; c0 < ns; c0 += kSrcChunk) {
      const int nc = min(kSrcChunk, ns - c0);
      __syncthreads();
      for (int j = threadIdx.x; j < nc; j += kThr) {
        const long long kf = tb.src_f[j0 + c0 + j];
        double k1, k2, k3;
        kof(kf, g.N, k1, k2, k3);
        v_s[j] = cm(expi64(phik3(g.ph, x0, k1, k2, k3)), f[(long long)r * NNN + kf]);
      }
      for (int idx = threadIdx.x; idx < nc * 3 * Q; idx += kThr)
        w_s[idx / (3 * Q)][idx % (3 * Q)] = tb.src_w[(long long)(j0 + c0) * 3 * Q + idx];
      __syncthreads();
#pragma unroll
      for (int c = 0; c < PT; c++) {
        const int t = threadIdx.x + c * kThr;
        if (t < Q3) {
          const int t1 = t / (Q * Q), t2 = (t / Q) % Q, t3 = t % Q;
          for (int j = 0; j < nc; j++) {
            const double w = w_s[j][t1] * w_s[j][Q + t2] * w_s[j][2 * Q + t3];
            acc[c].x += w * v_s[j].x;
            acc[c].y += w * v_s[j].y;
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < PT; c++) {
      const int t = threadIdx.x + c * kThr;
      if (t < Q3) {
        const double th = thp(tb, g, x0, lb, bb, t / (Q * Q), (t / Q) % Q, t % Q);
        st[((A * nB + b) * g.nrhs + r) * Q3 + t] = cm(cj(expi64(th)), acc[c]);
      }
    }
  }
}

// Conjugate transpose of the initialization:
//   fbar(k) = sum_A conj e(x0(A), k) sum_t L^B_t(p(k)) e(x0(A), p^B_t) delta^{AB}_t.
// One CTA per (box B, RHS); a thread per source of a chunk.
template <int Q>
__global__ void __launch_bounds__(kThr) k3_init_adj(Tab3 tb, G3 g, const double2 *__restrict__ st,
                                                    double2 *__restrict__ fbar) {
  constexpr int Q3 = Q * Q * Q;
  __shared__ double2 v_s[Q3];
  const int l = g.l, lb = g.L - l, e = g.e;
  const long long b = blockIdx.x, nB = nbox_b(lb, e);
  const int r = blockIdx.y;
  const Box3 bb = bdec(b, lb, e);
  const int j0 = tb.box_off[b], ns = tb.box_off[b + 1] - j0;
  const long long NNN = (long long)g.N * g.N * g.N;
  const long long nA = 1LL << (3 * l);
  for (int c0 = 0; c0 < ns; c0 += kThr) {
    const int j = c0 + threadIdx.x;
    const bool live = j < ns;
    long long kf = 0;
    double k1 = 0, k2 = 0, k3 = 0, w[3 * Q];
    if (live) {
      kf = tb.src_f[j0 + j];
      kof(kf, g.N, k1, k2, k3);
#pragma unroll
      for (int i = 0; i < 3 * Q; i++) w[i] = tb.src_w[(long long)(j0 + j) * 3 * Q + i];
    }
    double2 acc = make_double2(0.0, 0.0);
    for (long long A = 0; A < nA; A++) {
      const Box3 ab = adec(A, l);
      const XP x0 = xat(tb, g.ph, l, ab, Q, Q, Q, Q);
      __syncthreads();
      for (int t = threadIdx.x; t < Q3; t += kThr) {
        const double th = thp(tb, g, x0, lb, bb, t / (Q * Q), (t / Q) % Q, t % Q);
        v_s[t] = cm(expi64(th), st[((A * nB + b) * g.nrhs + r) * Q3 + t]);
      }
      __syncthreads();
      if (live) {
        double2 part = make_double2(0.0, 0.0);
        for (int t1 = 0; t1 < Q; t1++) {
          double2 p2 = make_double2(0.0, 0.0);
          for (int t2 = 0; t2 < Q; t2++) {
            double2 p3 = make_double2(0.0, 0.0);
#pragma unroll
            for (int t3 = 0; t3 < Q; t3++) {
              const double2 v = v_s[(t1 * Q + t2) * Q + t3];
              p3.x += w[2 * Q + t3] * v.x;
              p3.y += w[2 * Q + t3] * v.y;
            }
            p2.x += w[Q + t2] * p3.x;
            p2.y += w[Q + t2] * p3.y;
          }
          part.x += w[t1] * p2.x;
          part.y += w[t1] * p2.y;
        }
        const double2 ph = cj(expi64(phik3(g.ph, x0, k1, k2, k3)));
        const double2 pc = cm(ph, part);
        acc.x += pc.x;
        acc.y += pc.y;
      }
    }
    if (live) fbar[(long long)r * NNN + kf] = acc;
  }
}

}  // namespace f3

namespace f3 {

// Translation shapes: the recursion in p (eq. alg2b) and in x (eq. alg2c), and their
// conjugate transposes (level l -> l-1).
enum { V_PF = 0, V_XF = 1, V_PA = 2, V_XA = 3 };

// One dimension pass of the 3D Lagrange transform on a q^3 block: along axis D
// (0: t1, 1: t2, 2: t3), out[.., a, ..] = sum_b M[a][b] in[.., b, ..] with
// M[a][b] = T^{kd}[a][b] (TR false) or T^{kd}[b][a] (TR true).
template <int Q, int D, bool TR>
__device__ __forceinline__ void pass3(const Mats<Q> &mt, int kd, const double2 *in, double2 *out) {
  constexpr int Q3 = Q * Q * Q;
  constexpr int SD = D == 0 ? Q * Q : D == 1 ? Q : 1;  // stride of axis D
  for (int t = threadIdx.x; t < Q3; t += kThr) {
    const int a = (t / SD) % Q;
    const int base = t - a * SD;
    double2 s = make_double2(0.0, 0.0);
#pragma unroll
    for (int b = 0; b < Q; b++) {
      const double m = TR ? mt.T[kd][b][a] : mt.T[kd][a][b];
      const double2 v = in[base + b * SD];
      s.x += m * v.x;
      s.y += m * v.y;
    }
    out[t] = s;
  }
}

// One CTA per translation unit (A_p at level l-1, B at level L-l) and RHS.
//   PF (o = sigma, i = c): R = e(x0(A_sigma), p^{B_c}_u), T^c, P = conj e(x0(A_sigma), p^B_t)
//   XF (o = sigma, i = c): R = conj e(x^{A_p}_u, p0(B_c)), T^{sigma T}, Q = e(x^{A_sigma}_t, p0(B_c))
//   PA (o = c, i = sigma): R = e(x0(A_sigma), p^B_t), T^{c T}, Q = conj e(x0(A_sigma), p^{B_c}_u)
//   XA (o = c, i = sigma): R = conj e(x^{A_sigma}_t, p0(B_c)), T^sigma, P = e(x^{A_p}_u, p0(B_c))
template <int Q, int VV>
__global__ void __launch_bounds__(kThr) k3_trans(Tab3 tb, G3 g, Mats<Q> mt, const double2 *__restrict__ in,
                                                 double2 *__restrict__ out) {
  constexpr int Q3 = Q * Q * Q;
  constexpr bool FWD = VV == V_PF || VV == V_XF;
  constexpr bool TR = VV == V_XF || VV == V_PA;
  extern __shared__ __align__(16) unsigned char smem3[];
  double2 *in_s = (double2 *)smem3;  // [8][Q3]
  double2 *v = in_s + 8 * Q3, *w1 = v + Q3, *w2 = w1 + Q3, *acc = w2 + Q3;
  const int l = g.l, lb = g.L - l, e = g.e, r = blockIdx.y;
  const long long nBl = nbox_b(lb, e), nBc = nbox_b(lb + 1, e);
  const long long u_ = blockIdx.x;
  const long long ap = u_ / nBl, b = u_ - ap * nBl;
  const Box3 apb = adec(ap, l - 1), bb = bdec(b, lb, e);
  // pair index of A_p's child s with B (level l), and of A_p with B's child c (level l-1)
  auto pair_a = [&](int s_) { return aenc(child(apb, s_), l) * nBl + b; };
  auto pair_b = [&](int c) { return ap * nBc + benc(child(bb, c), lb + 1, e); };
  for (int i = 0; i < 8; i++) {
    const long long pr = FWD ? pair_b(i) : pair_a(i);
    for (int t = threadIdx.x; t < Q3; t += kThr) in_s[i * Q3 + t] = in[(pr * g.nrhs + r) * Q3 + t];
  }
  for (int o = 0; o < 8; o++) {
    for (int t = threadIdx.x; t < Q3; t += kThr) acc[t] = make_double2(0.0, 0.0);
    for (int i = 0; i < 8; i++) {
      const int sg = FWD ? o : i, c = FWD ? i : o;  // child of A_p, child of B
      const Box3 as = child(apb, sg), bc = child(bb, c);
      __syncthreads();  // in_s complete (first pass); v, w1, w2 free
      for (int t = threadIdx.x; t < Q3; t += kThr) {
        const int t1 = t / (Q * Q), t2 = (t / Q) % Q, t3 = t % Q;
        double2 R;
        if (VV == V_PF) R = expi64(thp(tb, g, xat(tb, g.ph, l, as, Q, Q, Q, Q), lb + 1, bc, t1, t2, t3));
        if (VV == V_XF) R = cj(expi64(thp(tb, g, xat(tb, g.ph, l - 1, apb, t1, t2, t3, Q), lb + 1, bc, Q, Q, Q)));
        if (VV == V_PA) R = expi64(thp(tb, g, xat(tb, g.ph, l, as, Q, Q, Q, Q), lb, bb, t1, t2, t3));
        if (VV == V_XA) R = cj(expi64(thp(tb, g, xat(tb, g.ph, l, as, t1, t2, t3, Q), lb + 1, bc, Q, Q, Q)));
        v[t] = cm(R, in_s[i * Q3 + t]);
      }
      __syncthreads();
      const int kk = (VV == V_PF || VV == V_PA) ? c : sg;  // whose translation matrix
      pass3<Q, 2, TR>(mt, kk & 1, v, w1);
      __syncthreads();
      pass3<Q, 1, TR>(mt, (kk >> 1) & 1, w1, w2);
      __syncthreads();
      pass3<Q, 0, TR>(mt, kk >> 2, w2, w1);
      __syncthreads();
      for (int t = threadIdx.x; t < Q3; t += kThr) {
        const int t1 = t / (Q * Q), t2 = (t / Q) % Q, t3 = t % Q;
        double2 x = w1[t];
        if (VV == V_XF) x = cm(expi64(thp(tb, g, xat(tb, g.ph, l, as, t1, t2, t3, Q), lb + 1, bc, Q, Q, Q)), x);
        if (VV == V_PA) x = cm(cj(expi64(thp(tb, g, xat(tb, g.ph, l, as, Q, Q, Q, Q), lb + 1, bc, t1, t2, t3))), x);
        acc[t].x += x.x;
        acc[t].y += x.y;
      }
    }
    __syncthreads();
    const long long po = FWD ? pair_a(o) : pair_b(o);
    const Box3 as = child(apb, o), bc = child(bb, o);
    for (int t = threadIdx.x; t < Q3; t += kThr) {
      const int t1 = t / (Q * Q), t2 = (t / Q) % Q, t3 = t % Q;
      double2 x = acc[t];
      if (VV == V_PF) x = cm(cj(expi64(thp(tb, g, xat(tb, g.ph, l, as, Q, Q, Q, Q), lb, bb, t1, t2, t3))), x);
      if (VV == V_XA) x = cm(expi64(thp(tb, g, xat(tb, g.ph, l - 1, apb, t1, t2, t3, Q), lb + 1, bc, Q, Q, Q)), x);
      out[(po * g.nrhs + r) * Q3 + t] = x;
    }
  }
}

}  // namespace f3

namespace f3 {

// Switch (3D form of eq. alg2m) at level lm, one CTA per pair (A, B) and RHS:
//   FWD: out[t] = sum_u e(x^A_t, p^B_u) in[u];   !FWD: out[u] = sum_t conj e(x^A_t, p^B_u) in[t].
template <int Q, bool FWD>
__global__ void __launch_bounds__(kThr) k3_switch(Tab3 tb, G3 g, const double2 *__restrict__ in,
                                                  double2 *__restrict__ out) {
  constexpr int Q3 = Q * Q * Q;
  __shared__ double2 in_s[Q3];
  const int l = g.l, lb = g.L - l, e = g.e, r = blockIdx.y;
  const long long pr = blockIdx.x, nB = nbox_b(lb, e);
  const long long a = pr / nB, b = pr - a * nB;
  const Box3 ab = adec(a, l), bb = bdec(b, lb, e);
  const double2 *src = in + (pr * g.nrhs + r) * Q3;
  for (int t = threadIdx.x; t < Q3; t += kThr) in_s[t] = src[t];
  __syncthreads();
  for (int o = threadIdx.x; o < Q3; o += kThr) {
    const int o1 = o / (Q * Q), o2 = (o / Q) % Q, o3 = o % Q;
    double2 s = make_double2(0.0, 0.0);
    if (FWD) {
      const XP x = xat(tb, g.ph, l, ab, o1, o2, o3, Q);
      for (int u = 0; u < Q3; u++) {
        const double2 k = expi64(thp(tb, g, x, lb, bb, u / (Q * Q), (u / Q) % Q, u % Q));
        const double2 p = cm(k, in_s[u]);
        s.x += p.x;
        s.y += p.y;
      }
    } else {
      for (int t = 0; t < Q3; t++) {
        const XP x = xat(tb, g.ph, l, ab, t / (Q * Q), (t / Q) % Q, t % Q, Q);
        const double2 k = cj(expi64(thp(tb, g, x, lb, bb, o1, o2, o3)));
        const double2 p = cm(k, in_s[t]);
        s.x += p.x;
        s.y += p.y;
      }
    }
    out[(pr * g.nrhs + r) * Q3 + o] = s;
  }
}

// Termination (3D form of eq. alg2d), A at level l1, summed over the boxes B at level s in
// order: u(x) = sum_B e(x, p0(B)) sum_t L^A_t(x) conj e(x^A_t, p0(B)) delta^{AB}_t.
// One CTA per (box A, RHS); M = 2^s grid points per axis in A; the interpolation one axis
// at a time (V), the M^3 outputs accumulated in registers.
template <int Q>
__global__ void __launch_bounds__(kThr) k3_term(Tab3 tb, const XN3 *__restrict__ xg, G3 g, Mats<Q> mt,
                                                const double2 *__restrict__ st, double2 *__restrict__ u) {
  constexpr int Q3 = Q * Q * Q, MM = 8, PT = (MM * MM * MM + kThr - 1) / kThr;
  __shared__ double2 src[Q3], w1[Q * Q * MM], w2[Q * MM * MM];
  const int l = g.l, lb = g.L - l, e = g.e, r = blockIdx.y, M = 1 << g.s, M3 = M * M * M;
  const long long A = blockIdx.x, nB = nbox_b(lb, e);
  const Box3 ab = adec(A, l);
  const long long NNN = (long long)g.N * g.N * g.N;
  double2 acc[PT];
#pragma unroll
  for (int c = 0; c < PT; c++) acc[c] = make_double2(0.0, 0.0);
  for (long long B = 0; B < nB; B++) {
    const Box3 bb = bdec(B, lb, e);
    __syncthreads();
    for (int t = threadIdx.x; t < Q3; t += kThr) {
      const XP x = xat(tb, g.ph, l, ab, t / (Q * Q), (t / Q) % Q, t % Q, Q);
      src[t] = cm(cj(expi64(thp(tb, g, x, lb, bb, Q, Q, Q))), st[((A * nB + B) * g.nrhs + r) * Q3 + t]);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < Q * Q * M; idx += kThr) {  // w1[t1][t2][m3]
      const int tq = idx / M, m3 = idx % M;
      double2 s = make_double2(0.0, 0.0);
#pragma unroll
      for (int t3 = 0; t3 < Q; t3++) {
        s.x += mt.V[m3][t3] * src[tq * Q + t3].x;
        s.y += mt.V[m3][t3] * src[tq * Q + t3].y;
      }
      w1[idx] = s;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < Q * M * M; idx += kThr) {  // w2[t1][m2][m3]
      const int t1 = idx / (M * M), m2 = (idx / M) % M, m3 = idx % M;
      double2 s = make_double2(0.0, 0.0);
#pragma unroll
      for (int t2 = 0; t2 < Q; t2++) {
        s.x += mt.V[m2][t2] * w1[(t1 * Q + t2) * M + m3].x;
        s.y += mt.V[m2][t2] * w1[(t1 * Q + t2) * M + m3].y;
      }
      w2[idx] = s;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < PT; c++) {
      const int j = threadIdx.x + c * kThr;
      if (j < M3) {
        const int m1 = j / (M * M), m2 = (j / M) % M, m3 = j % M;
        double2 s = make_double2(0.0, 0.0);
#pragma unroll
        for (int t1 = 0; t1 < Q; t1++) {
          s.x += mt.V[m1][t1] * w2[(t1 * M + m2) * M + m3].x;
          s.y += mt.V[m1][t1] * w2[(t1 * M + m2) * M + m3].y;
        }
        const XP x = xpoint(g.ph, xg[ab.c0 * M + m1], xg[ab.c1 * M + m2], xg[ab.c2 * M + m3]);
        const double2 p = cm(expi64(thp(tb, g, x, lb, bb, Q, Q, Q)), s);
        acc[c].x += p.x;
        acc[c].y += p.y;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < PT; c++) {
    const int j = threadIdx.x + c * kThr;
    if (j < M3) {
      const long long i1 = ab.c0 * M + j / (M * M), i2 = ab.c1 * M + (j / M) % M, i3 = ab.c2 * M + j % M;
      u[(long long)r * NNN + (i1 * g.N + i2) * g.N + i3] = acc[c];
    }
  }
}

// Conjugate transpose of the termination, one CTA per (box A, RHS): for every B at level s,
//   delta^{AB}_t = e(x^A_t, p0(B)) sum_{x in A} L^A_t(x) conj e(x, p0(B)) g(x).
template <int Q>
__global__ void __launch_bounds__(kThr) k3_term_adj(Tab3 tb, const XN3 *__restrict__ xg, G3 g, Mats<Q> mt,
                                                    const double2 *__restrict__ gin, double2 *__restrict__ st) {
  constexpr int Q3 = Q * Q * Q, MM = 8;
  __shared__ double2 gv[MM * MM * MM], v[MM * MM * MM], w1[MM * MM * Q], w2[MM * Q * Q];
  const int l = g.l, lb = g.L - l, e = g.e, r = blockIdx.y, M = 1 << g.s, M3 = M * M * M;
  const long long A = blockIdx.x, nB = nbox_b(lb, e);
  const Box3 ab = adec(A, l);
  const long long NNN = (long long)g.N * g.N * g.N;
  for (int j = threadIdx.x; j < M3; j += kThr) {
    const long long i1 = ab.c0 * M + j / (M * M), i2 = ab.c1 * M + (j / M) % M, i3 = ab.c2 * M + j % M;
    gv[j] = gin[(long long)r * NNN + (i1 * g.N + i2) * g.N + i3];
  }
  for (long long B = 0; B < nB; B++) {
    const Box3 bb = bdec(B, lb, e);
    __syncthreads();
    for (int j = threadIdx.x; j < M3; j += kThr) {
      const int m1 = j / (M * M), m2 = (j / M) % M, m3 = j % M;
      const XP x = xpoint(g.ph, xg[ab.c0 * M + m1], xg[ab.c1 * M + m2], xg[ab.c2 * M + m3]);
      v[j] = cm(cj(expi64(thp(tb, g, x, lb, bb, Q, Q, Q))), gv[j]);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < M * M * Q; idx += kThr) {  // w1[m1][m2][t3]
      const int mm = idx / Q, t3 = idx % Q;
      double2 s = make_double2(0.0, 0.0);
      for (int m3 = 0; m3 < M; m3++) {
        s.x += mt.V[m3][t3] * v[mm * M + m3].x;
        s.y += mt.V[m3][t3] * v[mm * M + m3].y;
      }
      w1[idx] = s;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < M * Q * Q; idx += kThr) {  // w2[m1][t2][t3]
      const int m1 = idx / (Q * Q), t2 = (idx / Q) % Q, t3 = idx % Q;
      double2 s = make_double2(0.0, 0.0);
      for (int m2 = 0; m2 < M; m2++) {
        s.x += mt.V[m2][t2] * w1[(m1 * M + m2) * Q + t3].x;
        s.y += mt.V[m2][t2] * w1[(m1 * M + m2) * Q + t3].y;
      }
      w2[idx] = s;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < Q3; t += kThr) {
      const int t1 = t / (Q * Q), t23 = t % (Q * Q);
      double2 s = make_double2(0.0, 0.0);
      for (int m1 = 0; m1 < M; m1++) {
        s.x += mt.V[m1][t1] * w2[m1 * Q * Q + t23].x;
        s.y += mt.V[m1][t1] * w2[m1 * Q * Q + t23].y;
      }
      const XP x = xat(tb, g.ph, l, ab, t1, t23 / Q, t23 % Q, Q);
      st[((A * nB + B) * g.nrhs + r) * Q3 + t] = cm(expi64(thp(tb, g, x, lb, bb, Q, Q, Q)), s);
    }
  }
}

}  // namespace f3

// ------------------------------------------------------------------ host side

struct fio3_plan_s {
  f3::Tab3 tb;
  const f3::XN3 *xg;  // the N grid coordinates i/N (device)
  f3::Ph3 ph;
  int N, L, q, s, e, l0, lm, l1, nrhs_max, maxsrc, nbox_init, device, smem_optin;
  double T[2][f3::kQ3Max][f3::kQ3Max];
  double V[8][f3::kQ3Max];
  void *tables;
  void *state[2];
  long long table_bytes, state_bytes;
};

namespace {

using namespace f3;

int f3fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  fio::set_last_error(buf);
  return code;
}

const double kTwoPi3 = 6.283185307179586476925286766559;

// Lagrange polynomials of the q-point Chebyshev grid z_j = cos(j pi / (q-1)) / 2 at t
// (barycentric form; the weights of that grid are (-1)^j, halved at both ends).
void lagr(int q, const double *z, double t, double *out) {
  for (int j = 0; j < q; j++)
    if (t == z[j]) {
      for (int i = 0; i < q; i++) out[i] = i == j ? 1.0 : 0.0;
      return;
    }
  double den = 0.0;
  for (int j = 0; j < q; j++) {
    double w = (j & 1) ? -1.0 : 1.0;
    if (j == 0 || j == q - 1) w *= 0.5;
    out[j] = w / (t - z[j]);
    den += out[j];
  }
  for (int j = 0; j < q; j++) out[j] /= den;
}

template <int Q> Mats<Q> mats_of(const fio3_plan_s *p) {
  Mats<Q> m;
  for (int sg = 0; sg < 2; sg++)
    for (int i = 0; i < Q; i++)
      for (int j = 0; j < Q; j++) m.T[sg][i][j] = p->T[sg][i][j];
  for (int i = 0; i < 8; i++)
    for (int j = 0; j < Q; j++) m.V[i][j] = p->V[i][j];
  return m;
}

G3 geom3(const fio3_plan_s *p, int l, int nrhs) {
  G3 g;
  g.L = p->L;
  g.e = p->e;
  g.q = p->q;
  g.s = p->s;
  g.l = l;
  g.nrhs = nrhs;
  g.N = p->N;
  g.ph = p->ph;
  return g;
}

long long nbox_h(int lb, int e) { return (1LL << lb) << (2 * (lb + e)); }

template <int Q> int run3(const fio3_plan_s *p, bool fwd, const void *in, void *out, int nrhs, cudaStream_t st) {
  constexpr int Q3 = Q * Q * Q;
  const Mats<Q> mt = mats_of<Q>(p);
  double2 *S[2] = {(double2 *)p->state[0], (double2 *)p->state[1]};
  int cur = 0;
  const size_t tsmem = (size_t)12 * Q3 * sizeof(double2);
  auto trans = [&](int vv, int l) {
    const long long nunits = (1LL << (3 * (l - 1))) * nbox_h(p->L - l, p->e);
    dim3 grid((unsigned)nunits, (unsigned)nrhs);
    const G3 g = geom3(p, l, nrhs);
    switch (vv) {
    case V_PF:
      cudaFuncSetAttribute(k3_trans<Q, V_PF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem);
      k3_trans<Q, V_PF><<<grid, kThr, tsmem, st>>>(p->tb, g, mt, S[cur], S[cur ^ 1]);
      break;
    case V_XF:
      cudaFuncSetAttribute(k3_trans<Q, V_XF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem);
      k3_trans<Q, V_XF><<<grid, kThr, tsmem, st>>>(p->tb, g, mt, S[cur], S[cur ^ 1]);
      break;
    case V_PA:
      cudaFuncSetAttribute(k3_trans<Q, V_PA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem);
      k3_trans<Q, V_PA><<<grid, kThr, tsmem, st>>>(p->tb, g, mt, S[cur], S[cur ^ 1]);
      break;
    default:
      cudaFuncSetAttribute(k3_trans<Q, V_XA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem);
      k3_trans<Q, V_XA><<<grid, kThr, tsmem, st>>>(p->tb, g, mt, S[cur], S[cur ^ 1]);
    }
    cur ^= 1;
  };
  const long long pairs = ((long long)p->N * p->N * p->N) << (2 * p->e);
  if (fwd) {
    k3_init<Q><<<dim3((unsigned)p->nbox_init, nrhs), kThr, 0, st>>>(p->tb, geom3(p, p->l0, nrhs), (const double2 *)in,
                                                                   S[cur]);
    for (int l = p->l0 + 1; l <= p->lm; l++) trans(V_PF, l);
    k3_switch<Q, true><<<dim3((unsigned)pairs, nrhs), kThr, 0, st>>>(p->tb, geom3(p, p->lm, nrhs), S[cur], S[cur ^ 1]);
    cur ^= 1;
    for (int l = p->lm + 1; l <= p->l1; l++) trans(V_XF, l);
    const long long nA = 1LL << (3 * p->l1);
    k3_term<Q><<<dim3((unsigned)nA, nrhs), kThr, 0, st>>>(p->tb, p->xg, geom3(p, p->l1, nrhs), mt, S[cur],
                                                         (double2 *)out);
  } else {
    const long long nA = 1LL << (3 * p->l1);
    k3_term_adj<Q><<<dim3((unsigned)nA, nrhs), kThr, 0, st>>>(p->tb, p->xg, geom3(p, p->l1, nrhs), mt,
                                                             (const double2 *)in, S[cur]);
    for (int l = p->l1; l >= p->lm + 1; l--) trans(V_XA, l);
    k3_switch<Q, false><<<dim3((unsigned)pairs, nrhs), kThr, 0, st>>>(p->tb, geom3(p, p->lm, nrhs), S[cur],
                                                                     S[cur ^ 1]);
    cur ^= 1;
    for (int l = p->lm; l >= p->l0 + 1; l--) trans(V_PA, l);
    k3_init_adj<Q><<<dim3((unsigned)p->nbox_init, nrhs), kThr, 0, st>>>(p->tb, geom3(p, p->l0, nrhs), S[cur],
                                                                       (double2 *)out);
  }
  const cudaError_t ce = cudaGetLastError();
  return ce == cudaSuccess ? 0 : (int)ce;
}

int apply3(fio3_plan_t p, bool fwd, const void *in, void *out, int nrhs, void *stream) {
  if (!p) return f3fail(FIO_EINVAL, "plan is NULL");
  if (!in || !out) return f3fail(FIO_EINVAL, "NULL data pointer");
  if (((uintptr_t)in | (uintptr_t)out) & 15) return f3fail(FIO_EINVAL, "data pointers must be 16-byte aligned");
  if (nrhs < 1 || nrhs > p->nrhs_max) return f3fail(FIO_EINVAL, "nrhs=%d outside [1, %d]", nrhs, p->nrhs_max);
  const size_t bytes = (size_t)nrhs * p->N * p->N * p->N * 16;
  if ((const char *)in < (const char *)out + bytes && (const char *)out < (const char *)in + bytes)
    return f3fail(FIO_EINVAL, "input and output overlap");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != p->device) return f3fail(FIO_EINVAL, "plan was built on device %d but device %d is current", p->device, dev);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = p->q == 3 ? run3<3>(p, fwd, in, out, nrhs, st)
           : p->q == 5 ? run3<5>(p, fwd, in, out, nrhs, st)
                       : run3<7>(p, fwd, in, out, nrhs, st);
  if (rc) return f3fail(FIO_ECUDA, "%s: %s", fwd ? "fio3_apply" : "fio3_apply_adjoint", cudaGetErrorString((cudaError_t)rc));
  return FIO_OK;
}

}  // namespace

extern "C" {

int fio3_plan(fio3_plan_t *out, int N, int q, int phase_id, const double *params, int nparams, int nrhs_max, int s,
              int e) {
  if (!out) return f3fail(FIO_EINVAL, "out is NULL");
  *out = nullptr;
  int L = 0;
  while ((1 << L) < N && L < 30) L++;
  if (N < 4 || N > 256 || (1 << L) != N) return f3fail(FIO_EINVAL, "N=%d must be a power of two in [4, 256]", N);
  if (q != 3 && q != 5 && q != 7) return f3fail(FIO_EINVAL, "q=%d must be 3, 5 or 7", q);
  if (phase_id != FIO3_PHASE_LINEAR && phase_id != FIO3_PHASE_SPHERE) return f3fail(FIO_EINVAL, "unknown phase_id %d", phase_id);
  if (phase_id == FIO3_PHASE_SPHERE && (nparams != 4 || !params || params[2] == 0.0))
    return f3fail(FIO_EINVAL, "the sphere phase needs params [a, m, b, lambda] with b != 0");
  if (nrhs_max < 1) return f3fail(FIO_EINVAL, "nrhs_max=%d must be >= 1", nrhs_max);
  if (s < 0) s = 3;
  if (s > L / 2) s = L / 2;
  if (s > 3) return f3fail(FIO_EINVAL, "s=%d must be <= 3", s);
  if (e < 0) e = 1;
  if (e > 3) return f3fail(FIO_EINVAL, "e=%d must be in [0, 3]", e);
  if (L + e >= kMaxLev) return f3fail(FIO_EINVAL, "N and e too large");
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return f3fail(FIO_EDEVICE, "no CUDA device: %s", cudaGetErrorString(ce));

  fio3_plan_s *p = new (std::nothrow) fio3_plan_s();
  if (!p) return f3fail(FIO_ENOMEM, "host allocation failed");
  p->N = N;
  p->L = L;
  p->q = q;
  p->s = s;
  p->e = e;
  p->l0 = s;
  p->lm = L / 2;
  p->l1 = L - s;
  p->nrhs_max = nrhs_max;
  p->device = dev;
  cudaDeviceGetAttribute(&p->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  p->ph.id = phase_id;
  if (phase_id == FIO3_PHASE_SPHERE) {
    p->ph.a = params[0];
    p->ph.m = params[1];
    p->ph.ib = 1.0 / params[2];
    p->ph.lam = params[3];
  }
  double z[kQ3Max], lg[kQ3Max];
  for (int j = 0; j < q; j++) z[j] = 0.5 * std::cos(j * M_PI / (q - 1));
  memset(p->T, 0, sizeof p->T);
  memset(p->V, 0, sizeof p->V);
  for (int sg = 0; sg < 2; sg++)
    for (int jp = 0; jp < q; jp++) {
      lagr(q, z, (2 * sg - 1) / 4.0 + 0.5 * z[jp], lg);
      for (int j = 0; j < q; j++) p->T[sg][j][jp] = lg[j];
    }
  const int M = 1 << s;
  for (int m = 0; m < M; m++) {
    lagr(q, z, (double)m / M - 0.5, lg);
    for (int j = 0; j < q; j++) p->V[m][j] = lg[j];
  }
  // node tables: x per level 0..L, rho per radial level 0..L, angular per level 0..L+e
  std::vector<XN3> xn;
  std::vector<double> rho;
  std::vector<PA3> pa;
  for (int l = 0; l <= L + e; l++) {
    const double w = 1.0 / (double)(1LL << l);
    if (l <= L) {
      p->tb.xoff[l] = (int)xn.size();
      p->tb.roff[l] = (int)rho.size();
    }
    p->tb.aoff[l] = (int)pa.size();
    for (long long b = 0; b < (1LL << l); b++)
      for (int j = 0; j <= q; j++) {
        const double c = (b + 0.5 + (j < q ? z[j] : 0.0)) * w;
        if (l <= L) {
          xn.push_back({c, std::sin(kTwoPi3 * c)});
          rho.push_back(0.5 * std::sqrt(3.0) * N * c);
        }
        pa.push_back({std::sin(M_PI * c), std::cos(M_PI * c), std::cos(kTwoPi3 * c), std::sin(kTwoPi3 * c)});
      }
  }
  std::vector<XN3> xg(N);
  for (int i = 0; i < N; i++) xg[i] = {(double)i / N, std::sin(kTwoPi3 * ((double)i / N))};
  // sources: spherical coordinates, initialization box at level L - s, sorted by box
  const int lb0 = L - s;
  const long long nb1 = 1LL << lb0, nb2 = 1LL << (lb0 + e), nbox = nb1 * nb2 * nb2;
  const long long n3 = (long long)N * N * N;
  std::vector<double> sp(3 * n3);
  std::vector<long long> bk(n3);
  std::vector<int> cnt(nbox + 1, 0);
  auto boxi = [](double v, long long n) {
    long long b = (long long)std::floor(v * (double)n);
    return b > n - 1 ? n - 1 : b;
  };
  for (long long k = 0; k < n3; k++) {
    const int k1 = (int)(k / ((long long)N * N)) - N / 2, k2 = (int)((k / N) % N) - N / 2, k3 = (int)(k % N) - N / 2;
    const double kk = (double)k1 * k1 + (double)k2 * k2 + (double)k3 * k3, r = std::sqrt(kk);
    double *pk = &sp[3 * k];
    pk[0] = 2.0 * r / (std::sqrt(3.0) * N);
    if (r == 0.0) {
      pk[1] = pk[2] = 0.0;
    } else {
      pk[1] = std::acos(k3 / r) / M_PI;
      double az = std::atan2((double)k2, (double)k1) / kTwoPi3;
      if (az < 0.0) az += 1.0;
      if (k1 == 0 && k2 == 0) az = 0.0;
      pk[2] = az;
    }
    bk[k] = (boxi(pk[0], nb1) * nb2 + boxi(pk[1], nb2)) * nb2 + boxi(pk[2], nb2);
    cnt[bk[k] + 1]++;
  }
  int maxsrc = 0;
  for (long long b = 0; b < nbox; b++) {
    maxsrc = std::max(maxsrc, cnt[b + 1]);
    cnt[b + 1] += cnt[b];
  }
  std::vector<int> pos(cnt.begin(), cnt.end() - 1), srcf(n3);
  std::vector<double> srcw(3 * q * n3);
  for (long long k = 0; k < n3; k++) {
    const int j = pos[bk[k]]++;
    srcf[j] = (int)k;
    const long long b1 = bk[k] / (nb2 * nb2), b2 = (bk[k] / nb2) % nb2, b3 = bk[k] % nb2;
    const double *pk = &sp[3 * k];
    lagr(q, z, (pk[0] - (b1 + 0.5) / (double)nb1) * (double)nb1, &srcw[(size_t)j * 3 * q]);
    lagr(q, z, (pk[1] - (b2 + 0.5) / (double)nb2) * (double)nb2, &srcw[(size_t)j * 3 * q + q]);
    lagr(q, z, (pk[2] - (b3 + 0.5) / (double)nb2) * (double)nb2, &srcw[(size_t)j * 3 * q + 2 * q]);
  }
  p->maxsrc = maxsrc;
  p->nbox_init = (int)nbox;
  // one device allocation for the tables
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t bx = al(xn.size() * sizeof(XN3)), br = al(rho.size() * 8), bp = al(pa.size() * sizeof(PA3)),
               bg = al(N * sizeof(XN3)), bo = al(cnt.size() * 4), bf = al(srcf.size() * 4), bw = al(srcw.size() * 8);
  p->table_bytes = (long long)(bx + br + bp + bg + bo + bf + bw);
  const size_t sb = (size_t)n3 * ((size_t)1 << (2 * e)) * nrhs_max * q * q * q * 16;
  p->state_bytes = 2LL * (long long)sb;
  if ((ce = cudaMalloc(&p->tables, p->table_bytes)) != cudaSuccess) {
    delete p;
    return f3fail(FIO_ENOMEM, "cudaMalloc(tables): %s", cudaGetErrorString(ce));
  }
  for (int i = 0; i < 2; i++)
    if ((ce = cudaMalloc(&p->state[i], sb)) != cudaSuccess) {
      fio3_destroy(p);
      return f3fail(FIO_ENOMEM, "cudaMalloc(state, %zu bytes): %s", sb, cudaGetErrorString(ce));
    }
  char *d = (char *)p->tables;
  auto up = [&](const void *src, size_t n, size_t span) {
    void *dst = d;
    cudaMemcpy(dst, src, n, cudaMemcpyHostToDevice);
    d += span;
    return dst;
  };
  p->tb.xn = (const XN3 *)up(xn.data(), xn.size() * sizeof(XN3), bx);
  p->tb.rho = (const double *)up(rho.data(), rho.size() * 8, br);
  p->tb.pa = (const PA3 *)up(pa.data(), pa.size() * sizeof(PA3), bp);
  p->xg = (const XN3 *)up(xg.data(), N * sizeof(XN3), bg);
  p->tb.box_off = (const int *)up(cnt.data(), cnt.size() * 4, bo);
  p->tb.src_f = (const int *)up(srcf.data(), srcf.size() * 4, bf);
  p->tb.src_w = (const double *)up(srcw.data(), srcw.size() * 8, bw);
  if ((ce = cudaGetLastError()) != cudaSuccess) {
    fio3_destroy(p);
    return f3fail(FIO_ECUDA, "table upload: %s", cudaGetErrorString(ce));
  }
  *out = p;
  return FIO_OK;
}

int fio3_destroy(fio3_plan_t p) {
  if (!p) return FIO_OK;
  cudaDeviceSynchronize();
  cudaFree(p->state[0]);
  cudaFree(p->state[1]);
  cudaFree(p->tables);
  delete p;
  return FIO_OK;
}

int fio3_apply(fio3_plan_t p, const void *f, void *u, int nrhs, void *stream) { return apply3(p, true, f, u, nrhs, stream); }

int fio3_apply_adjoint(fio3_plan_t p, const void *g, void *fbar, int nrhs, void *stream) {
  return apply3(p, false, g, fbar, nrhs, stream);
}

int fio3_plan_info(fio3_plan_t p, fio3_plan_info_t *info) {
  if (!p || !info) return f3fail(FIO_EINVAL, "NULL argument");
  memset(info, 0, sizeof *info);
  info->N = p->N;
  info->L = p->L;
  info->q = p->q;
  info->s = p->s;
  info->e = p->e;
  info->l0 = p->l0;
  info->lm = p->lm;
  info->l1 = p->l1;
  info->phase_id = p->ph.id;
  info->nrhs_max = p->nrhs_max;
  info->pairs_per_level = ((long long)p->N * p->N * p->N) << (2 * p->e);
  info->state_bytes = p->state_bytes;
  info->table_bytes = p->table_bytes;
  info->max_box_sources = p->maxsrc;
  return FIO_OK;
}

}  // extern "C"
