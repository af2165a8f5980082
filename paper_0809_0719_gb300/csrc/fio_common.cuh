// fio_common.cuh -- types and device helpers shared by the butterfly kernels.
//
// Notation (Candes, Demanet & Ying 2008): N = 2^L, q Chebyshev points per
// dimension, pairs (A, B) with A a box of T_X at level l and B a box of T_P at
// level L - l.  A box of T_P at level j is 2^-j wide in p1 and 2^-(j+e) wide in
// p2 (angular refinement e).  theta(x, p) = N Psi(x, p) = Phi(x, kappa(p)),
// kappa(p) = (sqrt2/2) N p1 (cos 2 pi p2, sin 2 pi p2) (Sec. 1.1, eq. polar).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fio {

constexpr int kQMax = 11;     // largest compiled q
constexpr int kMMax = 64;     // largest 2^s (termination box side)
constexpr int kThreads = 256; // threads per CTA of every kernel

template <typename R> struct C2;
template <> struct C2<float> { typedef float2 T; };
template <> struct C2<double> { typedef double2 T; };

template <typename R> __device__ __forceinline__ typename C2<R>::T cmk(R x, R y) {
  typename C2<R>::T v;
  v.x = x;
  v.y = y;
  return v;
}
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  V r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
// conj(a) * b
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {
  V r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.x * b.y - a.y * b.x;
  return r;
}

// One coordinate of a box's Chebyshev node (or centre) in T_X: x, sin 2 pi x, cos 2 pi x.
struct XNode {
  double x, s, c;
};
// One p1 coordinate of a T_P node: p1 and rho = (sqrt2/2) N p1.
struct P1Node {
  double p1, rho;
};
// One p2 coordinate of a T_P node: cos 2 pi p2, sin 2 pi p2.
struct P2Node {
  double c, s;
};

// Phase function Phi and its constants, FP64.
struct Phase {
  int id;     // 0 linear, 1 ellipse, 2 circle, 3 separable (test)
  double a, m, ib, lam;  // ellipse / circle: speed = (a + m * trig) * ib, ib = 1/b
  double sa, sm, sb, sl; // separable: N (sa sin cos + sm x1 x2 + sb p1 cos2pi p2 + sl p1^2)
  double N;
};

// theta at x = (x1, x2) and a p-node given by p1 (P1Node) and p2 (P2Node).
__device__ __forceinline__ double theta_xp(const Phase &P, const XNode &x1, const XNode &x2, const P1Node &u,
                                           const P2Node &v) {
  if (P.id == 3) {
    return P.N * (P.sa * x1.s * x2.c + P.sm * x1.x * x2.x + P.sb * u.p1 * v.c + P.sl * u.p1 * u.p1);
  }
  const double k1 = u.rho * v.c, k2 = u.rho * v.s;
  const double lin = x1.x * k1 + x2.x * k2;
  if (P.id == 0) return lin;
  if (P.id == 1) {
    const double c1 = (P.a + P.m * x1.s * x2.s) * P.ib;
    const double c2 = (P.a + P.m * x1.c * x2.c) * P.ib;
    return P.lam * lin + sqrt(c1 * c1 * k1 * k1 + c2 * c2 * k2 * k2);
  }
  const double c = (P.a + P.m * x1.s * x2.s) * P.ib;
  return P.lam * lin + c * u.rho;
}

// theta at x and a lattice source k (exact integer coordinates; kr = |k|, p1, cos 2 pi p2 for
// the separable test phase).
struct Src {
  double k1, k2, kr, p1, c2;
};
__device__ __forceinline__ double theta_xk(const Phase &P, const XNode &x1, const XNode &x2, const Src &k) {
  if (P.id == 3) {
    return P.N * (P.sa * x1.s * x2.c + P.sm * x1.x * x2.x + P.sb * k.p1 * k.c2 + P.sl * k.p1 * k.p1);
  }
  const double lin = x1.x * k.k1 + x2.x * k.k2;
  if (P.id == 0) return lin;
  if (P.id == 1) {
    const double c1 = (P.a + P.m * x1.s * x2.s) * P.ib;
    const double c2 = (P.a + P.m * x1.c * x2.c) * P.ib;
    return P.lam * lin + sqrt(c1 * c1 * k.k1 * k.k1 + c2 * c2 * k.k2 * k.k2);
  }
  const double c = (P.a + P.m * x1.s * x2.s) * P.ib;
  return P.lam * lin + c * k.kr;
}

// e^{2 pi i theta}: theta reduced modulo 1 in FP64, then sin/cos in the working precision.
template <typename R> __device__ __forceinline__ typename C2<R>::T expi(double th);
template <> __device__ __forceinline__ double2 expi<double>(double th) {
  const double r = th - rint(th);
  double s, c;
  sincospi(2.0 * r, &s, &c);
  return make_double2(c, s);
}
template <> __device__ __forceinline__ float2 expi<float>(double th) {
  const float r = (float)(th - rint(th));
  float s, c;
  sincospif(2.0f * r, &s, &c);
  return make_float2(c, s);
}

// Device tables of a plan (all FP64 unless noted).
struct Tables {
  const XNode *xnode;   // per T_X level l: 2^l boxes x (q+1) entries (node j<q, centre j=q), at xoff[l]
  const P1Node *p1node; // per T_P level j: 2^j x (q+1), at p1off[j]
  const P2Node *p2node; // per T_P level j: 2^(j+e) x (q+1), at p2off[j]
  const XNode *xgrid;   // N entries: x = i/N
  const Src *src;       // sources sorted by initialization box
  const int *src_f;     // flat index (k1+N/2)*N + (k2+N/2) of each sorted source
  const double *src_w;  // 2q Lagrange weights per sorted source: L_j(phat1), then L_j(phat2)
  const int *box_off;   // initialization box b -> first sorted source; size nbox+1
  int xoff[13], p1off[13], p2off[13];
};

// Per-launch geometry.
struct Geom {
  int L, e, q, s;
  int l;     // level of this step (A's level of the pairs written, or read for adjoint steps)
  int nrhs;  // RHS stride of the state and of f/u
  int rt;    // RHS per CTA
  int U;     // units per CTA
  long long nunits;
};

__device__ __forceinline__ const XNode &xn(const Tables &tb, int l, int box, int j, int q) {
  return tb.xnode[tb.xoff[l] + box * (q + 1) + j];
}
__device__ __forceinline__ const P1Node &pn1(const Tables &tb, int j, int box, int t, int q) {
  return tb.p1node[tb.p1off[j] + box * (q + 1) + t];
}
__device__ __forceinline__ const P2Node &pn2(const Tables &tb, int j, int box, int t, int q) {
  return tb.p2node[tb.p2off[j] + box * (q + 1) + t];
}

}  // namespace fio
