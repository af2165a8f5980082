// fio_df.cuh -- double-float ("df") arithmetic on the FP32 pipe and the FP32
// form's phase evaluation.
//
// A df value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  The algorithms are the classical error-free
// transformations: TwoSum (Knuth), Fast-TwoSum (Dekker 1971) and TwoProduct with
// a fused multiply-add (Ogita, Rump & Oishi 2005); the square root takes one
// Newton correction from the FP32 root (Dekker 1971).
//
// The FP32 form needs each phase theta = Phi(x, kappa(p)) modulo 1 to ~1e-8
// absolute although |theta| reaches ~N; df keeps ~1e-14 relative, i.e. ~1e-11
// absolute at N = 1024, and runs on the FMA pipe, which GB300 executes ~70x
// faster than FP64.  The reduced phase r = theta - rint(theta) is formed from
// hi - rint(hi), which is exact, plus lo, and then goes to an FP32 sin/cos.
//
// The phases are homogeneous of degree 1 in k (Sec. 1), so for a T_P node with
// polar coordinates (p1, p2): theta(x, p) = rho(p1) G(x, phi(p2)) with
// rho = (sqrt2/2) N p1 and G(x, phi) = Phi(x, (cos 2 pi p2, sin 2 pi p2)).
#pragma once
#include "fio_common.cuh"

namespace fio {

struct df {
  float h, l;
};

__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ df df_add(df a, df b) {
  const df s = df_two_sum(a.h, b.h);
  return df_fast_two_sum(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = a.h * b.h;
  const float e = __fmaf_rn(a.h, b.h, -p);
  return df_fast_two_sum(p, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e)));
}
__device__ __forceinline__ df df_mulf(df a, float b) {
  const float p = a.h * b;
  const float e = __fmaf_rn(a.h, b, -p);
  return df_fast_two_sum(p, __fmaf_rn(a.l, b, e));
}
__device__ __forceinline__ df df_sqr(df a) {
  const float p = a.h * a.h;
  const float e = __fmaf_rn(a.h, a.h, -p);
  return df_fast_two_sum(p, __fmaf_rn(2.0f * a.h, a.l, e));
}
// sqrt of a positive df (returns 0 for 0)
__device__ __forceinline__ df df_sqrt(df a) {
  if (a.h <= 0.0f) return {0.0f, 0.0f};
  const float h = __fsqrt_rn(a.h);
  const float p = h * h;
  const float e = __fmaf_rn(h, h, -p);
  const float r = ((a.h - p) - e) + a.l;
  return df_fast_two_sum(h, __fdividef(r, 2.0f * h));
}

// Host-side split of a double into a df.
__host__ __forceinline__ df df_split(double v) {
  df d;
  d.h = (float)v;
  d.l = (float)(v - (double)d.h);
  return d;
}

// df copies of the node tables (FIO_F32 plans).
struct XNodeF {
  df x, s, c;  // x, sin 2 pi x, cos 2 pi x
};
struct P1NodeF {
  df rho;  // (sqrt2/2) N p1
};
struct P2NodeF {
  df c, s;  // cos 2 pi p2, sin 2 pi p2
};
struct SrcF {
  float k1, k2;  // exact integer frequencies
};

// Phase constants as df.
struct PhaseF {
  int id;
  df a, m, ib, lam;
};

// Per-x quantities of the homogeneous phases: the point and its speed(s).
struct XDesc {
  df x1, x2, c1, c2;  // c1, c2: ellipse axes (c1 = speed for the circle)
};

__device__ __forceinline__ XDesc xdesc(const PhaseF &P, const XNodeF &u, const XNodeF &v) {
  XDesc d;
  d.x1 = u.x;
  d.x2 = v.x;
  if (P.id == 1) {
    d.c1 = df_mul(df_add(P.a, df_mul(P.m, df_mul(u.s, v.s))), P.ib);
    d.c2 = df_mul(df_add(P.a, df_mul(P.m, df_mul(u.c, v.c))), P.ib);
  } else if (P.id == 2) {
    d.c1 = df_mul(df_add(P.a, df_mul(P.m, df_mul(u.s, v.s))), P.ib);
    d.c2 = {0.f, 0.f};
  } else {
    d.c1 = d.c2 = {0.f, 0.f};
  }
  return d;
}

// G(x, phi) = Phi(x, (cos, sin)) for the homogeneous phases (ids 0, 1, 2).
__device__ __forceinline__ df g_eval(const PhaseF &P, const XDesc &x, const P2NodeF &v) {
  df lin = df_add(df_mul(x.x1, v.c), df_mul(x.x2, v.s));
  if (P.id == 0) return lin;
  lin = df_mul(P.lam, lin);
  if (P.id == 2) return df_add(lin, x.c1);
  const df h2 = df_add(df_sqr(df_mul(x.c1, v.c)), df_sqr(df_mul(x.c2, v.s)));
  return df_add(lin, df_sqrt(h2));
}

// Phi(x, k) at an integer lattice frequency (exact in float).
__device__ __forceinline__ df theta_k(const PhaseF &P, const XDesc &x, float k1, float k2) {
  df lin = df_add(df_mulf(x.x1, k1), df_mulf(x.x2, k2));
  if (P.id == 0) return lin;
  lin = df_mul(P.lam, lin);
  if (P.id == 2) return df_add(lin, df_mul(x.c1, df_sqrt({k1 * k1 + k2 * k2, 0.f})));  // |k|^2 exact in float
  const df h2 = df_add(df_sqr(df_mulf(x.c1, k1)), df_sqr(df_mulf(x.c2, k2)));
  return df_add(lin, df_sqrt(h2));
}

// e^{2 pi i theta} from a df theta: exact reduction of hi, then FP32 sin/cos.
__device__ __forceinline__ float2 expi_df(df th) {
  const float r = (th.h - rintf(th.h)) + th.l;
  float s, c;
  sincospif(2.0f * r, &s, &c);
  return make_float2(c, s);
}

}  // namespace fio
