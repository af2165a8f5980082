/*
 * fio_oracle3.c -- TEST INFRASTRUCTURE ONLY.
 *
 * The three-dimensional form of the butterfly FIO method of Candes, Demanet &
 * Ying (2008): the paper states that the algorithm carries over to three
 * dimensions with a three-dimensional Chebyshev grid for the interpolation of
 * e^{2 pi i R^{AB}(x,k)}, and reports it for the phase of eq. ex3,
 *     Phi(x,k) = x.k + c(x)|k|,  c(x) = (3 + sin 2pi x1 sin 2pi x2 sin 2pi x3)/4   (Table 3).
 * This file is a plain FP64 statement of that method (forward apply and its exact
 * conjugate transpose, the adjoint butterfly), in the
 * same order and notation as the two-dimensional oracle (fio_oracle.c), for
 * the tests only.  It shares no code with the CUDA library, nor with the
 * two-dimensional oracle (the small helpers are restated here).
 *
 *   u(x) = sum_{k in Omega} e^{2 pi i Phi(x,k)} f(k),  x in X = {0..N-1}^3 / N,
 *   Omega = {-N/2 .. N/2-1}^3; f[(k1+N/2) N^2 + (k2+N/2) N + (k3+N/2)], u[i1 N^2 + i2 N + i3].
 *
 * Phases (params [a, m, b, lambda]):
 *   0  linear x.k (no params used)
 *   2  sphere phase lambda x.k + c(x)|k|, c(x) = (a + m sin 2pi x1 sin 2pi x2 sin 2pi x3)/b
 *      (eq. ex3 is [3, 1, 4, 1]); lambda = m = 0 gives an x-independent phase.
 *
 * Readings taken for three dimensions (the paper gives no formulas for them):
 *   S1 spherical coordinates in frequency, the analogue of the polar map of Sec. 1.1:
 *      k = (sqrt3/2) N p1 (sin pi p2 cos 2pi p3, sin pi p2 sin 2pi p3, cos pi p2),
 *      p1 = 2|k|/(sqrt3 N) in [0,1], p2 = acos(k3/|k|)/pi in [0,1],
 *      p3 = atan2(k2,k1)/(2 pi) in [0,1); k = 0 maps to p = (0,0,0).
 *   S2 a box of T_P at level j has width 2^-j in p1 and 2^-(j+e) in p2 and in p3
 *      (angular refinement e, as in two dimensions); a box of T_X at level j is the
 *      cube of side 2^-j.  Box index at level j: min(floor(p 2^j), 2^j - 1).
 *   S3 levels are balanced (l(A) + l(B) = L), the recursion runs from A at level s
 *      to A at level L-s with the switch at lm = floor(L/2), and the termination
 *      sums the partial potentials of the boxes B at level s: as in two dimensions.
 * Every value is double; complex values use C99 complex.  OpenMP parallelises
 * the loops over independent outputs only; no sum is reordered.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC3_LINEAR 0
#define ORC3_SPHERE 2
#define ORC3_QMAX 9

static const double ORC3_TWO_PI = 6.283185307179586476925286766559;

typedef struct {
  int id, N;
  double prm[4];
} orc3_phase;

/* ---------------------------------------------------------------- phases */

/* Phi(x,k) at a Cartesian frequency k. */
static double orc3_phi(const orc3_phase *ph, const double *x, const double *k) {
  double lin = x[0] * k[0] + x[1] * k[1] + x[2] * k[2];
  if (ph->id == ORC3_LINEAR) return lin;
  double c = (ph->prm[0] + ph->prm[1] * sin(ORC3_TWO_PI * x[0]) * sin(ORC3_TWO_PI * x[1]) * sin(ORC3_TWO_PI * x[2])) /
             ph->prm[2];
  return ph->prm[3] * lin + c * sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
}

/* Spherical coordinates of a lattice frequency (reading S1). */
static void orc3_sph(int N, int k1, int k2, int k3, double *p) {
  double kk = (double)k1 * k1 + (double)k2 * k2 + (double)k3 * k3;
  double r = sqrt(kk);
  p[0] = 2.0 * r / (sqrt(3.0) * N);
  if (r == 0.0) {
    p[1] = p[2] = 0.0;
    return;
  }
  p[1] = acos(k3 / r) / M_PI;
  double az = atan2((double)k2, (double)k1) / ORC3_TWO_PI;
  if (az < 0.0) az += 1.0;
  if (k1 == 0 && k2 == 0) az = 0.0;
  p[2] = az;
}

/* kappa(p): the frequency of spherical coordinates p (reading S1). */
static void orc3_kappa(int N, const double *p, double *k) {
  double r = 0.5 * sqrt(3.0) * N * p[0];
  k[0] = r * sin(M_PI * p[1]) * cos(ORC3_TWO_PI * p[2]);
  k[1] = r * sin(M_PI * p[1]) * sin(ORC3_TWO_PI * p[2]);
  k[2] = r * cos(M_PI * p[1]);
}

/* theta(x,p) = Phi(x, kappa(p)). */
static double orc3_theta(const orc3_phase *ph, const double *x, const double *p) {
  double k[3];
  orc3_kappa(ph->N, p, k);
  return orc3_phi(ph, x, k);
}

/* e^{2 pi i t} with t reduced to [-1/2, 1/2] first. */
static double complex orc3_expi(double t) {
  double r = t - rint(t);
  return cos(ORC3_TWO_PI * r) + I * sin(ORC3_TWO_PI * r);
}

/* ------------------------------------------- Chebyshev grid, Lagrange basis */

/* z_i = cos(i pi / (q-1)) / 2 (Sec. 3.2). */
static void orc3_cheb(int q, double *z) {
  for (int i = 0; i < q; i++) z[i] = 0.5 * cos(i * M_PI / (q - 1));
}

/* L_i(t) = prod_{j != i} (t - z_j) / (z_i - z_j) (Sec. 3.2). */
static double orc3_lag(int q, const double *z, int i, double t) {
  double v = 1.0;
  for (int j = 0; j < q; j++)
    if (j != i) v *= (t - z[j]) / (z[i] - z[j]);
  return v;
}

/* -------------------------------------------------------------- direct sum */

void orc3_spherical_map(int N, int k1, int k2, int k3, double *p) { orc3_sph(N, k1, k2, k3, p); }

double orc3_theta_xp(int phase_id, const double *prm, int N, const double *x, const double *p) {
  orc3_phase ph = {phase_id, N, {prm[0], prm[1], prm[2], prm[3]}};
  return orc3_theta(&ph, x, p);
}

/* u[j] = sum_k e^{2 pi i Phi(x_j,k)} f(k) at the flat grid indices xi[j] = i1 N^2 + i2 N + i3. */
void orc3_direct(int N, int phase_id, const double *prm, const double complex *f, int nx, const long *xi,
                 double complex *u) {
  orc3_phase ph = {phase_id, N, {prm[0], prm[1], prm[2], prm[3]}};
  long n3 = (long)N * N * N;
#pragma omp parallel for schedule(dynamic, 16)
  for (int j = 0; j < nx; j++) {
    long x = xi[j];
    double xx[3] = {(double)(x / ((long)N * N)) / N, (double)((x / N) % N) / N, (double)(x % N) / N};
    double complex acc = 0;
    for (long k = 0; k < n3; k++) {
      double kk[3] = {(double)(k / ((long)N * N)) - N / 2, (double)((k / N) % N) - N / 2, (double)(k % N) - N / 2};
      acc += orc3_expi(orc3_phi(&ph, xx, kk)) * f[k];
    }
    u[j] = acc;
  }
}

/* ------------------------------------------------------------- butterfly */

typedef struct {
  orc3_phase ph;
  int N, L, q, q3, s, l0, lm, l1, e;
  double z[ORC3_QMAX];
  /* lag3[c][t][u]: the parent's 3D Lagrange polynomial t at the node u of child
   * c = 4 s1 + 2 s2 + s3 (the translation matrix of the 3D forms of eqs. alg2b, alg2c) */
  double *lag3;
  double *sp;  /* spherical coordinates of every lattice frequency, 3 per source */
} orc3_bf;

static int orc3_bf_init(orc3_bf *bf, int N, int q, int phase_id, const double *prm, int s, int lm, int e) {
  int L = 0;
  while ((1 << L) < N) L++;
  if ((1 << L) != N || N < 2 || q < 2 || q > ORC3_QMAX) return -1;
  if (phase_id != ORC3_LINEAR && phase_id != ORC3_SPHERE) return -1;
  if (phase_id == ORC3_SPHERE && prm[2] == 0.0) return -1;
  if (s < 0) s = 3;
  if (s > L / 2) s = L / 2;
  if (lm < 0) lm = L / 2;
  if (lm < s || lm > L - s) return -1;
  if (e < 0 || e > 3) return -1;
  bf->ph.id = phase_id;
  bf->ph.N = N;
  for (int i = 0; i < 4; i++) bf->ph.prm[i] = prm[i];
  bf->N = N;
  bf->L = L;
  bf->q = q;
  bf->q3 = q * q * q;
  bf->s = s;
  bf->l0 = s;
  bf->lm = lm;
  bf->l1 = L - s;
  bf->e = e;
  orc3_cheb(q, bf->z);
  int q3 = bf->q3;
  bf->lag3 = malloc(sizeof(double) * 8 * q3 * q3);
  for (int c = 0; c < 8; c++) {
    int sg[3] = {c >> 2, (c >> 1) & 1, c & 1};
    for (int t = 0; t < q3; t++)
      for (int u = 0; u < q3; u++) {
        int td[3] = {t / (q * q), (t / q) % q, t % q}, ud[3] = {u / (q * q), (u / q) % q, u % q};
        double v = 1.0;
        for (int d = 0; d < 3; d++) v *= orc3_lag(q, bf->z, td[d], (2 * sg[d] - 1) / 4.0 + bf->z[ud[d]] / 2.0);
        bf->lag3[((long)c * q3 + t) * q3 + u] = v;
      }
  }
  long n3 = (long)N * N * N;
  bf->sp = malloc(sizeof(double) * 3 * n3);
  for (long k = 0; k < n3; k++)
    orc3_sph(N, (int)(k / ((long)N * N)) - N / 2, (int)((k / N) % N) - N / 2, (int)(k % N) - N / 2, &bf->sp[3 * k]);
  return 0;
}

static void orc3_bf_free(orc3_bf *bf) {
  free(bf->lag3);
  free(bf->sp);
}

/* Box geometry (reading S2): centre and node t of a box of side 2^-j along one axis. */
static double orc3_ctr(int j, int i) { return (i + 0.5) / (double)(1 << j); }
static double orc3_node(const orc3_bf *bf, int j, int i, int t) { return orc3_ctr(j, i) + bf->z[t] / (double)(1 << j); }
static int orc3_box(double p, int j) {
  int n = 1 << j;
  int b = (int)floor(p * n);
  return b > n - 1 ? n - 1 : b;
}

/* Boxes: A at T_X level l is (a1,a2,a3) in [0,2^l)^3; B at T_P level lb is (b1,b2,b3) with
 * b1 in [0,2^lb) and b2, b3 in [0,2^(lb+e)).  Flat indices and their decoding. */
static void orc3_adec(int l, long a, int *ad) {
  long n = 1L << l;
  ad[0] = (int)(a / (n * n));
  ad[1] = (int)((a / n) % n);
  ad[2] = (int)(a % n);
}
static void orc3_bdec(const orc3_bf *bf, int lb, long b, int *bd) {
  long n2 = 1L << (lb + bf->e);
  bd[0] = (int)(b / (n2 * n2));
  bd[1] = (int)((b / n2) % n2);
  bd[2] = (int)(b % n2);
}
static long orc3_aenc(int l, const int *ad) {
  long n = 1L << l;
  return ((long)ad[0] * n + ad[1]) * n + ad[2];
}
static long orc3_benc(const orc3_bf *bf, int lb, const int *bd) {
  long n2 = 1L << (lb + bf->e);
  return ((long)bd[0] * n2 + bd[1]) * n2 + bd[2];
}
static long orc3_nb(const orc3_bf *bf, int lb) { return (1L << lb) << (2 * (lb + bf->e)); }

/* centre x0(A), node x^A_t, centre p0(B), node p^B_t */
static void orc3_xc(int l, const int *ad, double *x) {
  for (int d = 0; d < 3; d++) x[d] = orc3_ctr(l, ad[d]);
}
static void orc3_xn(const orc3_bf *bf, int l, const int *ad, int t, double *x) {
  int q = bf->q, td[3] = {t / (q * q), (t / q) % q, t % q};
  for (int d = 0; d < 3; d++) x[d] = orc3_node(bf, l, ad[d], td[d]);
}
static void orc3_pc(const orc3_bf *bf, int lb, const int *bd, double *p) {
  p[0] = orc3_ctr(lb, bd[0]);
  p[1] = orc3_ctr(lb + bf->e, bd[1]);
  p[2] = orc3_ctr(lb + bf->e, bd[2]);
}
static void orc3_pn(const orc3_bf *bf, int lb, const int *bd, int t, double *p) {
  int q = bf->q, td[3] = {t / (q * q), (t / q) % q, t % q};
  p[0] = orc3_node(bf, lb, bd[0], td[0]);
  p[1] = orc3_node(bf, lb + bf->e, bd[1], td[1]);
  p[2] = orc3_node(bf, lb + bf->e, bd[2], td[2]);
}

/* State at level l: pairs (A at level l, B at level L-l), q^3 coefficients each,
 * index (a nB + b) q^3 + t. */
static long orc3_idx(const orc3_bf *bf, int l, long a, long b, int t) {
  return (a * orc3_nb(bf, bf->L - l) + b) * bf->q3 + t;
}

/* Initialization (3D form of eq. alg2a), A at level l0, B at level L-l0:
 * delta^{AB}_t = e^{-2 pi i theta(x0(A),p^B_t)} sum_{p in B} L^B_t(p) e^{2 pi i Phi(x0(A),k)} f(k). */
static void orc3_init(const orc3_bf *bf, const double complex *f, double complex *st) {
  int N = bf->N, q = bf->q, q3 = bf->q3, l = bf->l0, lb = bf->L - l;
  long nA = 1L << (3 * l), nB = orc3_nb(bf, lb), n3 = (long)N * N * N;
  long *cnt = calloc((size_t)(nB + 1), sizeof(long)), *lst = malloc(sizeof(long) * n3), *pos = malloc(sizeof(long) * nB);
  long *bk = malloc(sizeof(long) * n3);
  for (long k = 0; k < n3; k++) {
    int bd[3] = {orc3_box(bf->sp[3 * k], lb), orc3_box(bf->sp[3 * k + 1], lb + bf->e),
                 orc3_box(bf->sp[3 * k + 2], lb + bf->e)};
    bk[k] = orc3_benc(bf, lb, bd);
    cnt[bk[k] + 1]++;
  }
  for (long b = 0; b < nB; b++) cnt[b + 1] += cnt[b];
  memcpy(pos, cnt, sizeof(long) * nB);
  for (long k = 0; k < n3; k++) lst[pos[bk[k]]++] = k;
#pragma omp parallel for schedule(dynamic, 1)
  for (long a = 0; a < nA; a++) {
    int ad[3];
    double x0[3];
    orc3_adec(l, a, ad);
    orc3_xc(l, ad, x0);
    double complex *acc = malloc(sizeof(double complex) * q3);
    for (long b = 0; b < nB; b++) {
      int bd[3];
      double p0[3];
      orc3_bdec(bf, lb, b, bd);
      orc3_pc(bf, lb, bd, p0);
      for (int t = 0; t < q3; t++) acc[t] = 0;
      for (long j = cnt[b]; j < cnt[b + 1]; j++) {
        long k = lst[j];
        double kk[3] = {(double)(k / ((long)N * N)) - N / 2, (double)((k / N) % N) - N / 2, (double)(k % N) - N / 2};
        double h[3] = {(bf->sp[3 * k] - p0[0]) * (1 << lb), (bf->sp[3 * k + 1] - p0[1]) * (1 << (lb + bf->e)),
                       (bf->sp[3 * k + 2] - p0[2]) * (1 << (lb + bf->e))};
        double w[3][ORC3_QMAX];
        for (int d = 0; d < 3; d++)
          for (int i = 0; i < q; i++) w[d][i] = orc3_lag(q, bf->z, i, h[d]);
        double complex v = orc3_expi(orc3_phi(&bf->ph, x0, kk)) * f[k];
        for (int t = 0; t < q3; t++) acc[t] += w[0][t / (q * q)] * w[1][(t / q) % q] * w[2][t % q] * v;
      }
      for (int t = 0; t < q3; t++) {
        double pt[3];
        orc3_pn(bf, lb, bd, t, pt);
        st[orc3_idx(bf, l, a, b, t)] = conj(orc3_expi(orc3_theta(&bf->ph, x0, pt))) * acc[t];
      }
    }
    free(acc);
  }
  free(cnt);
  free(lst);
  free(pos);
  free(bk);
}

/* Recursion in p (3D form of eq. alg2b), level l-1 -> l:
 * delta^{AB}_t = e^{-2 pi i theta(x0(A),p^B_t)} sum_c sum_u L^B_t(p^{Bc}_u) e^{2 pi i theta(x0(A),p^{Bc}_u)} delta^{Ap Bc}_u. */
static void orc3_step_p(const orc3_bf *bf, int l, const double complex *in, double complex *out) {
  int q3 = bf->q3, lb = bf->L - l;
  long nA = 1L << (3 * l), nB = orc3_nb(bf, lb);
#pragma omp parallel for schedule(dynamic, 1)
  for (long a = 0; a < nA; a++) {
    int ad[3], apd[3];
    double x0[3];
    orc3_adec(l, a, ad);
    orc3_xc(l, ad, x0);
    for (int d = 0; d < 3; d++) apd[d] = ad[d] / 2;
    long ap = orc3_aenc(l - 1, apd);
    double complex *src = malloc(sizeof(double complex) * 8 * q3);
    for (long b = 0; b < nB; b++) {
      int bd[3];
      orc3_bdec(bf, lb, b, bd);
      for (int c = 0; c < 8; c++) {
        int cd[3] = {2 * bd[0] + (c >> 2), 2 * bd[1] + ((c >> 1) & 1), 2 * bd[2] + (c & 1)};
        long bc = orc3_benc(bf, lb + 1, cd);
        for (int u = 0; u < q3; u++) {
          double pu[3];
          orc3_pn(bf, lb + 1, cd, u, pu);
          src[c * q3 + u] = orc3_expi(orc3_theta(&bf->ph, x0, pu)) * in[orc3_idx(bf, l - 1, ap, bc, u)];
        }
      }
      for (int t = 0; t < q3; t++) {
        double complex acc = 0;
        for (int c = 0; c < 8; c++)
          for (int u = 0; u < q3; u++) acc += bf->lag3[((long)c * q3 + t) * q3 + u] * src[c * q3 + u];
        double pt[3];
        orc3_pn(bf, lb, bd, t, pt);
        out[orc3_idx(bf, l, a, b, t)] = conj(orc3_expi(orc3_theta(&bf->ph, x0, pt))) * acc;
      }
    }
    free(src);
  }
}

/* Switch (3D form of eq. alg2m) at level lm: delta^{AB}_t <- sum_u e^{2 pi i theta(x^A_t,p^B_u)} delta^{AB}_u. */
static void orc3_switch(const orc3_bf *bf, const double complex *in, double complex *out) {
  int q3 = bf->q3, l = bf->lm, lb = bf->L - l;
  long nA = 1L << (3 * l), nB = orc3_nb(bf, lb);
#pragma omp parallel for schedule(dynamic, 1)
  for (long a = 0; a < nA; a++) {
    int ad[3];
    orc3_adec(l, a, ad);
    for (long b = 0; b < nB; b++) {
      int bd[3];
      orc3_bdec(bf, lb, b, bd);
      for (int t = 0; t < q3; t++) {
        double xt[3];
        orc3_xn(bf, l, ad, t, xt);
        double complex acc = 0;
        for (int u = 0; u < q3; u++) {
          double pu[3];
          orc3_pn(bf, lb, bd, u, pu);
          acc += orc3_expi(orc3_theta(&bf->ph, xt, pu)) * in[orc3_idx(bf, l, a, b, u)];
        }
        out[orc3_idx(bf, l, a, b, t)] = acc;
      }
    }
  }
}

/* Recursion in x (3D form of eq. alg2c), level l-1 -> l:
 * delta^{AB}_t = sum_c e^{2 pi i theta(x^A_t,p0(Bc))} sum_u L^{Ap}_u(x^A_t) e^{-2 pi i theta(x^{Ap}_u,p0(Bc))} delta^{Ap Bc}_u. */
static void orc3_step_x(const orc3_bf *bf, int l, const double complex *in, double complex *out) {
  int q3 = bf->q3, lb = bf->L - l;
  long nA = 1L << (3 * l), nB = orc3_nb(bf, lb);
#pragma omp parallel for schedule(dynamic, 1)
  for (long a = 0; a < nA; a++) {
    int ad[3], apd[3];
    orc3_adec(l, a, ad);
    for (int d = 0; d < 3; d++) apd[d] = ad[d] / 2;
    int sg = 4 * (ad[0] & 1) + 2 * (ad[1] & 1) + (ad[2] & 1);
    long ap = orc3_aenc(l - 1, apd);
    double complex *src = malloc(sizeof(double complex) * 8 * q3);
    for (long b = 0; b < nB; b++) {
      int bd[3];
      orc3_bdec(bf, lb, b, bd);
      double pcs[8][3];
      for (int c = 0; c < 8; c++) {
        int cd[3] = {2 * bd[0] + (c >> 2), 2 * bd[1] + ((c >> 1) & 1), 2 * bd[2] + (c & 1)};
        long bc = orc3_benc(bf, lb + 1, cd);
        orc3_pc(bf, lb + 1, cd, pcs[c]);
        for (int u = 0; u < q3; u++) {
          double xu[3];
          orc3_xn(bf, l - 1, apd, u, xu);
          src[c * q3 + u] = conj(orc3_expi(orc3_theta(&bf->ph, xu, pcs[c]))) * in[orc3_idx(bf, l - 1, ap, bc, u)];
        }
      }
      for (int t = 0; t < q3; t++) {
        double xt[3];
        orc3_xn(bf, l, ad, t, xt);
        double complex acc = 0;
        for (int c = 0; c < 8; c++) {
          double complex part = 0;
          /* L^{Ap}_u(x^A_t): the parent's polynomial u at the child node t */
          for (int u = 0; u < q3; u++) part += bf->lag3[((long)sg * q3 + u) * q3 + t] * src[c * q3 + u];
          acc += orc3_expi(orc3_theta(&bf->ph, xt, pcs[c])) * part;
        }
        out[orc3_idx(bf, l, a, b, t)] = acc;
      }
    }
    free(src);
  }
}

/* Termination (3D form of eq. alg2d), A at level l1, summed over the boxes B at level s:
 * u(x) = sum_B e^{2 pi i theta(x,p0(B))} sum_t L^A_t(x) e^{-2 pi i theta(x^A_t,p0(B))} delta^{AB}_t. */
static void orc3_term(const orc3_bf *bf, const double complex *st, double complex *u) {
  int N = bf->N, q = bf->q, q3 = bf->q3, l = bf->l1, lb = bf->L - l;
  long nA = 1L << (3 * l), nB = orc3_nb(bf, lb);
  int m = N >> l;
#pragma omp parallel for schedule(dynamic, 1)
  for (long a = 0; a < nA; a++) {
    int ad[3];
    double x0[3];
    orc3_adec(l, a, ad);
    orc3_xc(l, ad, x0);
    double complex *src = malloc(sizeof(double complex) * q3);
    for (int m1 = 0; m1 < m; m1++)
      for (int m2 = 0; m2 < m; m2++)
        for (int m3 = 0; m3 < m; m3++)
          u[((long)(ad[0] * m + m1) * N + ad[1] * m + m2) * N + ad[2] * m + m3] = 0;
    for (long b = 0; b < nB; b++) {
      int bd[3];
      double p0[3];
      orc3_bdec(bf, lb, b, bd);
      orc3_pc(bf, lb, bd, p0);
      for (int t = 0; t < q3; t++) {
        double xt[3];
        orc3_xn(bf, l, ad, t, xt);
        src[t] = conj(orc3_expi(orc3_theta(&bf->ph, xt, p0))) * st[orc3_idx(bf, l, a, b, t)];
      }
      for (int m1 = 0; m1 < m; m1++)
        for (int m2 = 0; m2 < m; m2++)
          for (int m3 = 0; m3 < m; m3++) {
            int id[3] = {ad[0] * m + m1, ad[1] * m + m2, ad[2] * m + m3};
            double x[3], w[3][ORC3_QMAX];
            for (int d = 0; d < 3; d++) {
              x[d] = (double)id[d] / N;
              for (int i = 0; i < q; i++) w[d][i] = orc3_lag(q, bf->z, i, (x[d] - x0[d]) * (1 << l));
            }
            double complex part = 0;
            for (int t = 0; t < q3; t++) part += w[0][t / (q * q)] * w[1][(t / q) % q] * w[2][t % q] * src[t];
            u[((long)id[0] * N + id[1]) * N + id[2]] += orc3_expi(orc3_theta(&bf->ph, x, p0)) * part;
          }
    }
    free(src);
  }
}

/* ---------------------------------------------------- adjoint butterfly */

/* Conjugate transpose of the termination: for every A at level l1 and B at level s,
 * d_t = e^{2 pi i theta(x^A_t,p0B)} sum_{x in A} L^A_t(x) e^{-2 pi i theta(x,p0B)} g(x). */
static void orc3_adj_term(const orc3_bf *bf, const double complex *g, double complex *st) {
  int N = bf->N, q = bf->q, q3 = bf->q3, l = bf->l1, lb = bf->L - l;
  long nA = 1L << (3 * l), nB = orc3_nb(bf, lb);
  int m = N >> l, m3 = m * m * m;
#pragma omp parallel for schedule(dynamic, 1)
  for (long a = 0; a < nA; a++) {
    int ad[3];
    double x0[3];
    orc3_adec(l, a, ad);
    orc3_xc(l, ad, x0);
    double complex *v = malloc(sizeof(double complex) * m3);
    double *w = malloc(sizeof(double) * 3 * m * q);  /* w[d][m_d][i] = L_i of the local offset m_d */
    for (int d = 0; d < 3; d++)
      for (int md = 0; md < m; md++)
        for (int i = 0; i < q; i++)
          w[(d * m + md) * q + i] = orc3_lag(q, bf->z, i, ((double)(ad[d] * m + md) / N - x0[d]) * (1 << l));
    for (long b = 0; b < nB; b++) {
      int bd[3];
      double p0[3];
      orc3_bdec(bf, lb, b, bd);
      orc3_pc(bf, lb, bd, p0);
      /* e^{-2 pi i theta(x,p0B)} g(x) for the grid points x of A */
      for (int j = 0; j < m3; j++) {
        int id[3] = {ad[0] * m + j / (m * m), ad[1] * m + (j / m) % m, ad[2] * m + j % m};
        double x[3] = {(double)id[0] / N, (double)id[1] / N, (double)id[2] / N};
        v[j] = conj(orc3_expi(orc3_theta(&bf->ph, x, p0))) * g[((long)id[0] * N + id[1]) * N + id[2]];
      }
      for (int t = 0; t < q3; t++) {
        int td[3] = {t / (q * q), (t / q) % q, t % q};
        double complex acc = 0;
        for (int j = 0; j < m3; j++) {
          int md[3] = {j / (m * m), (j / m) % m, j % m};
          acc += w[(0 * m + md[0]) * q + td[0]] * w[(1 * m + md[1]) * q + td[1]] * w[(2 * m + md[2]) * q + td[2]] * v[j];
        }
        double xt[3];
        orc3_xn(bf, l, ad, t, xt);
        st[orc3_idx(bf, l, a, b, t)] = orc3_expi(orc3_theta(&bf->ph, xt, p0)) * acc;
      }
    }
    free(v);
    free(w);
  }
}

/* Conjugate transpose of the x-recursion at level l (l -> l-1):
 * d^{Ap Bc}_u = e^{2 pi i theta(x^{Ap}_u,p0Bc)} sum_{A in Ap} sum_t L^{Ap}_u(x^A_t) e^{-2 pi i theta(x^A_t,p0Bc)} d^{AB}_t. */
static void orc3_adj_x(const orc3_bf *bf, int l, const double complex *in, double complex *out) {
  int q3 = bf->q3, lb = bf->L - l;
  long nAp = 1L << (3 * (l - 1)), nBc = orc3_nb(bf, lb + 1);
#pragma omp parallel for schedule(dynamic, 1)
  for (long ap = 0; ap < nAp; ap++) {
    int apd[3];
    orc3_adec(l - 1, ap, apd);
    double complex *v = malloc(sizeof(double complex) * 8 * q3);
    for (long bc = 0; bc < nBc; bc++) {
      int cd[3], bd[3];
      double pc[3];
      orc3_bdec(bf, lb + 1, bc, cd);
      for (int d = 0; d < 3; d++) bd[d] = cd[d] / 2;
      long b = orc3_benc(bf, lb, bd);
      orc3_pc(bf, lb + 1, cd, pc);
      /* e^{-2 pi i theta(x^A_t,p0Bc)} d^{AB}_t for the eight children A of Ap */
      for (int sg = 0; sg < 8; sg++) {
        int ad[3] = {2 * apd[0] + (sg >> 2), 2 * apd[1] + ((sg >> 1) & 1), 2 * apd[2] + (sg & 1)};
        long a = orc3_aenc(l, ad);
        for (int t = 0; t < q3; t++) {
          double xt[3];
          orc3_xn(bf, l, ad, t, xt);
          v[sg * q3 + t] = conj(orc3_expi(orc3_theta(&bf->ph, xt, pc))) * in[orc3_idx(bf, l, a, b, t)];
        }
      }
      for (int u = 0; u < q3; u++) {
        double complex acc = 0;
        for (int sg = 0; sg < 8; sg++)
          for (int t = 0; t < q3; t++) acc += bf->lag3[((long)sg * q3 + u) * q3 + t] * v[sg * q3 + t];
        double xu[3];
        orc3_xn(bf, l - 1, apd, u, xu);
        out[orc3_idx(bf, l - 1, ap, bc, u)] = orc3_expi(orc3_theta(&bf->ph, xu, pc)) * acc;
      }
    }
    free(v);
  }
}

/* Conjugate transpose of the switch: d_u = sum_t e^{-2 pi i theta(x^A_t,p^B_u)} d_t. */
static void orc3_adj_switch(const orc3_bf *bf, const double complex *in, double complex *out) {
  int q3 = bf->q3, l = bf->lm, lb = bf->L - l;
  long nA = 1L << (3 * l), nB = orc3_nb(bf, lb);
#pragma omp parallel for schedule(dynamic, 1)
  for (long a = 0; a < nA; a++) {
    int ad[3];
    orc3_adec(l, a, ad);
    for (long b = 0; b < nB; b++) {
      int bd[3];
      orc3_bdec(bf, lb, b, bd);
      for (int u = 0; u < q3; u++) {
        double pu[3];
        orc3_pn(bf, lb, bd, u, pu);
        double complex acc = 0;
        for (int t = 0; t < q3; t++) {
          double xt[3];
          orc3_xn(bf, l, ad, t, xt);
          acc += conj(orc3_expi(orc3_theta(&bf->ph, xt, pu))) * in[orc3_idx(bf, l, a, b, t)];
        }
        out[orc3_idx(bf, l, a, b, u)] = acc;
      }
    }
  }
}

/* Conjugate transpose of the p-recursion at level l (l -> l-1):
 * d^{Ap Bc}_u = sum_{A in Ap} e^{-2 pi i theta(x0A,p^{Bc}_u)} sum_t L^B_t(p^{Bc}_u) e^{2 pi i theta(x0A,p^B_t)} d^{AB}_t. */
static void orc3_adj_p(const orc3_bf *bf, int l, const double complex *in, double complex *out) {
  int q3 = bf->q3, lb = bf->L - l;
  long nAp = 1L << (3 * (l - 1)), nB = orc3_nb(bf, lb);
#pragma omp parallel for schedule(dynamic, 1)
  for (long ap = 0; ap < nAp; ap++) {
    int apd[3];
    orc3_adec(l - 1, ap, apd);
    double complex *v = malloc(sizeof(double complex) * 8 * q3);
    for (long b = 0; b < nB; b++) {
      int bd[3];
      orc3_bdec(bf, lb, b, bd);
      double x0s[8][3];
      /* e^{2 pi i theta(x0A,p^B_t)} d^{AB}_t for the eight children A of Ap */
      for (int sg = 0; sg < 8; sg++) {
        int ad[3] = {2 * apd[0] + (sg >> 2), 2 * apd[1] + ((sg >> 1) & 1), 2 * apd[2] + (sg & 1)};
        long a = orc3_aenc(l, ad);
        orc3_xc(l, ad, x0s[sg]);
        for (int t = 0; t < q3; t++) {
          double pt[3];
          orc3_pn(bf, lb, bd, t, pt);
          v[sg * q3 + t] = orc3_expi(orc3_theta(&bf->ph, x0s[sg], pt)) * in[orc3_idx(bf, l, a, b, t)];
        }
      }
      for (int c = 0; c < 8; c++) {
        int cd[3] = {2 * bd[0] + (c >> 2), 2 * bd[1] + ((c >> 1) & 1), 2 * bd[2] + (c & 1)};
        long bc = orc3_benc(bf, lb + 1, cd);
        for (int u = 0; u < q3; u++) {
          double pu[3];
          orc3_pn(bf, lb + 1, cd, u, pu);
          double complex acc = 0;
          for (int sg = 0; sg < 8; sg++) {
            double complex part = 0;
            /* L^B_t(p^{Bc}_u) */
            for (int t = 0; t < q3; t++) part += bf->lag3[((long)c * q3 + t) * q3 + u] * v[sg * q3 + t];
            acc += conj(orc3_expi(orc3_theta(&bf->ph, x0s[sg], pu))) * part;
          }
          out[orc3_idx(bf, l - 1, ap, bc, u)] = acc;
        }
      }
    }
    free(v);
  }
}

/* Conjugate transpose of the initialization:
 * fbar(k) = sum_{A at l0} e^{-2 pi i Phi(x0A,k)} sum_t L^B_t(p(k)) e^{2 pi i theta(x0A,p^B_t)} d^{AB}_t,
 * B the box of p(k) at level L-l0. */
static void orc3_adj_init(const orc3_bf *bf, const double complex *st, double complex *fbar) {
  int N = bf->N, q = bf->q, q3 = bf->q3, l = bf->l0, lb = bf->L - l;
  long nA = 1L << (3 * l), nB = orc3_nb(bf, lb), n3 = (long)N * N * N;
  /* v^{AB}_t = e^{2 pi i theta(x0A,p^B_t)} d^{AB}_t */
  double complex *v = malloc(sizeof(double complex) * nA * nB * q3);
#pragma omp parallel for schedule(dynamic, 1)
  for (long a = 0; a < nA; a++) {
    int ad[3];
    double x0[3];
    orc3_adec(l, a, ad);
    orc3_xc(l, ad, x0);
    for (long b = 0; b < nB; b++) {
      int bd[3];
      orc3_bdec(bf, lb, b, bd);
      for (int t = 0; t < q3; t++) {
        double pt[3];
        orc3_pn(bf, lb, bd, t, pt);
        long i = orc3_idx(bf, l, a, b, t);
        v[i] = orc3_expi(orc3_theta(&bf->ph, x0, pt)) * st[i];
      }
    }
  }
#pragma omp parallel for schedule(dynamic, 16)
  for (long k = 0; k < n3; k++) {
    double kk[3] = {(double)(k / ((long)N * N)) - N / 2, (double)((k / N) % N) - N / 2, (double)(k % N) - N / 2};
    int bd[3] = {orc3_box(bf->sp[3 * k], lb), orc3_box(bf->sp[3 * k + 1], lb + bf->e),
                 orc3_box(bf->sp[3 * k + 2], lb + bf->e)};
    long b = orc3_benc(bf, lb, bd);
    double p0[3];
    orc3_pc(bf, lb, bd, p0);
    double h[3] = {(bf->sp[3 * k] - p0[0]) * (1 << lb), (bf->sp[3 * k + 1] - p0[1]) * (1 << (lb + bf->e)),
                   (bf->sp[3 * k + 2] - p0[2]) * (1 << (lb + bf->e))};
    double w[3][ORC3_QMAX];
    for (int d = 0; d < 3; d++)
      for (int i = 0; i < q; i++) w[d][i] = orc3_lag(q, bf->z, i, h[d]);
    double complex acc = 0;
    for (long a = 0; a < nA; a++) {
      int ad[3];
      double x0[3];
      orc3_adec(l, a, ad);
      orc3_xc(l, ad, x0);
      double complex part = 0;
      for (int t = 0; t < q3; t++) part += w[0][t / (q * q)] * w[1][(t / q) % q] * w[2][t % q] * v[orc3_idx(bf, l, a, b, t)];
      acc += conj(orc3_expi(orc3_phi(&bf->ph, x0, kk))) * part;
    }
    fbar[k] = acc;
  }
  free(v);
}

/* Adjoint direct sum: fbar(k) = sum_x e^{-2 pi i Phi(x,k)} g(x) at flat frequency indices ki. */
void orc3_direct_adjoint(int N, int phase_id, const double *prm, const double complex *g, int nk, const long *ki,
                         double complex *fbar) {
  orc3_phase ph = {phase_id, N, {prm[0], prm[1], prm[2], prm[3]}};
  long n3 = (long)N * N * N;
#pragma omp parallel for schedule(dynamic, 16)
  for (int j = 0; j < nk; j++) {
    long k = ki[j];
    double kk[3] = {(double)(k / ((long)N * N)) - N / 2, (double)((k / N) % N) - N / 2, (double)(k % N) - N / 2};
    double complex acc = 0;
    for (long x = 0; x < n3; x++) {
      double xx[3] = {(double)(x / ((long)N * N)) / N, (double)((x / N) % N) / N, (double)(x % N) / N};
      acc += conj(orc3_expi(orc3_phi(&ph, xx, kk))) * g[x];
    }
    fbar[j] = acc;
  }
}

/*
 * Forward 3D butterfly: f, u are N^3 complex (layout of orc3_direct).  s: truncation
 * depth (-1 = 3, at most floor(L/2)); lm: switch level (-1 = floor(L/2)); e: angular
 * refinement (0..3).  Returns 0, or -1 on bad arguments or allocation failure.
 */
int orc3_butterfly(int N, int q, int phase_id, const double *prm, int s, int lm, int e, const double complex *f,
                   double complex *u) {
  orc3_bf bf;
  if (orc3_bf_init(&bf, N, q, phase_id, prm, s, lm, e)) return -1;
  long sz = ((long)N * N * N << (2 * bf.e)) * bf.q3;
  double complex *a = malloc(sizeof(double complex) * sz), *b = malloc(sizeof(double complex) * sz);
  if (!a || !b) {
    free(a);
    free(b);
    orc3_bf_free(&bf);
    return -1;
  }
  orc3_init(&bf, f, a);
  for (int l = bf.l0 + 1; l <= bf.lm; l++) {
    orc3_step_p(&bf, l, a, b);
    double complex *t = a;
    a = b;
    b = t;
  }
  orc3_switch(&bf, a, b);
  {
    double complex *t = a;
    a = b;
    b = t;
  }
  for (int l = bf.lm + 1; l <= bf.l1; l++) {
    orc3_step_x(&bf, l, a, b);
    double complex *t = a;
    a = b;
    b = t;
  }
  orc3_term(&bf, a, u);
  free(a);
  free(b);
  orc3_bf_free(&bf);
  return 0;
}

/* Adjoint 3D butterfly: fbar = B^H g, the exact conjugate transpose of orc3_butterfly. */
int orc3_butterfly_adjoint(int N, int q, int phase_id, const double *prm, int s, int lm, int e,
                           const double complex *g, double complex *fbar) {
  orc3_bf bf;
  if (orc3_bf_init(&bf, N, q, phase_id, prm, s, lm, e)) return -1;
  long sz = ((long)N * N * N << (2 * bf.e)) * bf.q3;
  double complex *a = malloc(sizeof(double complex) * sz), *b = malloc(sizeof(double complex) * sz);
  if (!a || !b) {
    free(a);
    free(b);
    orc3_bf_free(&bf);
    return -1;
  }
  orc3_adj_term(&bf, g, a);
  for (int l = bf.l1; l >= bf.lm + 1; l--) {
    orc3_adj_x(&bf, l, a, b);
    double complex *t = a;
    a = b;
    b = t;
  }
  orc3_adj_switch(&bf, a, b);
  {
    double complex *t = a;
    a = b;
    b = t;
  }
  for (int l = bf.lm; l >= bf.l0 + 1; l--) {
    orc3_adj_p(&bf, l, a, b);
    double complex *t = a;
    a = b;
    b = t;
  }
  orc3_adj_init(&bf, a, fbar);
  free(a);
  free(b);
  orc3_bf_free(&bf);
  return 0;
}
