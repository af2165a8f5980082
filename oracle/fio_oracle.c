/*
 * fio_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU statement of what the butterfly FIO path computes,
 * written from Candes, Demanet & Ying, "A Fast Butterfly Algorithm for the
 * Computation of Fourier Integral Operators" (2008).  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
 * no code, header, table or helper with the CUDA library: the two are
 * independent statements of the same mathematics.
 *
 * Contents
 *   - phase functions Phi(x,k) and theta(x,p) = N Psi(x,p)      (Sec. 1, eq. polar)
 *   - polar map of the frequency lattice                       (Sec. 1.1, eq. polar)
 *   - Chebyshev grid and Lagrange polynomials, product form    (Sec. 3.2)
 *   - direct O(N^4) sum and its adjoint                        (Sec. 1, eq. dfio)
 *   - the butterfly, step by step in the paper's order           (Sec. 4, eqs. alg2a-alg2d)
 *     with the level truncation of Sec. 5, and its exact
 *     conjugate transpose (the adjoint butterfly).
 *
 * Every floating-point value is double; complex values use C99 complex.
 * The code favours being checkable by eye over speed: the translation steps
 * apply the dense 2D Lagrange matrix of eq. alg2b / alg2c, not the
 * dimension-wise factorisation.  OpenMP parallelises the loops over
 * independent outputs only; no sum is reordered.
 *
 * Readings of the paper taken here (all also listed in the design notes):
 *   R1 levels are balanced, l(A)+l(B)=L; the recursion starts with A at
 *      level s (default 3) and ends with A at level L-s (Sec. 5 truncation);
 *      the switch happens at lm = floor(L/2) (Sec. 4, step 4) unless given.
 *   R2 the polar angle is p2 = atan2(k2,k1)/(2 pi) taken in [0,1); k=0 maps to
 *      p=(0,0); the box index at level j is min(floor(p*2^j), 2^j-1).
 *   R3 the termination sums the partial potentials of the boxes B at level
 *      s (u = sum_B u^B, Sec. 2).
 *   R4 angular refinement e: a box of T_P at level j has width 2^-j in p1 and
 *      2^-(j+e) in p2 (2^j x 2^(j+e) boxes), so the angular side, stretched by
 *      2 pi (sqrt2/2) p1 in k-space, is not wider than the radial one.  e = 0
 *      is the literal square-box statement of Sec. 1.1; e = 2 reproduces the
 *      error decay with q reported in Sec. 5 (about 30x per q+2, flat in N).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_LINEAR 0
#define ORC_ELLIPSE 1
#define ORC_CIRCLE 2
#define ORC_SEPARABLE 3

/* largest q, and largest number of grid points per termination box (2^s)^2 */
#define ORC_QMAX 24
#define ORC_MMAX 4096

static const double TWO_PI = 6.283185307179586476925286766559;

typedef struct {
  int id;
  int N;
  double prm[4];
} orc_phase;

/* ---------------------------------------------------------------- phases */

/* Phi(x,k) for the phases defined on the Cartesian frequency k (Sec. 1, Sec. 5
 * eq. ex1 and eq. ex2 with the scaling constants passed in prm). */
static double orc_phi_xk(const orc_phase *ph, double x1, double x2, double k1, double k2) {
  double a = ph->prm[0], m = ph->prm[1], b = ph->prm[2], lam = ph->prm[3];
  switch (ph->id) {
  case ORC_LINEAR:
    return x1 * k1 + x2 * k2;
  case ORC_ELLIPSE: {
    double c1 = (a + m * sin(TWO_PI * x1) * sin(TWO_PI * x2)) / b;
    double c2 = (a + m * cos(TWO_PI * x1) * cos(TWO_PI * x2)) / b;
    return lam * (x1 * k1 + x2 * k2) + sqrt(c1 * c1 * k1 * k1 + c2 * c2 * k2 * k2);
  }
  case ORC_CIRCLE: {
    double c = (a + m * sin(TWO_PI * x1) * sin(TWO_PI * x2)) / b;
    return lam * (x1 * k1 + x2 * k2) + c * sqrt(k1 * k1 + k2 * k2);
  }
  }
  return 0.0;
}

/* The test-only separable phase, defined directly in p-space:
 * theta = N (alpha(x) + beta(p)).  For it the residual R^{AB} of eq. RAB is
 * identically zero, so every interpolation step is exact. */
static double orc_sep_theta(const orc_phase *ph, double x1, double x2, double p1, double p2) {
  double alpha = ph->prm[0] * sin(TWO_PI * x1) * cos(TWO_PI * x2) + ph->prm[1] * x1 * x2;
  double beta = ph->prm[2] * p1 * cos(TWO_PI * p2) + ph->prm[3] * p1 * p1;
  return (double)ph->N * (alpha + beta);
}

/* Polar map of Sec. 1.1 (eq. polar): k = (sqrt2/2) N p1 (cos 2pi p2, sin 2pi p2). */
static void orc_polar(int N, int k1, int k2, double *p1, double *p2) {
  double kk = (double)k1 * k1 + (double)k2 * k2;
  *p1 = sqrt(2.0 * kk) / N;
  double ang = atan2((double)k2, (double)k1) / TWO_PI;
  if (ang < 0.0) ang += 1.0;
  if (k1 == 0 && k2 == 0) ang = 0.0;
  *p2 = ang;
}

/* theta(x,p) = N Psi(x,p) = Phi(x, kappa(p)) (Sec. 1.1). */
static double orc_theta(const orc_phase *ph, double x1, double x2, double p1, double p2) {
  if (ph->id == ORC_SEPARABLE) return orc_sep_theta(ph, x1, x2, p1, p2);
  double r = 0.5 * sqrt(2.0) * ph->N * p1;
  return orc_phi_xk(ph, x1, x2, r * cos(TWO_PI * p2), r * sin(TWO_PI * p2));
}

/* Phi(x,k) at a lattice frequency k. */
static double orc_theta_k(const orc_phase *ph, double x1, double x2, int k1, int k2) {
  if (ph->id == ORC_SEPARABLE) {
    double p1, p2;
    orc_polar(ph->N, k1, k2, &p1, &p2);
    return orc_sep_theta(ph, x1, x2, p1, p2);
  }
  return orc_phi_xk(ph, x1, x2, (double)k1, (double)k2);
}

/* e^{2 pi i t}, with t reduced to [-1/2,1/2] first so that the argument of
 * cos/sin stays small however large t is. */
static double complex orc_expi(double t) {
  double r = t - rint(t);
  return cos(TWO_PI * r) + I * sin(TWO_PI * r);
}

/* ------------------------------------------- Chebyshev grid, Lagrange basis */

/* z_i = cos(i pi / (q-1)) / 2, i = 0..q-1 (Sec. 3.2). */
static void orc_cheb(int q, double *z) {
  for (int i = 0; i < q; i++) z[i] = 0.5 * cos(i * M_PI / (q - 1));
}

/* L_i(t) = prod_{j != i} (t - z_j) / (z_i - z_j) (Sec. 3.2), product form. */
static double orc_lagrange(int q, const double *z, int i, double t) {
  double v = 1.0;
  for (int j = 0; j < q; j++)
    if (j != i) v *= (t - z[j]) / (z[i] - z[j]);
  return v;
}

/* -------------------------------------------------------------- exported */

int orc_version(void) { return 1; }

int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

void orc_cheb_nodes(int q, double *z) { orc_cheb(q, z); }

/* out[i] = L_i(t) for i = 0..q-1. */
void orc_lagrange_row(int q, double t, double *out) {
  double z[ORC_QMAX];
  orc_cheb(q, z);
  for (int i = 0; i < q; i++) out[i] = orc_lagrange(q, z, i, t);
}

void orc_polar_map(int N, int k1, int k2, double *p) { orc_polar(N, k1, k2, &p[0], &p[1]); }

double orc_theta_xp(int phase_id, const double *prm, int N, double x1, double x2, double p1, double p2) {
  orc_phase ph = {phase_id, N, {prm[0], prm[1], prm[2], prm[3]}};
  return orc_theta(&ph, x1, x2, p1, p2);
}

double orc_phi_k(int phase_id, const double *prm, int N, double x1, double x2, int k1, int k2) {
  orc_phase ph = {phase_id, N, {prm[0], prm[1], prm[2], prm[3]}};
  return orc_theta_k(&ph, x1, x2, k1, k2);
}

/*
 * Direct sum, eq. dfio: u(x) = sum_{k in Omega} e^{2 pi i Phi(x,k)} f(k).
 * f is N x N complex, f[(k1+N/2)*N + (k2+N/2)].  The nx outputs are taken at
 * the flat grid indices xi[j] = i1*N + i2 (x = (i1/N, i2/N)); the inner sum runs
 * over k2 and the outer over k1.
 */
void orc_direct(int N, int phase_id, const double *prm, const double complex *f, int nx, const long *xi,
                double complex *u) {
  orc_phase ph = {phase_id, N, {prm[0], prm[1], prm[2], prm[3]}};
#pragma omp parallel for schedule(dynamic, 1)
  for (int j = 0; j < nx; j++) {
    int i1 = (int)(xi[j] / N), i2 = (int)(xi[j] % N);
    double x1 = (double)i1 / N, x2 = (double)i2 / N;
    double complex acc = 0;
    for (int a = 0; a < N; a++) {
      double complex row = 0;
      for (int b = 0; b < N; b++)
        row += orc_expi(orc_theta_k(&ph, x1, x2, a - N / 2, b - N / 2)) * f[(long)a * N + b];
      acc += row;
    }
    u[j] = acc;
  }
}

/* The same direct sum for nrhs sources at once (f holds nrhs N x N arrays one after
 * another; u[r * nx + j] is RHS r at xi[j]).  Each phase e^{2 pi i Phi(x,k)} is
 * evaluated once and multiplied into every RHS; per RHS the terms are added in the
 * order orc_direct adds them, so each result equals orc_direct's bit for bit. */
void orc_direct_multi(int N, int phase_id, const double *prm, int nrhs, const double complex *f, int nx,
                      const long *xi, double complex *u) {
  orc_phase ph = {phase_id, N, {prm[0], prm[1], prm[2], prm[3]}};
  const long NN = (long)N * N;
#pragma omp parallel for schedule(dynamic, 1)
  for (int j = 0; j < nx; j++) {
    int i1 = (int)(xi[j] / N), i2 = (int)(xi[j] % N);
    double x1 = (double)i1 / N, x2 = (double)i2 / N;
    double complex *acc = calloc((size_t)nrhs, sizeof(double complex));
    double complex *row = malloc(sizeof(double complex) * (size_t)nrhs);
    for (int a = 0; a < N; a++) {
      for (int r = 0; r < nrhs; r++) row[r] = 0;
      for (int b = 0; b < N; b++) {
        const double complex e = orc_expi(orc_theta_k(&ph, x1, x2, a - N / 2, b - N / 2));
        for (int r = 0; r < nrhs; r++) row[r] += e * f[r * NN + (long)a * N + b];
      }
      for (int r = 0; r < nrhs; r++) acc[r] += row[r];
    }
    for (int r = 0; r < nrhs; r++) u[(long)r * nx + j] = acc[r];
    free(acc);
    free(row);
  }
}

/* Adjoint direct sum: fbar(k) = sum_{x in X} e^{-2 pi i Phi(x,k)} g(x), at the
 * flat frequency indices ki[j] = (k1+N/2)*N + (k2+N/2). */
void orc_direct_adjoint(int N, int phase_id, const double *prm, const double complex *g, int nk, const long *ki,
                        double complex *fbar) {
  orc_phase ph = {phase_id, N, {prm[0], prm[1], prm[2], prm[3]}};
#pragma omp parallel for schedule(dynamic, 1)
  for (int j = 0; j < nk; j++) {
    int k1 = (int)(ki[j] / N) - N / 2, k2 = (int)(ki[j] % N) - N / 2;
    double complex acc = 0;
    for (int a = 0; a < N; a++) {
      double complex row = 0;
      for (int b = 0; b < N; b++)
        row += conj(orc_expi(orc_theta_k(&ph, (double)a / N, (double)b / N, k1, k2))) * g[(long)a * N + b];
      acc += row;
    }
    fbar[j] = acc;
  }
}

/* ------------------------------------------------------------- butterfly */

typedef struct {
  orc_phase ph;
  int N, L, q, s, l0, lm, l1, e;
  double z[ORC_QMAX];
  /* Lagrange matrices of the translation steps: lag2[c][t][t'] is the parent's
   * 2D Lagrange polynomial t evaluated at the node t' of child c = 2*s1+s2
   * (L^B_t(p^{Bc}_t') of eq. alg2b; the same numbers are L^{Ap}_t(x^A_t') of
   * eq. alg2c).  Position- and level-independent (Sec. 4). */
  double *lag2;
  /* polar coordinates of every lattice frequency */
  double *p1, *p2;
} orc_bf;

static int orc_bf_init(orc_bf *bf, int N, int q, int phase_id, const double *prm, int s, int lm, int e) {
  int L = 0;
  while ((1 << L) < N) L++;
  if ((1 << L) != N || N < 2 || q < 2 || q > ORC_QMAX) return -1;
  if (s < 0) s = 3;
  if (s > L / 2) s = L / 2;
  if (lm < 0) lm = L / 2;
  if (lm < s || lm > L - s) return -1;
  if ((1L << (2 * s)) > ORC_MMAX) return -1;
  if (e < 0 || e > 4) return -1;
  bf->ph.id = phase_id;
  bf->ph.N = N;
  for (int i = 0; i < 4; i++) bf->ph.prm[i] = prm[i];
  bf->N = N;
  bf->L = L;
  bf->q = q;
  bf->s = s;
  bf->l0 = s;
  bf->lm = lm;
  bf->l1 = L - s;
  bf->e = e;
  orc_cheb(q, bf->z);
  int q2 = q * q;
  bf->lag2 = malloc(sizeof(double) * 4 * q2 * q2);
  for (int c = 0; c < 4; c++) {
    int s1 = c >> 1, s2 = c & 1;
    for (int t = 0; t < q2; t++)
      for (int u = 0; u < q2; u++) {
        double y1 = (2 * s1 - 1) / 4.0 + bf->z[u / q] / 2.0;
        double y2 = (2 * s2 - 1) / 4.0 + bf->z[u % q] / 2.0;
        bf->lag2[((long)c * q2 + t) * q2 + u] = orc_lagrange(q, bf->z, t / q, y1) * orc_lagrange(q, bf->z, t % q, y2);
      }
  }
  bf->p1 = malloc(sizeof(double) * N * N);
  bf->p2 = malloc(sizeof(double) * N * N);
  for (int a = 0; a < N; a++)
    for (int b = 0; b < N; b++) orc_polar(N, a - N / 2, b - N / 2, &bf->p1[a * N + b], &bf->p2[a * N + b]);
  return 0;
}

static void orc_bf_free(orc_bf *bf) {
  free(bf->lag2);
  free(bf->p1);
  free(bf->p2);
}

/* Box geometry.  A box of T_X at level j with index (i1,i2) has width 2^-j
 * and centre ((i1+1/2) 2^-j, (i2+1/2) 2^-j); its Chebyshev node t is
 * centre + width (z_{t1}, z_{t2}) (Sec. 3.2).  A box of T_P at level j is the
 * same in p1 and has width 2^-(j+e) in p2 (reading R4). */
static double orc_ctr(int j, int i) { return (i + 0.5) / (double)(1 << j); }
static double orc_node(const orc_bf *bf, int j, int i, int t) { return orc_ctr(j, i) + bf->z[t] / (double)(1 << j); }
static double orc_pctr2(const orc_bf *bf, int j, int i) { return orc_ctr(j + bf->e, i); }
static double orc_pnode2(const orc_bf *bf, int j, int i, int t) { return orc_node(bf, j + bf->e, i, t); }

static int orc_box(double p, int j) {
  int n = 1 << j;
  int b = (int)floor(p * n);
  return b > n - 1 ? n - 1 : b;
}

/* State at a level l: pairs (A,B), A at level l of T_X, B at level L-l of T_P,
 * each with q^2 coefficients.  Index (((a1*nA + a2)*nB + b1)*nB2 + b2)*q^2 + t,
 * nA = 2^l, nB = 2^{L-l}, nB2 = 2^{L-l+e}, t = t1*q + t2. */
static long orc_idx(const orc_bf *bf, int l, int a1, int a2, int b1, int b2, int t) {
  long nA = 1L << l, nB = 1L << (bf->L - l), nB2 = nB << bf->e;
  return (((a1 * nA + a2) * nB + b1) * nB2 + b2) * (long)(bf->q * bf->q) + t;
}

/* Step 2, Initialization (eq. alg2a), with A at level l0 and B at level L-l0:
 * delta^{AB}_t = e^{-2 pi i theta(x0(A),p^B_t)} sum_{p in B} L^B_t(p) e^{2 pi i theta(x0(A),p)} f(p). */
static void orc_step_init(const orc_bf *bf, const double complex *f, double complex *st) {
  int N = bf->N, q = bf->q, q2 = q * q, lb = bf->L - bf->l0;
  int nA = 1 << bf->l0, nB = 1 << lb;
  long nsrc = (long)N * N;
  /* sources bucketed by their box B at level L-l0 */
  long nB2 = (long)nB << bf->e;
  long *cnt = calloc((size_t)(nB * nB2 + 1), sizeof(long));
  long *lst = malloc(sizeof(long) * nsrc);
  for (long k = 0; k < nsrc; k++) cnt[orc_box(bf->p1[k], lb) * nB2 + orc_box(bf->p2[k], lb + bf->e) + 1]++;
  for (long b = 0; b < nB * nB2; b++) cnt[b + 1] += cnt[b];
  long *pos = malloc(sizeof(long) * nB * nB2);
  memcpy(pos, cnt, sizeof(long) * nB * nB2);
  for (long k = 0; k < nsrc; k++) lst[pos[orc_box(bf->p1[k], lb) * nB2 + orc_box(bf->p2[k], lb + bf->e)]++] = k;
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
  for (int a1 = 0; a1 < nA; a1++)
    for (int a2 = 0; a2 < nA; a2++) {
      double x1 = orc_ctr(bf->l0, a1), x2 = orc_ctr(bf->l0, a2);
      double w1[ORC_QMAX], w2[ORC_QMAX];
      for (int b1 = 0; b1 < nB; b1++)
        for (int b2 = 0; b2 < (nB << bf->e); b2++) {
          double complex acc[ORC_QMAX * ORC_QMAX];
          for (int t = 0; t < q2; t++) acc[t] = 0;
          long bb = (long)b1 * nB2 + b2;
          for (long j = cnt[bb]; j < cnt[bb + 1]; j++) {
            long k = lst[j];
            int k1 = (int)(k / N) - N / 2, k2 = (int)(k % N) - N / 2;
            double h1 = (bf->p1[k] - orc_ctr(lb, b1)) * (1 << lb);
            double h2 = (bf->p2[k] - orc_pctr2(bf, lb, b2)) * (1 << (lb + bf->e));
            for (int i = 0; i < q; i++) {
              w1[i] = orc_lagrange(q, bf->z, i, h1);
              w2[i] = orc_lagrange(q, bf->z, i, h2);
            }
            double complex v = orc_expi(orc_theta_k(&bf->ph, x1, x2, k1, k2)) * f[k];
            for (int t = 0; t < q2; t++) acc[t] += w1[t / q] * w2[t % q] * v;
          }
          for (int t = 0; t < q2; t++) {
            double pt1 = orc_node(bf, lb, b1, t / q), pt2 = orc_pnode2(bf, lb, b2, t % q);
            st[orc_idx(bf, bf->l0, a1, a2, b1, b2, t)] = conj(orc_expi(orc_theta(&bf->ph, x1, x2, pt1, pt2))) * acc[t];
          }
        }
    }
  free(cnt);
  free(lst);
  free(pos);
}

/* Step 3, Recursion in p (eq. alg2b), level l-1 -> l:
 * delta^{AB}_t = e^{-2 pi i theta(x0(A),p^B_t)} sum_c sum_t' L^B_t(p^{Bc}_t') e^{2 pi i theta(x0(A),p^{Bc}_t')} delta^{Ap Bc}_t'. */
static void orc_step_p(const orc_bf *bf, int l, const double complex *in, double complex *out) {
  int q = bf->q, q2 = q * q, lb = bf->L - l;
  int nA = 1 << l, nB = 1 << lb;
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
  for (int a1 = 0; a1 < nA; a1++)
    for (int a2 = 0; a2 < nA; a2++) {
      double x1 = orc_ctr(l, a1), x2 = orc_ctr(l, a2);
      double complex src[4 * ORC_QMAX * ORC_QMAX];
      for (int b1 = 0; b1 < nB; b1++)
        for (int b2 = 0; b2 < (nB << bf->e); b2++) {
          for (int c = 0; c < 4; c++) {
            int c1 = 2 * b1 + (c >> 1), c2 = 2 * b2 + (c & 1);
            for (int u = 0; u < q2; u++) {
              double pc1 = orc_node(bf, lb + 1, c1, u / q), pc2 = orc_pnode2(bf, lb + 1, c2, u % q);
              src[c * q2 + u] = orc_expi(orc_theta(&bf->ph, x1, x2, pc1, pc2)) *
                                in[orc_idx(bf, l - 1, a1 / 2, a2 / 2, c1, c2, u)];
            }
          }
          for (int t = 0; t < q2; t++) {
            double complex acc = 0;
            for (int c = 0; c < 4; c++)
              for (int u = 0; u < q2; u++) acc += bf->lag2[((long)c * q2 + t) * q2 + u] * src[c * q2 + u];
            double pt1 = orc_node(bf, lb, b1, t / q), pt2 = orc_pnode2(bf, lb, b2, t % q);
            out[orc_idx(bf, l, a1, a2, b1, b2, t)] = conj(orc_expi(orc_theta(&bf->ph, x1, x2, pt1, pt2))) * acc;
          }
        }
    }
}

/* Step 4, Switch (eq. alg2m) at level lm: delta^{AB}_t <- sum_s e^{2 pi i theta(x^A_t,p^B_s)} delta^{AB}_s. */
static void orc_step_switch(const orc_bf *bf, const double complex *in, double complex *out) {
  int q = bf->q, q2 = q * q, l = bf->lm, lb = bf->L - l;
  int nA = 1 << l, nB = 1 << lb;
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
  for (int a1 = 0; a1 < nA; a1++)
    for (int a2 = 0; a2 < nA; a2++)
      for (int b1 = 0; b1 < nB; b1++)
        for (int b2 = 0; b2 < (nB << bf->e); b2++)
          for (int t = 0; t < q2; t++) {
            double xt1 = orc_node(bf, l, a1, t / q), xt2 = orc_node(bf, l, a2, t % q);
            double complex acc = 0;
            for (int u = 0; u < q2; u++) {
              double ps1 = orc_node(bf, lb, b1, u / q), ps2 = orc_pnode2(bf, lb, b2, u % q);
              acc += orc_expi(orc_theta(&bf->ph, xt1, xt2, ps1, ps2)) * in[orc_idx(bf, l, a1, a2, b1, b2, u)];
            }
            out[orc_idx(bf, l, a1, a2, b1, b2, t)] = acc;
          }
}

/* Step 5, Recursion in x (eq. alg2c), level l-1 -> l:
 * delta^{AB}_t = sum_c e^{2 pi i theta(x^A_t,p0(Bc))} sum_t' L^{Ap}_t'(x^A_t) e^{-2 pi i theta(x^{Ap}_t',p0(Bc))} delta^{Ap Bc}_t'. */
static void orc_step_x(const orc_bf *bf, int l, const double complex *in, double complex *out) {
  int q = bf->q, q2 = q * q, lb = bf->L - l;
  int nA = 1 << l, nB = 1 << lb;
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
  for (int a1 = 0; a1 < nA; a1++)
    for (int a2 = 0; a2 < nA; a2++) {
      int ap1 = a1 / 2, ap2 = a2 / 2, sg = 2 * (a1 & 1) + (a2 & 1);
      double complex src[4 * ORC_QMAX * ORC_QMAX];
      for (int b1 = 0; b1 < nB; b1++)
        for (int b2 = 0; b2 < (nB << bf->e); b2++) {
          /* e^{-2 pi i theta(x^{Ap}_t',p0(Bc))} delta^{Ap Bc}_t' for the four children Bc */
          for (int c = 0; c < 4; c++) {
            int c1 = 2 * b1 + (c >> 1), c2 = 2 * b2 + (c & 1);
            double pc1 = orc_ctr(lb + 1, c1), pc2 = orc_pctr2(bf, lb + 1, c2);
            for (int u = 0; u < q2; u++) {
              double xp1 = orc_node(bf, l - 1, ap1, u / q), xp2 = orc_node(bf, l - 1, ap2, u % q);
              src[c * q2 + u] = conj(orc_expi(orc_theta(&bf->ph, xp1, xp2, pc1, pc2))) *
                                in[orc_idx(bf, l - 1, ap1, ap2, c1, c2, u)];
            }
          }
          for (int t = 0; t < q2; t++) {
            double xt1 = orc_node(bf, l, a1, t / q), xt2 = orc_node(bf, l, a2, t % q);
            double complex acc = 0;
            for (int c = 0; c < 4; c++) {
              int c1 = 2 * b1 + (c >> 1), c2 = 2 * b2 + (c & 1);
              double pc1 = orc_ctr(lb + 1, c1), pc2 = orc_pctr2(bf, lb + 1, c2);
              double complex part = 0;
              /* L^{Ap}_t'(x^A_t): parent polynomial t' at the child node t */
              for (int u = 0; u < q2; u++) part += bf->lag2[((long)sg * q2 + u) * q2 + t] * src[c * q2 + u];
              acc += orc_expi(orc_theta(&bf->ph, xt1, xt2, pc1, pc2)) * part;
            }
            out[orc_idx(bf, l, a1, a2, b1, b2, t)] = acc;
          }
        }
    }
}

/* Step 6, Termination (eq. alg2d) with A at level l1 and the 4^s boxes B at
 * level s: u(x) = sum_B e^{2 pi i theta(x,p0(B))} sum_t L^A_t(x) e^{-2 pi i theta(x^A_t,p0(B))} delta^{AB}_t. */
static void orc_step_term(const orc_bf *bf, const double complex *st, double complex *u) {
  int N = bf->N, q = bf->q, q2 = q * q, l = bf->l1, lb = bf->L - l;
  int nA = 1 << l, nB = 1 << lb, m = N / nA;
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
  for (int a1 = 0; a1 < nA; a1++)
    for (int a2 = 0; a2 < nA; a2++) {
      double complex src[ORC_QMAX * ORC_QMAX];
      for (int m1 = 0; m1 < m; m1++)
        for (int m2 = 0; m2 < m; m2++) u[(long)(a1 * m + m1) * N + a2 * m + m2] = 0;
      for (int b1 = 0; b1 < nB; b1++)
        for (int b2 = 0; b2 < (nB << bf->e); b2++) {
          double p01 = orc_ctr(lb, b1), p02 = orc_pctr2(bf, lb, b2);
          for (int t = 0; t < q2; t++) {
            double xt1 = orc_node(bf, l, a1, t / q), xt2 = orc_node(bf, l, a2, t % q);
            src[t] = conj(orc_expi(orc_theta(&bf->ph, xt1, xt2, p01, p02))) * st[orc_idx(bf, l, a1, a2, b1, b2, t)];
          }
          for (int m1 = 0; m1 < m; m1++)
            for (int m2 = 0; m2 < m; m2++) {
              int i1 = a1 * m + m1, i2 = a2 * m + m2;
              double x1 = (double)i1 / N, x2 = (double)i2 / N;
              double h1 = (x1 - orc_ctr(l, a1)) * nA, h2 = (x2 - orc_ctr(l, a2)) * nA;
              double complex part = 0;
              for (int t = 0; t < q2; t++)
                part += orc_lagrange(q, bf->z, t / q, h1) * orc_lagrange(q, bf->z, t % q, h2) * src[t];
              u[(long)i1 * N + i2] += orc_expi(orc_theta(&bf->ph, x1, x2, p01, p02)) * part;
            }
        }
    }
}

/* ---------------------------------------------------- adjoint butterfly */

/* Conjugate transpose of the termination: for every A at level l1 and B at level s,
 * d_t = e^{2 pi i theta(x^A_t,p0B)} sum_{x in A} L^A_t(x) e^{-2 pi i theta(x,p0B)} g(x). */
static void orc_adj_term(const orc_bf *bf, const double complex *g, double complex *st) {
  int N = bf->N, q = bf->q, q2 = q * q, l = bf->l1, lb = bf->L - l;
  int nA = 1 << l, nB = 1 << lb, m = N / nA;
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
  for (int a1 = 0; a1 < nA; a1++)
    for (int a2 = 0; a2 < nA; a2++) {
      double complex v[ORC_MMAX];
      for (int b1 = 0; b1 < nB; b1++)
        for (int b2 = 0; b2 < (nB << bf->e); b2++) {
          double p01 = orc_ctr(lb, b1), p02 = orc_pctr2(bf, lb, b2);
          /* e^{-2 pi i theta(x,p0B)} g(x) for the grid points x of A */
          for (int m1 = 0; m1 < m; m1++)
            for (int m2 = 0; m2 < m; m2++) {
              int i1 = a1 * m + m1, i2 = a2 * m + m2;
              v[m1 * m + m2] = conj(orc_expi(orc_theta(&bf->ph, (double)i1 / N, (double)i2 / N, p01, p02))) *
                               g[(long)i1 * N + i2];
            }
          for (int t = 0; t < q2; t++) {
            double complex acc = 0;
            for (int m1 = 0; m1 < m; m1++)
              for (int m2 = 0; m2 < m; m2++) {
                double h1 = ((double)(a1 * m + m1) / N - orc_ctr(l, a1)) * nA;
                double h2 = ((double)(a2 * m + m2) / N - orc_ctr(l, a2)) * nA;
                acc += orc_lagrange(q, bf->z, t / q, h1) * orc_lagrange(q, bf->z, t % q, h2) * v[m1 * m + m2];
              }
            double xt1 = orc_node(bf, l, a1, t / q), xt2 = orc_node(bf, l, a2, t % q);
            st[orc_idx(bf, l, a1, a2, b1, b2, t)] = orc_expi(orc_theta(&bf->ph, xt1, xt2, p01, p02)) * acc;
          }
        }
    }
}

/* Conjugate transpose of the x-recursion at level l (l -> l-1):
 * d^{Ap Bc}_u = e^{2 pi i theta(x^{Ap}_u,p0Bc)} sum_{A in Ap} sum_t L^{Ap}_u(x^A_t) e^{-2 pi i theta(x^A_t,p0Bc)} d^{AB}_t. */
static void orc_adj_x(const orc_bf *bf, int l, const double complex *in, double complex *out) {
  int q = bf->q, q2 = q * q, lb = bf->L - l;
  int nAp = 1 << (l - 1), nBc = 1 << (lb + 1);
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
  for (int ap1 = 0; ap1 < nAp; ap1++)
    for (int ap2 = 0; ap2 < nAp; ap2++) {
      double complex v[4 * ORC_QMAX * ORC_QMAX];
      for (int c1 = 0; c1 < nBc; c1++)
        for (int c2 = 0; c2 < (nBc << bf->e); c2++) {
          int b1 = c1 / 2, b2 = c2 / 2;
          double pc1 = orc_ctr(lb + 1, c1), pc2 = orc_pctr2(bf, lb + 1, c2);
          /* e^{-2 pi i theta(x^A_t,p0Bc)} d^{AB}_t for the four children A of Ap */
          for (int sg = 0; sg < 4; sg++) {
            int a1 = 2 * ap1 + (sg >> 1), a2 = 2 * ap2 + (sg & 1);
            for (int t = 0; t < q2; t++) {
              double xt1 = orc_node(bf, l, a1, t / q), xt2 = orc_node(bf, l, a2, t % q);
              v[sg * q2 + t] = conj(orc_expi(orc_theta(&bf->ph, xt1, xt2, pc1, pc2))) *
                               in[orc_idx(bf, l, a1, a2, b1, b2, t)];
            }
          }
          for (int u = 0; u < q2; u++) {
            double complex acc = 0;
            for (int sg = 0; sg < 4; sg++)
              for (int t = 0; t < q2; t++) acc += bf->lag2[((long)sg * q2 + u) * q2 + t] * v[sg * q2 + t];
            double xp1 = orc_node(bf, l - 1, ap1, u / q), xp2 = orc_node(bf, l - 1, ap2, u % q);
            out[orc_idx(bf, l - 1, ap1, ap2, c1, c2, u)] = orc_expi(orc_theta(&bf->ph, xp1, xp2, pc1, pc2)) * acc;
          }
        }
    }
}

/* Conjugate transpose of the switch: d_s = sum_t e^{-2 pi i theta(x^A_t,p^B_s)} d_t. */
static void orc_adj_switch(const orc_bf *bf, const double complex *in, double complex *out) {
  int q = bf->q, q2 = q * q, l = bf->lm, lb = bf->L - l;
  int nA = 1 << l, nB = 1 << lb;
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
  for (int a1 = 0; a1 < nA; a1++)
    for (int a2 = 0; a2 < nA; a2++)
      for (int b1 = 0; b1 < nB; b1++)
        for (int b2 = 0; b2 < (nB << bf->e); b2++)
          for (int u = 0; u < q2; u++) {
            double ps1 = orc_node(bf, lb, b1, u / q), ps2 = orc_pnode2(bf, lb, b2, u % q);
            double complex acc = 0;
            for (int t = 0; t < q2; t++) {
              double xt1 = orc_node(bf, l, a1, t / q), xt2 = orc_node(bf, l, a2, t % q);
              acc += conj(orc_expi(orc_theta(&bf->ph, xt1, xt2, ps1, ps2))) * in[orc_idx(bf, l, a1, a2, b1, b2, t)];
            }
            out[orc_idx(bf, l, a1, a2, b1, b2, u)] = acc;
          }
}

/* Conjugate transpose of the p-recursion at level l (l -> l-1):
 * d^{Ap Bc}_u = sum_{A in Ap} e^{-2 pi i theta(x0A,p^{Bc}_u)} sum_t L^B_t(p^{Bc}_u) e^{2 pi i theta(x0A,p^B_t)} d^{AB}_t. */
static void orc_adj_p(const orc_bf *bf, int l, const double complex *in, double complex *out) {
  int q = bf->q, q2 = q * q, lb = bf->L - l;
  int nAp = 1 << (l - 1), nB = 1 << lb;
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
  for (int ap1 = 0; ap1 < nAp; ap1++)
    for (int ap2 = 0; ap2 < nAp; ap2++) {
      double complex v[4 * ORC_QMAX * ORC_QMAX];
      for (int b1 = 0; b1 < nB; b1++)
        for (int b2 = 0; b2 < (nB << bf->e); b2++) {
          /* e^{2 pi i theta(x0A,p^B_t)} d^{AB}_t for the four children A of Ap */
          for (int sg = 0; sg < 4; sg++) {
            int a1 = 2 * ap1 + (sg >> 1), a2 = 2 * ap2 + (sg & 1);
            double x1 = orc_ctr(l, a1), x2 = orc_ctr(l, a2);
            for (int t = 0; t < q2; t++) {
              double pt1 = orc_node(bf, lb, b1, t / q), pt2 = orc_pnode2(bf, lb, b2, t % q);
              v[sg * q2 + t] = orc_expi(orc_theta(&bf->ph, x1, x2, pt1, pt2)) * in[orc_idx(bf, l, a1, a2, b1, b2, t)];
            }
          }
          for (int c = 0; c < 4; c++) {
            int c1 = 2 * b1 + (c >> 1), c2 = 2 * b2 + (c & 1);
            for (int u = 0; u < q2; u++) {
              double pc1 = orc_node(bf, lb + 1, c1, u / q), pc2 = orc_pnode2(bf, lb + 1, c2, u % q);
              double complex acc = 0;
              for (int sg = 0; sg < 4; sg++) {
                int a1 = 2 * ap1 + (sg >> 1), a2 = 2 * ap2 + (sg & 1);
                double x1 = orc_ctr(l, a1), x2 = orc_ctr(l, a2);
                double complex part = 0;
                /* L^B_t(p^{Bc}_u) */
                for (int t = 0; t < q2; t++) part += bf->lag2[((long)c * q2 + t) * q2 + u] * v[sg * q2 + t];
                acc += conj(orc_expi(orc_theta(&bf->ph, x1, x2, pc1, pc2))) * part;
              }
              out[orc_idx(bf, l - 1, ap1, ap2, c1, c2, u)] = acc;
            }
          }
        }
    }
}

/* Conjugate transpose of the initialization:
 * fbar(k) = sum_{A at l0} e^{-2 pi i theta(x0A,p(k))} sum_t L^B_t(p(k)) e^{2 pi i theta(x0A,p^B_t)} d^{AB}_t,
 * B the box of p(k) at level L-l0. */
static void orc_adj_init(const orc_bf *bf, const double complex *st, double complex *fbar) {
  int N = bf->N, q = bf->q, q2 = q * q, lb = bf->L - bf->l0;
  int nA = 1 << bf->l0, nB = 1 << lb;
  /* v^{AB}_t = e^{2 pi i theta(x0A,p^B_t)} d^{AB}_t */
  double complex *v = malloc(sizeof(double complex) * ((long)N * N * q2 << bf->e));
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
  for (int a1 = 0; a1 < nA; a1++)
    for (int a2 = 0; a2 < nA; a2++)
      for (int b1 = 0; b1 < nB; b1++)
        for (int b2 = 0; b2 < (nB << bf->e); b2++)
          for (int t = 0; t < q2; t++) {
            double pt1 = orc_node(bf, lb, b1, t / q), pt2 = orc_pnode2(bf, lb, b2, t % q);
            long i = orc_idx(bf, bf->l0, a1, a2, b1, b2, t);
            v[i] = orc_expi(orc_theta(&bf->ph, orc_ctr(bf->l0, a1), orc_ctr(bf->l0, a2), pt1, pt2)) * st[i];
          }
#pragma omp parallel for schedule(dynamic, 16)
  for (long k = 0; k < (long)N * N; k++) {
    int k1 = (int)(k / N) - N / 2, k2 = (int)(k % N) - N / 2;
    int b1 = orc_box(bf->p1[k], lb), b2 = orc_box(bf->p2[k], lb + bf->e);
    double h1 = (bf->p1[k] - orc_ctr(lb, b1)) * (1 << lb);
    double h2 = (bf->p2[k] - orc_pctr2(bf, lb, b2)) * (1 << (lb + bf->e));
    double w1[ORC_QMAX], w2[ORC_QMAX];
    for (int i = 0; i < q; i++) {
      w1[i] = orc_lagrange(q, bf->z, i, h1);
      w2[i] = orc_lagrange(q, bf->z, i, h2);
    }
    double complex acc = 0;
    for (int a1 = 0; a1 < nA; a1++)
      for (int a2 = 0; a2 < nA; a2++) {
        double complex part = 0;
        for (int t = 0; t < q2; t++) part += w1[t / q] * w2[t % q] * v[orc_idx(bf, bf->l0, a1, a2, b1, b2, t)];
        acc += conj(orc_expi(orc_theta_k(&bf->ph, orc_ctr(bf->l0, a1), orc_ctr(bf->l0, a2), k1, k2))) * part;
      }
    fbar[k] = acc;
  }
  free(v);
}

/* --------------------------------------------------- exported butterfly */

/* Number of state snapshots ("stages") one butterfly produces:
 * init, one per p-level, the switch, one per x-level. */
int orc_num_stages(int N, int s, int lm) {
  int L = 0;
  while ((1 << L) < N) L++;
  if (s < 0) s = 3;
  if (s > L / 2) s = L / 2;
  if (lm < 0) lm = L / 2;
  return (lm - s) + 1 + 1 + (L - s - lm);
}

/* Level of the pairs (A's level) held after stage j. */
int orc_stage_level(int N, int s, int lm, int j) {
  int L = 0;
  while ((1 << L) < N) L++;
  if (s < 0) s = 3;
  if (s > L / 2) s = L / 2;
  if (lm < 0) lm = L / 2;
  if (j <= lm - s) return s + j;
  if (j == lm - s + 1) return lm;
  return lm + (j - (lm - s + 1));
}

/*
 * Forward butterfly (Sec. 4 with the Sec. 5 truncation).  f, u: N x N complex
 * (layout of orc_direct).  If stage >= 0, the state after that stage is copied
 * to snap (2^e N^2 q^2 complex, layout of orc_idx) and the rest still runs.
 * Returns 0, or -1 on bad arguments.
 */
int orc_butterfly(int N, int q, int phase_id, const double *prm, int s, int lm, int e, const double complex *f,
                  double complex *u, int stage, double complex *snap) {
  orc_bf bf;
  if (orc_bf_init(&bf, N, q, phase_id, prm, s, lm, e)) return -1;
  long sz = (long)N * N * q * q << bf.e;
  double complex *a = malloc(sizeof(double complex) * sz), *b = malloc(sizeof(double complex) * sz);
  int j = 0;
  orc_step_init(&bf, f, a);
  if (stage == j) memcpy(snap, a, sizeof(double complex) * sz);
  for (int l = bf.l0 + 1; l <= bf.lm; l++) {
    orc_step_p(&bf, l, a, b);
    double complex *t = a; a = b; b = t;
    if (stage == ++j) memcpy(snap, a, sizeof(double complex) * sz);
  }
  orc_step_switch(&bf, a, b);
  { double complex *t = a; a = b; b = t; }
  if (stage == ++j) memcpy(snap, a, sizeof(double complex) * sz);
  for (int l = bf.lm + 1; l <= bf.l1; l++) {
    orc_step_x(&bf, l, a, b);
    double complex *t = a; a = b; b = t;
    if (stage == ++j) memcpy(snap, a, sizeof(double complex) * sz);
  }
  orc_step_term(&bf, a, u);
  free(a);
  free(b);
  orc_bf_free(&bf);
  return 0;
}

/* Adjoint butterfly: fbar = B^H g, the exact conjugate transpose of orc_butterfly. */
int orc_butterfly_adjoint(int N, int q, int phase_id, const double *prm, int s, int lm, int e,
                          const double complex *g, double complex *fbar) {
  orc_bf bf;
  if (orc_bf_init(&bf, N, q, phase_id, prm, s, lm, e)) return -1;
  long sz = (long)N * N * q * q << bf.e;
  double complex *a = malloc(sizeof(double complex) * sz), *b = malloc(sizeof(double complex) * sz);
  orc_adj_term(&bf, g, a);
  for (int l = bf.l1; l >= bf.lm + 1; l--) {
    orc_adj_x(&bf, l, a, b);
    double complex *t = a; a = b; b = t;
  }
  orc_adj_switch(&bf, a, b);
  { double complex *t = a; a = b; b = t; }
  for (int l = bf.lm; l >= bf.l0 + 1; l--) {
    orc_adj_p(&bf, l, a, b);
    double complex *t = a; a = b; b = t;
  }
  orc_adj_init(&bf, a, fbar);
  free(a);
  free(b);
  orc_bf_free(&bf);
  return 0;
}
