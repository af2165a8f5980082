/*
 * fio3.h -- C ABI of the three-dimensional butterfly FIO apply (Candes, Demanet &
 * Ying, "A Fast Butterfly Algorithm for the Computation of Fourier Integral
 * Operators", 2008, Sec. 5 and Table 3: the algorithm carried over to three
 * dimensions with a three-dimensional Chebyshev grid, shown for eq. ex3).
 *
 *   u(x) = sum_{k in Omega} e^{2 pi i Phi(x,k)} f(k),  x in X = {0..N-1}^3 / N,
 *   Omega = {-N/2 .. N/2-1}^3.
 *
 * The paper gives no three-dimensional formulas; this library takes the
 * following readings (the same as the test oracle's):
 *   - spherical coordinates in frequency, the analogue of the polar map of
 *     Sec. 1.1: k = (sqrt3/2) N p1 (sin pi p2 cos 2 pi p3, sin pi p2 sin 2 pi p3,
 *     cos pi p2), p1 = 2|k|/(sqrt3 N), p2 = polar angle / pi, p3 = azimuth / 2 pi in
 *     [0,1); k = 0 maps to p = 0;
 *   - a box of T_P at level j is 2^-j wide in p1 and 2^-(j+e) in p2 and p3 (angular
 *     refinement e); a box of T_X at level j is a cube of side 2^-j; box index at
 *     level j: min(floor(p 2^j), 2^j - 1);
 *   - balanced levels (A at level l paired with B at level L-l), initialization with
 *     A at level s, switch at floor(L/2), termination summing the boxes B at level s;
 *     every translation and the termination use the q^3 tensor-product Chebyshev grid
 *     with Lagrange interpolation applied one dimension at a time.
 * fio3_apply_adjoint applies the exact conjugate transpose of that discrete
 * butterfly.  Arithmetic: FP64 throughout (this is the FP64 form only).
 *
 * Data layout (row-major, interleaved complex128; a torch tensor of shape
 * (nrhs, N, N, N)):
 *   f, fbar : element (r, k1+N/2, k2+N/2, k3+N/2) is the source of RHS r at k
 *   u, g    : element (r, i1, i2, i3) is the potential of RHS r at x = (i1, i2, i3)/N
 * Ownership and errors as in fio.h: data pointers belong to the caller (DEVICE
 * pointers, 16-byte aligned); a plan owns its tables and two state buffers;
 * every call returns FIO_OK (0) or a negative FIO_* status and sets
 * fio_last_error(); nothing falls back to a CPU computation.
 */
#ifndef FIO3_H_
#define FIO3_H_

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fio3_plan_s *fio3_plan_t;

/* Phases: FIO3_PHASE_LINEAR Phi = x.k (no params); FIO3_PHASE_SPHERE
 * Phi = lambda x.k + c(x)|k|, c(x) = (a + m sin 2pi x1 sin 2pi x2 sin 2pi x3)/b,
 * params [a, m, b, lambda] (eq. ex3 is [3, 1, 4, 1]). */
enum { FIO3_PHASE_LINEAR = 0, FIO3_PHASE_SPHERE = 2 };

/*
 * fio3_plan -- build a plan for N x N x N grids (host work in FP64, then one upload).
 *   N         power of two, 4 <= N <= 256
 *   q         Chebyshev points per dimension: 3, 5 or 7
 *   phase_id  FIO3_PHASE_*; params/nparams: 0 (LINEAR) or 4 doubles (SPHERE)
 *   nrhs_max  largest nrhs later passed to fio3_apply* (>= 1)
 *   s         truncation depth (-1 = 3), clipped to floor(L/2); 2^s <= 8
 *   e         angular refinement, 0..3 (-1 = 1)
 * Allocates the tables and two state buffers of N^3 4^e q^3 nrhs_max complex128
 * each on the current device.  FIO_EINVAL for bad arguments, FIO_ENOMEM when the
 * state does not fit, FIO_EDEVICE without a device.
 */
int fio3_plan(fio3_plan_t *out, int N, int q, int phase_id, const double *params, int nparams, int nrhs_max, int s,
              int e);

/* fio3_destroy -- free a plan (waits for the device). NULL is a no-op. */
int fio3_destroy(fio3_plan_t plan);

/* fio3_apply -- u = B f for nrhs right-hand sides; fio3_apply_adjoint -- fbar = B^H g.
 * DEVICE pointers, layout above, 1 <= nrhs <= nrhs_max; input and output must not
 * overlap.  Enqueued on `stream` (cudaStream_t as void*, NULL = default stream). */
int fio3_apply(fio3_plan_t plan, const void *f, void *u, int nrhs, void *stream);
int fio3_apply_adjoint(fio3_plan_t plan, const void *g, void *fbar, int nrhs, void *stream);

typedef struct {
  int N, L, q, s, e, l0, lm, l1, phase_id, nrhs_max;
  long long pairs_per_level; /* N^3 4^e */
  long long state_bytes;     /* the two state buffers */
  long long table_bytes;
  int max_box_sources;
} fio3_plan_info_t;
int fio3_plan_info(fio3_plan_t plan, fio3_plan_info_t *info);

#ifdef __cplusplus
}
#endif

#endif /* FIO3_H_ */
